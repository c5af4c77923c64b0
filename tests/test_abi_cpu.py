"""Host-side checks that need no GPU: the library builds, loads and exports the C ABI."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lgp.h")


def _declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lgp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_17898_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for name in ["lgp_kernel_matvec", "lgp_kernel_matvec_grad", "lgp_cg_solve", "lgp_lml_and_grad",
                 "lgp_batch_cg_solve", "lgp_rademacher_probes", "lgp_create", "lgp_destroy"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    cdll, path = lib
    for name in _declared_symbols():
        assert hasattr(cdll, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lgp_[a-z_0-9]+)\b", nm))
    assert set(_declared_symbols()) <= exported


def test_binding_names_match_header():
    import paper_2605_17898_gb300 as pkg
    assert sorted(pkg.EXPORTED) == _declared_symbols()
    for name in ["lgp_kernel_matvec", "lgp_kernel_matvec_grad", "lgp_cg_solve", "lgp_lml_and_grad",
                 "lgp_rademacher_probes", "lgp_batch_cg_solve"]:
        assert callable(getattr(pkg, name))


def test_host_only_entry_points(lib):
    import paper_2605_17898_gb300 as pkg
    l = pkg.load()
    assert l.lgp_version() == 10000
    assert l.lgp_status_string(pkg.LGP_ERR_TIMEOUT).decode() == "LGP_ERR_TIMEOUT"
    assert l.lgp_status_string(12345).decode() == "LGP_UNKNOWN_STATUS"
    assert l.lgp_last_error_message(None).decode() == "no context"
    assert l.lgp_workspace_bytes(None) == 0
    assert l.lgp_create(None, 0) == pkg.LGP_ERR_INVALID_ARG


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2605_17898_gb300 as pkg
    h = ctypes.c_void_p()
    s = pkg.load().lgp_create(ctypes.byref(h), 0)
    assert s < 0 and not h.value


def test_struct_layouts_are_packed_as_in_c():
    import paper_2605_17898_gb300 as pkg
    assert ctypes.sizeof(pkg.lgp_hyper) == 24
    assert ctypes.sizeof(pkg.lgp_options) == 40
    assert ctypes.sizeof(pkg.lgp_lml_info) == 64
    assert ctypes.sizeof(pkg.lgp_predict_info) == 24


def test_workloads_shapes_and_dtypes():
    import workloads as wl
    p = wl.cfg1()
    assert p.X.shape == (1024, 2) and p.X.dtype == np.float32 and p.y.shape == (1024,)
    q = wl.cfg3(N=500)
    assert q.X.shape == (500, 8) and q.kind == wl.MATERN52
    np.testing.assert_allclose(np.exp(q.log_lengthscale)[[0, -1]], [0.3, 2.0], rtol=1e-6)
    gps = wl.cfg5_batch(n_gp=64)
    Ns = [g.N for g in gps]
    assert min(Ns) >= 500 and max(Ns) <= 30000
    assert {g.D for g in gps} <= set(range(1, 7))
    # same seed, same data
    np.testing.assert_array_equal(wl.cfg1().X, wl.cfg1().X)
