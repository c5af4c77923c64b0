"""The allocation-free product against the allocating one and the FP64 oracle (collected last on
purpose, so that a failure here leaves every other test already run).

lgp_kernel_matvec_noalloc serves callers that cannot allocate device memory: programs whose
device memory belongs to another allocator, services under a fixed memory budget, and
latency-critical loops where cudaMalloc/cudaFree could synchronise the device. It uses a fixed
scratch array inside the library instead of a context workspace. Two calls in a row, with
different shapes, must each match lgp_kernel_matvec and the FP64 oracle within the product
tolerance, the status words must read back clean, and a repeated call must not change the
device's free memory.
"""
import numpy as np
import pytest

from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _colerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


def test_noalloc_matches_allocating_entry_and_oracle_on_two_calls(lgp):
    import torch
    cases = [(wl.random_problem(8000, 5, wl.MATERN52, seed=101), 32),
             (wl.random_problem(3001, 2, wl.RBF, seed=102), 16)]
    for p, t in cases:
        Vh = wl.rhs_block(p.N, t, seed=t)
        X = torch.as_tensor(p.X, device="cuda")
        V = torch.as_tensor(Vh, device="cuda")
        out = torch.full((p.N, t), float("nan"), device="cuda")
        s = lgp.lgp_kernel_matvec_noalloc(X, p, V, out)
        assert s == lgp.LGP_OK
        assert lgp.lgp_kernel_matvec_noalloc_status() == lgp.LGP_OK
        ref = lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _colerr(got, ref.cpu().numpy()) <= TOL
        assert _colerr(got, go.matvec(p.X, Vh, go.hyper_of(p))) <= TOL


def test_noalloc_repeated_call_allocates_nothing(lgp):
    import torch
    p = wl.random_problem(6000, 4, wl.RBF, seed=103)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=3), device="cuda")
    out = torch.empty((p.N, 32), device="cuda")
    assert lgp.lgp_kernel_matvec_noalloc(X, p, V, out) == lgp.LGP_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lgp.lgp_kernel_matvec_noalloc(X, p, V, out) == lgp.LGP_OK
    assert lgp.lgp_kernel_matvec_noalloc_status() == lgp.LGP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_limit(lgp):
    import torch
    p = wl.random_problem(8193, 2, wl.RBF, seed=104)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.zeros((p.N, 32), device="cuda")
    out = torch.empty_like(V)
    assert lgp.lgp_kernel_matvec_noalloc(X, p, V, out) == lgp.LGP_ERR_UNSUPPORTED
    q = wl.random_problem(100, 2, wl.RBF, seed=105)
    Xq = torch.as_tensor(q.X, device="cuda")
    V8 = torch.zeros((100, 8), device="cuda")
    assert lgp.lgp_kernel_matvec_noalloc(Xq, q, V8, torch.empty_like(V8)) == lgp.LGP_ERR_UNSUPPORTED
