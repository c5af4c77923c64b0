"""Parity of the symmetric-tile tensor-core product (each 128 x 128 tile of the upper triangle
generated once and applied as K_IJ V_J and K_IJ^T V_I) with the FP64 oracle.

The kernel is forced with LGP_TC_SYMMETRIC=1 on fresh contexts. Gates as for the row kernel:
column relative error <= 1e-5 (scaled float16 halves), <= 1e-4 (bfloat16 halves). Sizes span
several tile rows, the diagonal tiles, tile-row boundaries inside one CTA's range, and ragged
tails (padding rows inside the last tile).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5
BF16_TOL = 1e-4


def _colerr(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


@pytest.fixture
def sym(lgp):
    os.environ["LGP_TC_SYMMETRIC"] = "1"
    ctx = lgp.Context(0)
    yield ctx
    ctx.close()
    os.environ.pop("LGP_TC_SYMMETRIC", None)


def _run(lgp, ctx, p, V, prec, out=None):
    import torch
    X = torch.as_tensor(p.X, device="cuda")
    Vt = torch.as_tensor(V, device="cuda")
    o = lgp.lgp_kernel_matvec(X, p, Vt, prec=prec, ctx=ctx, out=out)
    torch.cuda.synchronize()
    return o.cpu().numpy()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("t", [16, 32])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
@pytest.mark.parametrize("N", [769, 1000, 1025, 1500, 4099])  # 769: the last tile row is all padding
def test_symmetric_matvec(lgp, sym, kind, t, N, fmt):
    p = wl.random_problem(N, 3, kind, seed=N + t + 5)
    V = wl.rhs_block(N, t, seed=N + 1)
    prec = lgp.LGP_PREC_SPLIT_F16 if fmt == "f16" else lgp.LGP_PREC_SPLIT_BF16
    got = _run(lgp, sym, p, V, prec)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(got, ref).max()
    print(f"symmetric {fmt} kind={kind} t={t} N={N}: max column rel err {err:.2e}")
    assert err <= (TOL if fmt == "f16" else BF16_TOL)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7, 8])
def test_symmetric_every_dimension(lgp, sym, D):
    p = wl.random_problem(2100, D, wl.MATERN52 if D % 2 else wl.RBF, seed=140 + D)
    V = wl.rhs_block(p.N, 32, seed=D + 11)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max() <= TOL
    assert _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_BF16), ref).max() <= BF16_TOL


def test_symmetric_column_scaling_extremes(lgp, sym):
    p = wl.random_problem(3000, 4, wl.MATERN52, seed=78)
    V = wl.rhs_block(p.N, 16, seed=78)
    V[:, 1] *= 1e-20
    V[:, 2] *= 1e20
    V[:, 3] = 0.0
    V[:, 4] = np.abs(V[:, 4]) + 1e3
    got = _run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert np.all(got[:, 3] == 0.0)
    keep = [c for c in range(16) if c != 3]
    assert _colerr(got[:, keep], ref[:, keep]).max() <= TOL


def test_symmetric_unaligned_output_uses_scalar_reductions(lgp, sym):
    """An output whose rows are not 16-byte aligned takes the one-float reduction path."""
    import torch
    p = wl.random_problem(2500, 5, wl.RBF, seed=91)
    V = wl.rhs_block(p.N, 32, seed=91)
    buf = torch.zeros(p.N * 32 + 1, device="cuda", dtype=torch.float32)
    out = buf[1:].view(p.N, 32)
    assert out.data_ptr() % 16 != 0
    got = _run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16, out=out)
    assert buf[0].item() == 0.0
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(got, ref).max() <= TOL


def test_symmetric_full_size_cfg3_sampled_rows(lgp, sym):
    """N=100000, D=8, Matern-5/2, t=32: sampled rows against the C oracle."""
    p = wl.cfg3(t=32)
    V = wl.rhs_block(p.N, 32, seed=21, kind="sign")
    V[:, 0] = p.y
    got = _run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16)
    rows = np.random.default_rng(5).choice(p.N, 300, replace=False)
    rows[:3] = [0, p.N - 1, 99967]  # first row, last row, last row before the final tile
    ref, _ = oracle.kyv_rows_c(p.X, V, go.hyper_of(p), rows=rows)
    assert _colerr(got[rows], ref).max() <= TOL


@pytest.mark.parametrize("t", [16, 32])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_banded_tile_order(lgp, sym, kind, t):
    """LGP_TC_BANDS=1: the dot-form product walks the triangle in column bands (48 MiB of column-side
    operands each: 1228 tiles at t = 32, 2048 at t = 16), so N = 280000 (2188 tiles a side) takes two
    bands with a narrow second one. Sampled rows against the FP64 row oracle at the product gate, and
    the whole result against the single-band order (the two differ only in the order of the float32
    additions onto out). Lengthscales in [0.1, 0.3] keep the draw inside the dot form's gate and its
    cancellation (sum_j |k_ij v_j| over |(K v)_i|, below ~400 on sampled rows) below that of the
    N = 500000 workload, whose product meets the same gate."""
    import torch
    p = wl.random_problem(280000, 3, kind, seed=280 + t + kind, lo=0.1, hi=0.3)
    V = wl.rhs_block(p.N, t, seed=t)
    one = _run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16)
    os.environ["LGP_TC_BANDS"] = "1"
    try:
        banded = _run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16)
    finally:
        os.environ.pop("LGP_TC_BANDS", None)
    assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT
    rows = np.random.default_rng(3).choice(p.N, 96, replace=False)
    ref, _ = oracle.kyv_rows_c(p.X, V, go.hyper_of(p), rows=rows)
    err = _colerr(banded[rows], ref).max()
    diff = _colerr(banded, one.astype(np.float64)).max()
    print(f"banded kind={kind} t={t}: sampled-row err {err:.2e}, against the single-band order {diff:.2e}")
    assert err <= TOL
    assert diff <= TOL


def test_symmetric_agrees_with_row_kernel(lgp):
    """The two tensor-core kernels give the same product to the split error level, and repeated
    symmetric products agree to float32 summation-order level."""
    import torch
    p = wl.cfg3(N=7000, t=32)
    V = wl.rhs_block(p.N, 32, seed=12)
    outs = {}
    for flag in ["0", "1"]:
        os.environ["LGP_TC_SYMMETRIC"] = flag
        ctx = lgp.Context(0)
        outs[flag] = [_run(lgp, ctx, p, V, lgp.LGP_PREC_SPLIT_F16).astype(np.float64) for _ in range(2)]
        ctx.close()
    os.environ.pop("LGP_TC_SYMMETRIC", None)
    a, b = outs["0"][0], outs["1"][0]
    assert (np.linalg.norm(a - b, axis=0) / np.linalg.norm(a, axis=0)).max() <= TOL
    np.testing.assert_array_equal(outs["0"][0], outs["0"][1])  # the row kernel is deterministic
    c = outs["1"][1]
    assert (np.linalg.norm(c - b, axis=0) / np.linalg.norm(b, axis=0)).max() <= 1e-6


def test_kernel_choice_follows_the_switch_and_the_autotuner(lgp):
    """LGP_TC_SYMMETRIC=1 / 0 pin the kernel; with neither, the autotuner times both and keeps
    one (the choice is reported per shape, and is absent before the first product)."""
    import torch
    p = wl.cfg3(N=3000, t=32)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=1), device="cuda")
    for flag, want in [("1", [lgp.LGP_TC_SYMMETRIC]), ("0", [lgp.LGP_TC_ROW]),
                       (None, [lgp.LGP_TC_ROW, lgp.LGP_TC_SYMMETRIC])]:
        if flag is None:
            os.environ.pop("LGP_TC_SYMMETRIC", None)
        else:
            os.environ["LGP_TC_SYMMETRIC"] = flag
        ctx = lgp.Context(0)
        assert ctx.tc_kernel_choice(p.N, 8, wl.MATERN52, 32) == lgp.LGP_TC_UNTUNED
        lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.tc_kernel_choice(p.N, 8, wl.MATERN52, 32) in want
        assert ctx.tc_kernel_choice(p.N, 8, wl.MATERN52, 16) == lgp.LGP_TC_UNTUNED
        assert ctx.tc_kernel_choice(p.N, 8, wl.MATERN52, 8) < 0  # t=8 runs on the FP32 path
        ctx.close()
    os.environ.pop("LGP_TC_SYMMETRIC", None)


def test_symmetric_cg_solve(lgp, sym):
    """CG on the symmetric product reaches the Cholesky solution."""
    import torch
    p = wl.cfg3(N=3000, t=32)
    B = wl.rhs_block(p.N, 32, seed=3)
    B[:, 0] = p.y
    ref = go.cholesky_solve(go.noisy_kernel_matrix(p.X, go.hyper_of(p)), B.astype(np.float64))
    x, iters, rel, status = lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p,
                                             torch.as_tensor(B, device="cuda"), tol=1e-6, max_iter=3000,
                                             prec=lgp.LGP_PREC_SPLIT_F16, ctx=sym)
    assert status == lgp.LGP_OK
    assert (rel <= 1e-6).all()
    err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-4


def test_symmetric_lml_and_grad(lgp, sym):
    """The mBCG / SLQ / adjoint pipeline on the symmetric product against the FP64 estimator."""
    import torch
    p, m = wl.cfg3(N=2000, t=32), 31
    hyp = go.hyper_of(p)
    L, seed, tol = 50, 1234, 1e-6
    lml, grad, info = lgp.lgp_lml_and_grad(torch.as_tensor(p.X, device="cuda"), torch.as_tensor(p.y, device="cuda"),
                                           p, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=2000,
                                           ctx=sym)
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=2000)
    tg = go.probe_conditioned_targets(p.X, p.y, hyp, est["Z"])
    assert lml == pytest.approx(est["lml"], rel=1e-3)
    scale = np.maximum(np.abs(tg["grad"]), 1e-2 * np.abs(tg["grad"]).max())
    assert (np.abs(np.asarray(grad) - tg["grad"]) / scale).max() <= 1e-3


def test_autotune_cache_file(lgp, tmp_path):
    """LGP_AUTOTUNE_CACHE: the first context tunes and writes its choice; a second context reads it
    back (same choice, no new line)."""
    import torch
    path = tmp_path / "tune.txt"
    os.environ["LGP_AUTOTUNE_CACHE"] = str(path)
    os.environ.pop("LGP_TC_SYMMETRIC", None)
    try:
        p = wl.cfg3(N=2600, t=32)
        X = torch.as_tensor(p.X, device="cuda")
        V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=2), device="cuda")
        choices = []
        for _ in range(2):
            ctx = lgp.Context(0)
            lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, ctx=ctx)
            torch.cuda.synchronize()
            choices.append(ctx.tc_kernel_choice(p.N, p.D, p.kind, 32, lgp.LGP_PREC_SPLIT_F16))
            ctx.close()
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and "|2816|32|1|8|1 " in lines[0], lines
        assert choices[0] == choices[1] and choices[0] in (lgp.LGP_TC_ROW, lgp.LGP_TC_SYMMETRIC)
    finally:
        os.environ.pop("LGP_AUTOTUNE_CACHE", None)


def test_kernel_timing_hook(lgp):
    """lgp_set_kernel_timing / lgp_last_kernel_ms: with timing on, a product records CUDA events around its
    kernel alone; the kernel time is positive and no longer than the whole call (which also splits V).
    Reading it before any timed product is refused."""
    import torch
    p = wl.cfg3(N=20000, t=32)
    ctx = lgp.Context(0)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=3, kind="sign"), device="cuda")
    out = torch.empty_like(V)
    ctx.set_kernel_timing(True)
    with pytest.raises(lgp.LGPError) as e:
        ctx.last_kernel_ms()
    assert e.value.status == lgp.LGP_ERR_INVALID_ARG
    lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, out=out, ctx=ctx)
    for _ in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, out=out, ctx=ctx)
        b.record()
        torch.cuda.synchronize()
        call_ms, kernel_ms = a.elapsed_time(b), ctx.last_kernel_ms()
        print(f"call {call_ms:.4f} ms, kernel {kernel_ms:.4f} ms")
        assert 0.0 < kernel_ms <= call_ms
    ctx.set_kernel_timing(False)
    ctx.close()
