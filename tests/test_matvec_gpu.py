"""Parity of the fused product K_y V (CUDA, through the C ABI) with the FP64 oracle.

Gate: relative 2-norm error per column <= 1e-5 against the oracle evaluated in
float64 on the same float32 inputs. Sizes span several row and column tiles
with ragged tails; full-size workloads are checked on sampled rows.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _colerr(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


def _run(lgp, p, V, prec=None):
    import torch
    X = torch.as_tensor(p.X, device="cuda")
    Vt = torch.as_tensor(V, device="cuda")
    kw = {} if prec is None else {"prec": prec}
    out = lgp.lgp_kernel_matvec(X, p, Vt, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("t", [1, 2, 3, 4, 5, 8, 13, 16, 32, 33])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_fp32_matvec_small(lgp, kind, t):
    p = wl.random_problem(1500, 3, kind, seed=10 + t)
    V = wl.rhs_block(p.N, t, seed=t)
    got = _run(lgp, p, V, prec=lgp.LGP_PREC_FP32)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(got, ref).max() <= TOL


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7, 8])
def test_fp32_matvec_every_dimension(lgp, D):
    p = wl.random_problem(777, D, wl.MATERN52 if D % 2 else wl.RBF, seed=D)
    V = wl.rhs_block(p.N, 4, seed=D)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, p, V, prec=lgp.LGP_PREC_FP32), ref).max() <= TOL


@pytest.mark.parametrize("N", [1, 2, 3, 63, 64, 65, 127, 129, 255, 257, 511, 513, 4099])
def test_fp32_matvec_ragged_sizes(lgp, N):
    p = wl.random_problem(N, 2, wl.RBF, seed=N)
    V = wl.rhs_block(N, 2, seed=N)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, p, V, prec=lgp.LGP_PREC_FP32), ref).max() <= TOL


def test_cfg1_matvec(lgp):
    p = wl.cfg1()
    got = _run(lgp, p, p.y[:, None])
    ref = go.matvec(p.X, p.y[:, None], go.hyper_of(p))
    assert _colerr(got, ref).max() <= TOL


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_cfg2_matvec_full_size_sampled_rows(lgp, kind):
    """N=20000, D=3, t=1 (the paper's fused-product scale), rows sampled for the oracle."""
    p = wl.cfg2(kind=kind)
    got = _run(lgp, p, p.y[:, None], prec=lgp.LGP_PREC_FP32)
    rows = np.random.default_rng(0).choice(p.N, 300, replace=False)
    ref = go.matvec_rows(p.X, p.y[:, None], go.hyper_of(p), rows)
    assert _colerr(got[rows], ref).max() <= TOL


def test_cfg3_matvec_full_size_sampled_rows(lgp):
    """N=100000, D=8, Matern-5/2, t=32: the product inside the mBCG solve."""
    p = wl.cfg3()
    V = wl.rhs_block(p.N, 32, seed=3, kind="sign")
    V[:, 0] = p.y
    got = _run(lgp, p, V)
    rows = np.random.default_rng(1).choice(p.N, 256, replace=False)
    ref, _ = oracle.kyv_rows_c(p.X, V, go.hyper_of(p), rows=rows)
    assert _colerr(got[rows], ref).max() <= TOL


def test_cfg5_large_matvec_sampled_rows(lgp):
    """N=500000, D=2, RBF, t=32 with N(0,1) columns (O(N) memory: no N x N storage)."""
    p, V = wl.cfg5_large()
    got = _run(lgp, p, V)
    rows = np.random.default_rng(2).choice(p.N, 128, replace=False)
    ref, _ = oracle.kyv_rows_c(p.X, V, go.hyper_of(p), rows=rows)
    assert _colerr(got[rows], ref).max() <= TOL


def test_matvec_is_linear_and_noise_exact(lgp):
    """Properties at any size: K_y(aV) = a K_y V; zero outputscale gives sigma^2 V exactly."""
    p = wl.random_problem(3000, 4, wl.MATERN52, seed=5)
    V = wl.rhs_block(p.N, 4, seed=5)
    a = _run(lgp, p, V, prec=lgp.LGP_PREC_FP32)
    b = _run(lgp, p, 2.0 * V, prec=lgp.LGP_PREC_FP32)
    np.testing.assert_array_equal(b, 2.0 * a)
    q = wl.random_problem(3000, 4, wl.RBF, seed=6, log_os=-80.0, log_noise=math.log(0.25))
    c = _run(lgp, q, V, prec=lgp.LGP_PREC_FP32)
    np.testing.assert_allclose(c, 0.25 * V, rtol=1e-7, atol=0)


def test_matvec_rejects_bad_arguments(lgp):
    import torch
    p = wl.random_problem(100, 2, wl.RBF, seed=1)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.ones((100, 2), device="cuda")
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_kernel_matvec(X, p, V, out=V)
    assert e.value.status == lgp.LGP_ERR_INVALID_ARG
    Vh = torch.ones((100, 2))  # host memory
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_kernel_matvec(X, p, Vh.cuda(), out=torch.empty((100, 2)))
    assert e.value.status == lgp.LGP_ERR_INVALID_ARG
    bad = wl.random_problem(100, 9, wl.RBF, seed=2)
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_kernel_matvec(torch.as_tensor(bad.X, device="cuda"), bad, V)
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_kernel_matvec(X, p, torch.ones((100, 65), device="cuda"))
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED


def test_matvec_grad_blocks(lgp):
    """Derivative blocks dK_p W for all P = D + 2 hyperparameters against the oracle."""
    import torch
    for kind, D, t in [(wl.RBF, 3, 1), (wl.MATERN52, 5, 4), (wl.RBF, 8, 6), (wl.MATERN52, 2, 9)]:
        p = wl.random_problem(900 + 7 * t, D, kind, seed=20 + D)
        W = wl.rhs_block(p.N, t, seed=t)
        G = lgp.lgp_kernel_matvec_grad(torch.as_tensor(p.X, device="cuda"), p, torch.as_tensor(W, device="cuda"))
        G = G.cpu().numpy()
        ref = go.dK_matvec(p.X, W, go.hyper_of(p))
        assert G.shape == ref.shape
        for q in range(D + 2):
            assert _colerr(G[q], ref[q]).max() <= TOL, (kind, D, t, q)


# ----------------------------------------------------------------------------- tcgen05 split paths

# hi+lo bfloat16 keeps about 16 significant bits per factor: entries and V carry a
# representation error up to 2^-16 and the three-product sum drops a 2^-16 term, so the
# column error is a few 1e-5 once the sum cancels; its gate is 1e-4 (the scaled float16
# split, 22 bits per factor, is the one held to the 1e-5 product gate).
BF16_TOL = 1e-4


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("t", [16, 32])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
@pytest.mark.parametrize("N", [1, 100, 129, 1500, 4099])
def test_split_matvec(lgp, kind, t, N, fmt):
    p = wl.random_problem(N, 3, kind, seed=N + t)
    V = wl.rhs_block(N, t, seed=N)
    prec = lgp.LGP_PREC_SPLIT_F16 if fmt == "f16" else lgp.LGP_PREC_SPLIT_BF16
    got = _run(lgp, p, V, prec=prec)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(got, ref).max()
    print(f"split-{fmt} kind={kind} t={t} N={N}: max column rel err {err:.2e}")
    assert err <= (TOL if fmt == "f16" else BF16_TOL)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("t", [1, 5, 8, 20, 31])
@pytest.mark.parametrize("N", [129, 4099])
def test_split_matvec_zero_padded_columns(lgp, t, N, fmt):
    """An explicit split precision at t not in {16, 32}: the product runs on the columns zero-padded to 16 or
    32 and returns the caller's t columns, held to the same gates as the unpadded split products."""
    p = wl.random_problem(N, 3, wl.MATERN52, seed=N + 3 * t)
    V = wl.rhs_block(N, t, seed=N + t)
    prec = lgp.LGP_PREC_SPLIT_F16 if fmt == "f16" else lgp.LGP_PREC_SPLIT_BF16
    got = _run(lgp, p, V, prec=prec)
    assert got.shape == (N, t)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(got, ref).max()
    print(f"padded split-{fmt} t={t} N={N}: max column rel err {err:.2e}")
    assert err <= (TOL if fmt == "f16" else BF16_TOL)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7, 8])
def test_split_f16_every_dimension(lgp, D):
    p = wl.random_problem(2000, D, wl.MATERN52 if D % 2 else wl.RBF, seed=40 + D)
    V = wl.rhs_block(p.N, 32, seed=D)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, p, V, prec=lgp.LGP_PREC_SPLIT_F16), ref).max() <= TOL
    assert _colerr(_run(lgp, p, V, prec=lgp.LGP_PREC_SPLIT_BF16), ref).max() <= BF16_TOL


def test_split_column_scaling_extremes(lgp):
    """Columns of very different magnitude (and an all-zero column) keep their own scale."""
    p = wl.random_problem(3000, 4, wl.MATERN52, seed=77)
    V = wl.rhs_block(p.N, 16, seed=77)
    V[:, 1] *= 1e-20
    V[:, 2] *= 1e20
    V[:, 3] = 0.0
    V[:, 4] = np.abs(V[:, 4]) + 1e3
    got = _run(lgp, p, V, prec=lgp.LGP_PREC_SPLIT_F16)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert np.all(got[:, 3] == 0.0)
    keep = [c for c in range(16) if c != 3]
    assert _colerr(got[:, keep], ref[:, keep]).max() <= TOL


def test_split_f16_selected_by_auto(lgp):
    ctx = lgp.default_context()
    assert ctx.matvec_precision(32) == lgp.LGP_PREC_SPLIT_F16
    assert ctx.matvec_precision(16) == lgp.LGP_PREC_SPLIT_F16
    assert ctx.matvec_precision(8) == lgp.LGP_PREC_FP32
    # an explicit split precision at other t runs on zero-padded columns; above 32 columns it has none
    assert ctx.matvec_precision(8, lgp.LGP_PREC_SPLIT_BF16) == lgp.LGP_PREC_SPLIT_BF16
    assert ctx.matvec_precision(1, lgp.LGP_PREC_SPLIT_F16) == lgp.LGP_PREC_SPLIT_F16
    assert ctx.matvec_precision(33, lgp.LGP_PREC_SPLIT_F16) == lgp.LGP_ERR_UNSUPPORTED
    assert ctx.matvec_precision(32, lgp.LGP_PREC_SPLIT_BF16) == lgp.LGP_PREC_SPLIT_BF16


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_cfg2_split_t16_full_size(lgp, kind):
    """N=20000, D=3, t=16 (y + 15 probes) on the tensor-core path, sampled rows against the C oracle."""
    p = wl.cfg2(kind=kind, t=16)
    V = wl.rhs_block(p.N, 16, seed=7, kind="sign")
    V[:, 0] = p.y
    got = _run(lgp, p, V)
    rows = np.random.default_rng(3).choice(p.N, 400, replace=False)
    ref, _ = oracle.kyv_rows_c(p.X, V, go.hyper_of(p), rows=rows)
    assert _colerr(got[rows], ref).max() <= TOL


def test_tensor_core_agrees_with_fp32_path(lgp):
    """Two independent GPU routes to the same product agree to the split error level."""
    p = wl.cfg3(N=6000, t=32)
    V = wl.rhs_block(p.N, 32, seed=9)
    a = _run(lgp, p, V, prec=lgp.LGP_PREC_FP32).astype(np.float64)
    b = _run(lgp, p, V, prec=lgp.LGP_PREC_SPLIT_F16).astype(np.float64)
    assert (np.linalg.norm(a - b, axis=0) / np.linalg.norm(a, axis=0)).max() <= TOL


def test_autotuned_split_count_gives_the_same_product(lgp):
    """The autotuner only changes how the column range is split across CTAs: every candidate
    split must give the product within the tolerance (here: autotuning on vs off, fresh contexts)."""
    import os
    import torch
    p = wl.cfg3(N=9000, t=32)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=4), device="cuda")
    outs = []
    for flag in ["1", "0"]:
        os.environ["LGP_AUTOTUNE"] = flag
        ctx = lgp.Context(0)
        outs.append(lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, ctx=ctx).cpu().numpy())
        torch.cuda.synchronize()
        ctx.close()
    os.environ.pop("LGP_AUTOTUNE", None)
    ref = go.matvec(p.X, wl.rhs_block(p.N, 32, seed=4), go.hyper_of(p))
    for o in outs:
        assert _colerr(o, ref).max() <= TOL
