"""The four stationary kernels (RBF, Matern-1/2, -3/2, -5/2; Sec. 3 "Kernels") on every GPU path,
against the FP64 oracle: the FP32 product, both tensor-core products, the derivative blocks, the
LML estimator with its gradient, and the batched solver.

Gates as elsewhere: product column error <= 1e-5 (FP32 and scaled-FP16 split), <= 1e-4 (BF16
split); LML and gradient within 1e-3 of the oracle's FP64 run of the same estimator.
"""
import math
import os

import numpy as np
import pytest

from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5
BF16_TOL = 1e-4
ALL = [wl.RBF, wl.MATERN52, wl.MATERN32, wl.MATERN12]
NEW = [wl.MATERN32, wl.MATERN12]


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _colerr(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


def _matvec(lgp, p, V, prec, ctx=None):
    import torch
    out = lgp.lgp_kernel_matvec(_dev(p.X), p, _dev(V), prec=prec, ctx=ctx)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("t", [1, 3, 8, 16, 33])
@pytest.mark.parametrize("kind", NEW)
def test_fp32_product_new_kernels(lgp, kind, t):
    p = wl.random_problem(1300, 4, kind, seed=200 + t)
    V = wl.rhs_block(p.N, t, seed=t)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_matvec(lgp, p, V, lgp.LGP_PREC_FP32), ref).max() <= TOL


@pytest.mark.parametrize("sym", ["0", "1"])
@pytest.mark.parametrize("t", [16, 32])
@pytest.mark.parametrize("kind", ALL)
def test_split_products_every_kernel(lgp, kind, t, sym):
    """Row kernel (LGP_TC_SYMMETRIC=0) and symmetric-tile kernel (=1), both split formats."""
    os.environ["LGP_TC_SYMMETRIC"] = sym
    ctx = lgp.Context(0)
    try:
        for D in (3, 7):
            p = wl.random_problem(2333, D, kind, seed=300 + D + t)
            V = wl.rhs_block(p.N, t, seed=D)
            ref = go.matvec(p.X, V, go.hyper_of(p))
            assert _colerr(_matvec(lgp, p, V, lgp.LGP_PREC_SPLIT_F16, ctx), ref).max() <= TOL, (kind, D, t, sym)
            assert _colerr(_matvec(lgp, p, V, lgp.LGP_PREC_SPLIT_BF16, ctx), ref).max() <= BF16_TOL, (kind, D, t, sym)
            want = lgp.LGP_TC_SYMMETRIC if sym == "1" else lgp.LGP_TC_ROW
            assert ctx.tc_kernel_choice(p.N, D, kind, t, lgp.LGP_PREC_SPLIT_F16) == want
    finally:
        ctx.close()
        os.environ.pop("LGP_TC_SYMMETRIC", None)


@pytest.mark.parametrize("kind", NEW)
def test_derivative_blocks_new_kernels(lgp, kind):
    import torch
    for D, t in [(2, 1), (5, 4), (8, 3)]:
        p = wl.random_problem(800 + 11 * t, D, kind, seed=400 + D)
        W = wl.rhs_block(p.N, t, seed=t)
        G = lgp.lgp_kernel_matvec_grad(_dev(p.X), p, _dev(W)).cpu().numpy()
        torch.cuda.synchronize()
        ref = go.dK_matvec(p.X, W, go.hyper_of(p))
        for q in range(D + 2):
            assert _colerr(G[q], ref[q]).max() <= TOL, (kind, D, t, q)


def test_matern12_derivative_at_coincident_points(lgp):
    """Matern-1/2 at r = 0 between different rows (duplicated points): finite blocks, equal to the oracle's
    limit value 0 for those pairs."""
    p = wl.random_problem(600, 3, wl.MATERN12, seed=41)
    p.X[300:310] = p.X[0:10]
    W = wl.rhs_block(p.N, 2, seed=41)
    G = lgp.lgp_kernel_matvec_grad(_dev(p.X), p, _dev(W)).cpu().numpy()
    assert np.isfinite(G).all()
    ref = go.dK_matvec(p.X, W, go.hyper_of(p))
    for q in range(p.D + 2):
        assert _colerr(G[q], ref[q]).max() <= TOL


@pytest.mark.parametrize("kind", NEW)
def test_lml_and_grad_new_kernels(lgp, kind):
    p = wl.random_problem(1800, 4, kind, seed=500 + kind, log_noise=math.log(0.05))
    m, L, seed, tol = 15, 50, 77, 1e-6
    hyp = go.hyper_of(p)
    lml, grad, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=L, seed=seed,
                                           tol=tol, max_iter=3000)
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=3000)
    tg = go.probe_conditioned_targets(p.X, p.y, hyp, est["Z"])
    assert info["quad"] == pytest.approx(tg["quad"], rel=1e-4)
    assert lml == pytest.approx(est["lml"], rel=1e-3)
    scale = np.maximum(np.abs(tg["grad"]), 1e-2 * np.abs(tg["grad"]).max())
    assert (np.abs(np.asarray(grad) - tg["grad"]) / scale).max() <= 1e-3
    assert (np.abs(np.asarray(grad) - est["grad"]) / scale).max() <= 1e-3


def test_batch_mixed_kernels(lgp):
    """One batch holding all four kernels, uneven sizes, against each problem's Cholesky solve."""
    probs = [wl.random_problem(n, d, k, seed=600 + n, log_noise=math.log(0.05))
             for n, d, k in [(700, 2, wl.RBF), (1500, 3, wl.MATERN12), (400, 5, wl.MATERN32), (1100, 1, wl.MATERN52),
                             (900, 6, wl.MATERN12), (250, 4, wl.MATERN32)]]
    Bs = [wl.rhs_block(p.N, 8, seed=g) for g, p in enumerate(probs)]
    sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                 tol=1e-6, max_iter=4000)
    assert s == lgp.LGP_OK
    assert (rel <= 1e-6).all()
    for p, B, x in zip(probs, Bs, sols):
        Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
        ev = np.linalg.eigvalsh(Ky)
        gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
        ref = go.cholesky_solve(Ky, B.astype(np.float64))
        err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= gate, (p.kind, p.N, err.max(), gate)
