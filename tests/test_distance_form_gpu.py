"""The two ways the symmetric-tile product forms squared distances, against the FP64 oracle.

Difference form: r^2 = sum_d (x_id - x_jd)^2 in float32 registers (2 D operations per entry).
Dot form: r^2 = |u_i|^2 + |u_j|^2 - 2 u_i . u_j for the box-centred prescaled coordinates u,
the inner products as one tensor-core Gram tile per 128 x 128 tile (float16 hi/lo operands,
float32 accumulation) -- the rewriting of the distance that Sec. 3 gives as the reason the
product time barely depends on D. Its rounding error is absolute, about max |u|^2 2^-22, so the
library uses it only for kernels smooth in r^2 at r = 0 (RBF, Matern-3/2, Matern-5/2), at D >= 2,
and when max |u|^2 is below a per-kernel limit; the rest takes the difference form.

Gates as for every product: column relative error <= 1e-5 (scaled float16 halves), <= 1e-4
(bfloat16 halves); CG within 1e-4 of Cholesky; LML and gradient within 1e-3 of the oracle's
estimator.
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
SMOOTH = [wl.RBF, wl.MATERN52, wl.MATERN32]
# per-kernel limits on max |u|^2 (prescaled coordinates) above which the difference form runs
LIMIT = {wl.RBF: 97.0, wl.MATERN52: 403.0, wl.MATERN32: 134.0}
PRESCALE = {wl.RBF: math.sqrt(math.log2(math.e) / 2), wl.MATERN52: math.sqrt(5.0), wl.MATERN32: math.sqrt(3.0),
            wl.MATERN12: math.log2(math.e)}


def _colerr(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


@pytest.fixture(params=["auto", "diff"])
def form_ctx(lgp, request):
    os.environ["LGP_TC_SYMMETRIC"] = "1"
    if request.param == "diff":
        os.environ["LGP_DISTANCE"] = "diff"
    ctx = lgp.Context(0)
    yield request.param, ctx
    ctx.close()
    os.environ.pop("LGP_TC_SYMMETRIC", None)
    os.environ.pop("LGP_DISTANCE", None)


@pytest.fixture
def sym(lgp):
    os.environ["LGP_TC_SYMMETRIC"] = "1"
    ctx = lgp.Context(0)
    yield ctx
    ctx.close()
    os.environ.pop("LGP_TC_SYMMETRIC", None)


def _run(lgp, ctx, p, V, prec):
    import torch
    o = lgp.lgp_kernel_matvec(torch.as_tensor(p.X, device="cuda"), p, torch.as_tensor(V, device="cuda"), prec=prec,
                              ctx=ctx)
    torch.cuda.synchronize()
    return o.cpu().numpy()


def _norm_max(p):
    """max_j |u_j|^2 for the box-centred prescaled coordinates (float64, host)."""
    xs = p.X.astype(np.float64) * PRESCALE[p.kind] / np.exp(p.log_lengthscale.astype(np.float64))
    c = 0.5 * (xs.max(0) + xs.min(0))
    return float((((xs - c) ** 2).sum(1)).max())


@pytest.mark.parametrize("t", [16, 32])
@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("kind", SMOOTH)
def test_both_forms_match_the_oracle(lgp, form_ctx, kind, D, t):
    form, ctx = form_ctx
    # At D <= 2, lengthscales up to 2 on [0, 1]^D make K nearly rank one: sum_j |k_ij v_j| then exceeds
    # |(K v)_i| by up to ~1500x (RBF, D = 1), and a column-relative 1e-5 gate asks more than entries and V
    # carried to 22 bits can give, in either distance form (a CPU model with 2^-22 entry noise alone gives
    # 7e-6 there). The low-dimensional draws take lengthscales in [0.1, 0.5] (amplification <= ~420), the
    # range of the paper's low-dimensional workloads (lengthscale 0.2 at D = 2).
    lo, hi = (0.1, 0.5) if D <= 2 else (0.3, 2.0)
    p = wl.random_problem(1500, D, kind, seed=300 + 10 * D + kind, lo=lo, hi=hi)  # ragged: 11 tiles + 92 rows
    V = wl.rhs_block(p.N, t, seed=D + t)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(_run(lgp, ctx, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max()
    got_form, amax = ctx.tc_distance_form()
    print(f"{form} kind={kind} D={D} t={t}: form {got_form} max|u|^2 {amax:.2f} (host {_norm_max(p):.2f}) "
          f"err {err:.2e}")
    assert got_form == (lgp.LGP_DIST_DOT if form == "auto" and D >= 2 else lgp.LGP_DIST_DIFF)
    if got_form == lgp.LGP_DIST_DOT:
        assert amax == pytest.approx(_norm_max(p), rel=1e-3)
    assert err <= TOL


@pytest.mark.parametrize("kind", SMOOTH)
def test_dot_form_bfloat16_halves(lgp, sym, kind):
    p = wl.random_problem(2100, 7, kind, seed=330 + kind)
    V = wl.rhs_block(p.N, 32, seed=33)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_BF16), ref).max() <= BF16_TOL
    assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT


@pytest.mark.parametrize("kind", SMOOTH)
def test_dot_form_just_below_its_limit(lgp, sym, kind):
    """Lengthscales chosen so that max |u|^2 sits at 90% of the kernel's limit: the dot form still
    runs and still meets the product gate (the limit is where its error bound reaches ~1.6e-5)."""
    p = wl.cfg3(N=2500, kind=kind)
    ls = np.exp(p.log_lengthscale.astype(np.float64))
    scale = math.sqrt(_norm_max(p) / (0.9 * LIMIT[kind]))
    p.log_lengthscale = np.log(ls * scale).astype(np.float32)
    assert _norm_max(p) == pytest.approx(0.9 * LIMIT[kind], rel=1e-3)
    V = wl.rhs_block(p.N, 32, seed=44)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max()
    print(f"kind={kind}: max|u|^2 {_norm_max(p):.1f} err {err:.2e}")
    assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT
    assert err <= TOL


def test_wide_data_takes_the_difference_form(lgp, sym):
    """Points spread over many lengthscales (a long series): max |u|^2 is far above the limit, the
    gate hands the product to the difference form, and its result meets the gate."""
    rng = np.random.default_rng(7)
    N, D = 2000, 3
    X = rng.uniform(0.0, 300.0, size=(N, D)).astype(np.float32)
    p = wl.Problem(X, rng.standard_normal(N).astype(np.float32), wl.MATERN52, np.zeros(D, np.float32), 0.0,
                   float(np.float32(math.log(0.05))))
    V = wl.rhs_block(N, 16, seed=7)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    err = _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max()
    form, amax = sym.tc_distance_form()
    assert form == lgp.LGP_DIST_DIFF and amax > LIMIT[wl.MATERN52]
    assert err <= TOL


@pytest.mark.parametrize("kind,D", [(wl.MATERN12, 5), (wl.MATERN12, 2), (wl.RBF, 1), (wl.MATERN52, 1)])
def test_forms_without_a_dot_variant(lgp, sym, kind, D):
    p = wl.random_problem(1300, D, kind, seed=350 + D)
    V = wl.rhs_block(p.N, 16, seed=35)
    ref = go.matvec(p.X, V, go.hyper_of(p))
    assert _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max() <= TOL
    assert sym.tc_distance_form() == (lgp.LGP_DIST_DIFF, -1.0)


def test_no_symmetric_product_yet(lgp):
    ctx = lgp.Context(0)
    assert ctx.tc_distance_form() == (lgp.LGP_DIST_NONE, -1.0)
    ctx.close()


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN32])
def test_dot_form_cg_solve(lgp, sym, kind):
    """CG on the dot-form product reaches the Cholesky solution (cfg3 distribution, D = 8)."""
    import torch
    p = wl.cfg3(N=3000, t=32, kind=kind)
    B = wl.rhs_block(p.N, 16, seed=3)
    B[:, 0] = p.y
    ref = go.cholesky_solve(go.noisy_kernel_matrix(p.X, go.hyper_of(p)), B.astype(np.float64))
    x, iters, rel, status = lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p,
                                             torch.as_tensor(B, device="cuda"), tol=1e-6, max_iter=3000,
                                             prec=lgp.LGP_PREC_SPLIT_F16, ctx=sym)
    assert status == lgp.LGP_OK and (rel <= 1e-6).all()
    assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT
    err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    print(f"kind={kind}: iterations {iters.max()}, err {err.max():.2e}")
    assert err.max() <= 1e-4


def test_operands_follow_each_new_x(lgp, sym):
    """The dot-form operands are built once per prepared X and reused by the products of a solve:
    problems that alternate on one context (one workspace) must never see each other's operands,
    in single products and in solves (stale operands would give errors of order one)."""
    import torch
    probs = [wl.random_problem(2000, 6, wl.MATERN52, seed=seed, lo=0.3, log_noise=math.log(0.1)) for seed in (401, 402)]
    for p in probs + probs:
        V = wl.rhs_block(p.N, 32, seed=7)
        ref = go.matvec(p.X, V, go.hyper_of(p))
        err = _colerr(_run(lgp, sym, p, V, lgp.LGP_PREC_SPLIT_F16), ref).max()
        assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT
        assert err <= TOL
        B = V[:, :16].copy()
        Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
        ev = np.linalg.eigvalsh(Ky)
        gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
        refx = go.cholesky_solve(Ky, B.astype(np.float64))
        x, it, rel, s = lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p, torch.as_tensor(B, device="cuda"),
                                         tol=1e-6, max_iter=3000, prec=lgp.LGP_PREC_SPLIT_F16, ctx=sym)
        assert s == lgp.LGP_OK
        errx = (np.linalg.norm(x.cpu().numpy() - refx, axis=0) / np.linalg.norm(refx, axis=0)).max()
        print(f"product err {err:.2e}; solve err {errx:.2e} (gate {gate:.1e}, iterations {it.max()})")
        assert errx <= gate


@pytest.mark.parametrize("N", [1024, 4000])
def test_dot_form_cg_solve_two_dimensions(lgp, sym, N):
    """The plain-CG workload's distribution (X ~ U[0,1]^2, RBF, lengthscale 0.2, sigma^2 = 0.01) solved with the
    split product, whose distances at D = 2 now come from the tensor-core Gram tile: the solution of
    [y | 15 probes] against the dense Cholesky solution, at the gate that the product's error allows for the
    problem's condition number (1e-4, or 2e-8 kappa when that is larger)."""
    import torch
    p = wl.cfg1(N=N)
    B = wl.rhs_block(p.N, 16, seed=21)
    B[:, 0] = p.y
    Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
    ev = np.linalg.eigvalsh(Ky)
    gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
    ref = go.cholesky_solve(Ky, B.astype(np.float64))
    x, iters, rel, status = lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p,
                                             torch.as_tensor(B, device="cuda"), tol=1e-6, max_iter=3000,
                                             prec=lgp.LGP_PREC_SPLIT_F16, ctx=sym)
    assert status == lgp.LGP_OK and (rel <= 1e-6).all()
    assert sym.tc_distance_form()[0] == lgp.LGP_DIST_DOT
    err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    print(f"N={N}: kappa {ev[-1] / ev[0]:.2e}, iterations {iters.max()}, err {err.max():.2e} (gate {gate:.1e})")
    assert err.max() <= gate
