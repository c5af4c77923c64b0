"""Parity of CG solves and of the LML / gradient pipeline with the FP64 oracle.

Gates: CG solution relative error <= 1e-4 against the Cholesky solve when run to
relative residual 1e-6; LML and gradient within 1e-3 relative of the oracle's
value for the same probes (gradient components relative to
max(|g_p|, 1e-2 max_q |g_q|)).
"""
import math

import numpy as np
import pytest

from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _solve_err(x, ref):
    x = np.asarray(x, dtype=np.float64).reshape(ref.shape)
    return np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)


def test_cfg1_cg_solve(lgp):
    p = wl.cfg1()
    hyp = go.hyper_of(p)
    Ky = go.noisy_kernel_matrix(p.X, hyp)
    ref = go.cholesky_solve(Ky, p.y.astype(np.float64))[:, None]
    x, iters, rel, status = lgp.lgp_cg_solve(_dev(p.X), p, _dev(p.y[:, None]), tol=1e-6, max_iter=2000)
    assert status == lgp.LGP_OK
    assert rel[0] <= 1e-6
    err = _solve_err(x.cpu().numpy(), ref)
    true_res = np.linalg.norm(p.y - Ky @ x.cpu().numpy()[:, 0].astype(np.float64)) / np.linalg.norm(p.y)
    print(f"cfg1: iters {iters[0]} sol err {err[0]:.2e} true residual {true_res:.2e}")
    assert err.max() <= 1e-4


@pytest.mark.parametrize("t", [1, 3])
def test_cg_solve_split_precision_zero_padded(lgp, t):
    """lgp_cg_solve with an explicit split precision at t < 16: the solve runs on 16 zero-padded columns (the
    zero ones take no iteration) and returns t columns. Against the Cholesky solve with the gates of the
    full-size split solves: forward error <= max(1e-4, 2e-8 kappa) and componentwise backward error <= 1e-5
    (the split product's own error, ~1e-6, is amplified by kappa in the forward error). A warm start from
    that solution (padded the same way) needs fewer iterations than the solve from zero."""
    p = wl.cfg2(N=3000, kind=wl.MATERN52)
    B = wl.rhs_block(p.N, t, seed=7)
    B[:, 0] = p.y
    Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
    ev = np.linalg.eigvalsh(Ky)
    ref = go.cholesky_solve(Ky, B.astype(np.float64))
    x, iters, rel, status = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=3000,
                                             prec=lgp.LGP_PREC_SPLIT_F16)
    assert status == lgp.LGP_OK and x.shape == (p.N, t) and len(iters) == t
    assert (rel <= 1e-6).all()
    xs = x.cpu().numpy().astype(np.float64)
    err = _solve_err(xs, ref)
    berr = np.abs(B - Ky @ xs) / (Ky @ np.abs(xs) + np.abs(B))
    gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
    print(f"padded split t={t}: iterations {list(iters)}, forward error {err.max():.2e} (gate {gate:.2e}), "
          f"backward error {berr.max():.2e}")
    assert err.max() <= gate
    assert berr.max() <= 1e-5
    x2, iters2, rel2, status2 = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=3000,
                                                 prec=lgp.LGP_PREC_SPLIT_F16, x0=x)
    assert status2 == lgp.LGP_OK and (rel2 <= 1e-6).all()
    # the restart recomputes the true residual with the split product, above the recursive one that met tol,
    # so it iterates again, but from the padded warm start: fewer iterations than from zero
    assert int(np.max(iters2)) < int(np.min(iters))


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_cfg2_cg_multi_rhs(lgp, kind):
    p = wl.cfg2(N=3000, kind=kind)
    B = wl.rhs_block(p.N, 4, seed=2)
    B[:, 0] = p.y
    ref = go.cholesky_solve(go.noisy_kernel_matrix(p.X, go.hyper_of(p)), B.astype(np.float64))
    x, iters, rel, status = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=3000,
                                             prec=lgp.LGP_PREC_FP32)
    assert status == lgp.LGP_OK
    assert (rel <= 1e-6).all()
    assert _solve_err(x.cpu().numpy(), ref).max() <= 1e-4


def test_cg_iteration_counts_match_fp64_cg(lgp):
    """Same recurrence as the oracle's textbook CG: float32 vectors need at least as many
    iterations as exact-arithmetic-like float64 CG, and not many more."""
    p = wl.random_problem(800, 2, wl.RBF, seed=3, log_noise=math.log(0.1))
    B = wl.rhs_block(p.N, 3, seed=3)
    Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
    res = go.cg(lambda P: Ky @ P, B.astype(np.float64), 1e-6, 2000)
    _, iters, _, _ = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=2000)
    assert (iters >= res.iters - 1).all()
    assert (iters <= 2 * res.iters + 10).all(), (iters, res.iters)


def test_cg_edge_cases(lgp):
    import torch
    p = wl.random_problem(300, 3, wl.MATERN52, seed=4)
    B = wl.rhs_block(p.N, 3, seed=4)
    B[:, 1] = 0.0
    x, iters, rel, status = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=1000)
    assert iters[1] == 0 and np.all(x.cpu().numpy()[:, 1] == 0.0)
    # max_iter=1: valid outputs with a warning
    x, iters, rel, status = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=1)
    assert status == lgp.LGP_WARN_NOT_CONVERGED and iters.max() == 1
    # N = 1: one step solves b / (s^2 + sigma^2)
    q = wl.random_problem(1, 2, wl.RBF, seed=5)
    x, iters, _, status = lgp.lgp_cg_solve(_dev(q.X), q, _dev(np.array([[2.0]], np.float32)), tol=1e-6)
    assert status == lgp.LGP_OK
    assert abs(float(x.cpu()) - 2.0 / (math.exp(q.log_outputscale) + math.exp(q.log_noise))) < 1e-6
    # non-finite inputs are reported, not propagated
    Bn = B.copy()
    Bn[7, 0] = np.nan
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(_dev(p.X), p, _dev(Bn))
    assert e.value.status == lgp.LGP_ERR_NONFINITE
    Xn = p.X.copy()
    Xn[3, 1] = np.inf
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(_dev(Xn), p, _dev(B))
    assert e.value.status == lgp.LGP_ERR_NONFINITE
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=0.0)
    assert e.value.status == lgp.LGP_ERR_INVALID_ARG


def test_rademacher_probes_bit_exact(lgp):
    seed = 0xC0FFEE1234
    Z = lgp.lgp_rademacher_probes(seed, 5003, 31).cpu().numpy()
    np.testing.assert_array_equal(Z, go.rademacher(seed, 5003, 31).astype(np.float32))


def _grad_err(g, ref):
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())
    return np.abs(np.asarray(g) - ref) / scale


@pytest.mark.parametrize("case", ["cfg3-m52", "cfg4-rbf"])
def test_lml_and_grad_against_oracle(lgp, case):
    """Reduced-N draws of the mBCG workloads (same distributions): GPU estimator vs the FP64 oracle."""
    if case == "cfg3-m52":
        p, m = wl.cfg3(N=2000, t=32), 31
    else:
        p, m = wl.cfg4(N=2000, t=16), 15
    hyp = go.hyper_of(p)
    L, seed, tol = 50, 1234, 1e-6
    lml, grad, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=L, seed=seed,
                                           tol=tol, max_iter=2000)
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=2000)
    tg = go.probe_conditioned_targets(p.X, p.y, hyp, est["Z"])
    exact = go.lml(p.X, p.y, hyp)
    print(f"{case}: lml gpu {lml:.6f} fp64-est {est['lml']:.6f} probe-target {tg['lml']:.6f} exact {exact:.6f} "
          f"iters {info['iters_min']}..{info['iters_max']} prec {info['prec_used']}")
    assert info["quad"] == pytest.approx(tg["quad"], rel=1e-4)
    assert lml == pytest.approx(est["lml"], rel=1e-3)
    assert info["logdet"] == pytest.approx(est["logdet"], abs=1e-3 * abs(est["lml"]))
    assert _grad_err(grad, tg["grad"]).max() <= 1e-3
    assert _grad_err(grad, est["grad"]).max() <= 1e-3


@pytest.mark.parametrize("n,L", [(24, 64), (40, 64), (200, 3)])
def test_slq_quadrature_against_probe_targets(lgp, n, L):
    """The log-determinant quadrature, pinned tighter than the LML gate.

    With CG run until its Krylov space holds every probe (N <= L), Gauss quadrature on the Lanczos
    tridiagonal is exact: mean_i ||z_i||^2 e_1^T log(T_i) e_1 = mean_i z_i^T log(K_y) z_i, the oracle's
    probe-conditioned log-determinant (eigh of K_y), up to float32 CG rounding. With L = 3 steps on a
    larger problem the quadrature is the FP64 estimator's own truncated one, compared at its gate."""
    p = wl.random_problem(n, 2, wl.RBF, seed=21 + n, log_noise=math.log(0.1))
    hyp = go.hyper_of(p)
    m, seed = 7, 5
    lml, _, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=L, seed=seed,
                                        tol=1e-7, max_iter=400, want_grad=False)
    if n <= L:
        tg = go.probe_conditioned_targets(p.X, p.y, hyp, go.rademacher(seed, n, m))
        assert info["logdet"] == pytest.approx(tg["logdet"], rel=1e-5, abs=1e-5)
    else:
        est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=1e-7, max_iter=400)
        assert info["logdet"] == pytest.approx(est["logdet"], rel=1e-4)


@pytest.mark.parametrize("L", [512, 1024])
def test_long_lanczos_against_oracle(lgp, L):
    """Lanczos lengths beyond one quadrature thread per step (m > 256 steps kept), on a badly conditioned
    problem (Matern-5/2, D=3, lengthscales in [0.3, 1], noise 1e-3, N=2000: ~840 CG iterations at tol
    1e-6 in float64): the GPU log-determinant and LML against the FP64 estimator with the same L, probes
    and tolerance. L = 1024 is the largest accepted; 1025 is refused."""
    p, m = wl.random_problem(2000, 3, wl.MATERN52, seed=41, lo=0.3, hi=1.0, log_noise=math.log(1e-3)), 15
    hyp = go.hyper_of(p)
    seed, tol = 4321, 1e-6
    lml, _, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=L, seed=seed, tol=tol,
                                        max_iter=3000, want_grad=False)
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=3000)
    print(f"L={L}: logdet gpu {info['logdet']:.6f} fp64 {est['logdet']:.6f}, iterations "
          f"{info['iters_min']}..{info['iters_max']}")
    assert info["iters_max"] > 256  # the quadrature kernel's strided loads are exercised
    assert info["logdet"] == pytest.approx(est["logdet"], abs=1e-3 * abs(est["lml"]))
    assert lml == pytest.approx(est["lml"], rel=1e-3)
    if L == 1024:
        with pytest.raises(lgp.LGPError) as e:
            lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=lgp.LGP_MAX_LANCZOS_STEPS + 1,
                                 seed=seed, tol=tol)
        assert e.value.status == lgp.LGP_ERR_UNSUPPORTED


def test_single_column_path_and_batched_path_meet_the_same_gate(lgp):
    """Equal accuracy of the two paths the bench compares, on the mBCG workload's distribution at N=3000:
    the batched split-F16 mBCG step and the plain FP32 single-column step (every column its own CG run
    with the one-column product, one adjoint pass per column) use the same probes, tolerance and Lanczos
    length, and each meets the 1e-3 LML and gradient gates against the FP64 estimator and the
    probe-conditioned targets."""
    p, m = wl.cfg3(N=3000, t=32), 31
    hyp = go.hyper_of(p)
    L, seed, tol = 50, 77, 1e-6
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=3000)
    tg = go.probe_conditioned_targets(p.X, p.y, hyp, est["Z"])
    X, y = _dev(p.X), _dev(p.y)
    for single in (False, True):
        lml, grad, info = lgp.lgp_lml_and_grad(X, y, p, n_probes=m, lanczos_steps=L, seed=seed, tol=tol,
                                               max_iter=3000, single_rhs=single)
        label = "single-column FP32" if single else "batched"
        print(f"{label}: lml {lml:.6f} (fp64 estimator {est['lml']:.6f}), iterations "
              f"{info['iters_min']}..{info['iters_max']}, launches {info['launches']}")
        assert info["prec_used"] == (lgp.LGP_PREC_FP32 if single else lgp.LGP_PREC_SPLIT_F16)
        assert info["t"] == m + 1
        assert lml == pytest.approx(est["lml"], rel=1e-3)
        assert info["quad"] == pytest.approx(tg["quad"], rel=1e-4)
        assert _grad_err(grad, est["grad"]).max() <= 1e-3
        assert _grad_err(grad, tg["grad"]).max() <= 1e-3


def test_single_column_path_rejects_a_preconditioner(lgp):
    p = wl.cfg3(N=500, t=8)
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=7, single_rhs=True, precond_rank=4)
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED


def test_lml_gradient_matches_finite_differences_of_exact_lml(lgp):
    """cfg4-shaped check: the analytic gradient estimate against central FD (h=1e-3) of the exact LML.

    The estimator's trace term carries Hutchinson noise, so the gate is its
    standard error (four sigma, computed from the same probes) plus the FD error.
    """
    p = wl.cfg4(N=2000, t=64)
    hyp = go.hyper_of(p)
    m = 63
    lml, grad, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=50, seed=99,
                                           tol=1e-6, max_iter=2000)
    D = p.D
    theta = np.concatenate([hyp.log_lengthscale, [hyp.log_outputscale, hyp.log_noise]])
    h = 1e-3
    fd = np.zeros_like(theta)
    for q in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (go.lml(p.X, p.y, go.Hyper(p.kind, tp[:D], tp[D], tp[D + 1]))
                 - go.lml(p.X, p.y, go.Hyper(p.kind, tm[:D], tm[D], tm[D + 1]))) / (2 * h)
    Z = go.rademacher(99, p.N, m)
    Ky = go.noisy_kernel_matrix(p.X, hyp)
    U = go.cholesky_solve(Ky, Z)
    se = np.array([0.5 * np.std(np.sum(U * (M @ Z), axis=0), ddof=1) / math.sqrt(m)
                   for M in go.dK_matrices(p.X, hyp)])
    assert (np.abs(grad - fd) <= 4.0 * se + 1e-3 * np.abs(fd) + 1e-6).all(), (grad, fd, se)


def test_autograd_function(lgp):
    import torch
    p = wl.cfg4(N=1500, t=16)
    ll = torch.tensor(p.log_lengthscale, dtype=torch.float32, requires_grad=True)
    lo = torch.tensor(p.log_outputscale, dtype=torch.float32, requires_grad=True)
    ln = torch.tensor(p.log_noise, dtype=torch.float32, requires_grad=True)
    val = lgp.marginal_likelihood(_dev(p.X), _dev(p.y), ll, lo, ln, kind=p.kind, n_probes=15, lanczos_steps=50,
                                  seed=5, tol=1e-6)
    (-2.0 * val).backward()
    _, g, _ = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=15, lanczos_steps=50, seed=5, tol=1e-6)
    # a second call: equal up to the float32 summation order of the symmetric product's atomic
    # reductions (which moves the CG trajectory in the last bits), far inside the 1e-3 gate
    np.testing.assert_allclose(ll.grad.numpy(), -2.0 * g[:p.D], rtol=1e-4)
    assert float(lo.grad) == pytest.approx(-2.0 * g[p.D], rel=1e-4)
    assert float(ln.grad) == pytest.approx(-2.0 * g[p.D + 1], rel=1e-4)


def test_host_driven_loop_matches_the_graph_loop(lgp):
    """LGP_CG_GRAPH=0 (one launch per kernel, done flag read on the host) runs the same kernels as the
    device-side while loop: on the deterministic FP32 path the solutions agree bit for bit, and the
    LML info reports the same iterations."""
    import os
    p = wl.cfg2(N=3000, kind=wl.MATERN52)
    B = wl.rhs_block(p.N, 4, seed=12)
    outs = {}
    for flag in ("1", "0"):
        os.environ["LGP_CG_GRAPH"] = flag
        ctx = lgp.Context(0)
        x, it, rel, s = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=3000, prec=lgp.LGP_PREC_FP32,
                                         ctx=ctx)
        assert s == lgp.LGP_OK
        outs[flag] = (x.cpu().numpy(), it.copy())
        ctx.close()
    os.environ.pop("LGP_CG_GRAPH", None)
    np.testing.assert_array_equal(outs["1"][0], outs["0"][0])
    np.testing.assert_array_equal(outs["1"][1], outs["0"][1])
