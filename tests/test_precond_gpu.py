"""Pivoted-Cholesky preconditioned CG (the gap Sec. 5 names for the paper's CG loop) on the GPU,
against the FP64 oracle: the solve, the preconditioned LML / gradient estimator (probes with
covariance P, log|P| added to the stochastic log-determinant), and prediction.

Gates as for the unpreconditioned paths: solution within max(1e-4, 2e-8 kappa) of Cholesky; quad
term 1e-4, LML and gradient 1e-3 of the oracle's FP64 run of the same preconditioned estimator
(same pivots, same probes) and of its probe-conditioned targets.
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


@pytest.mark.parametrize("kind,D", [(wl.RBF, 2), (wl.MATERN52, 3), (wl.MATERN12, 2)])
def test_preconditioned_solve(lgp, kind, D):
    p = wl.random_problem(2500, D, kind, seed=900 + kind, log_noise=math.log(0.01))
    B = wl.rhs_block(p.N, 8, seed=9)
    B[:, 0] = p.y
    hyp = go.hyper_of(p)
    Ky = go.noisy_kernel_matrix(p.X, hyp)
    ev = np.linalg.eigvalsh(Ky)
    gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
    ref = go.cholesky_solve(Ky, B.astype(np.float64))
    x0, it0, rel0, s0 = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=5000)
    x1, it1, rel1, s1 = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=5000, precond_rank=20)
    assert s0 == lgp.LGP_OK and s1 == lgp.LGP_OK
    assert (rel1 <= 1e-6).all()
    err = np.linalg.norm(x1.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    print(f"kind={kind} D={D} kappa={ev[-1] / ev[0]:.1e}: iterations plain {it0.max()} preconditioned {it1.max()}, "
          f"err {err.max():.2e} (gate {gate:.1e})")
    assert err.max() <= gate
    assert it1.max() < it0.max()


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN32])
def test_preconditioned_lml_and_grad(lgp, kind):
    # a moderately conditioned problem (kappa(K_y) ~ 1e3): the float32 solves then carry errors well below
    # the 1e-3 gate, as in the unpreconditioned LML test (at kappa ~ 1e5 both float32 and float64 CG stop at
    # recursive residual 1e-6 with solutions that differ by up to kappa * 1e-6)
    p = wl.random_problem(1500, 3, kind, seed=950 + kind, lo=0.08, hi=0.2, log_noise=math.log(0.05))
    hyp = go.hyper_of(p)
    ev = np.linalg.eigvalsh(go.noisy_kernel_matrix(p.X, hyp))
    assert ev[-1] / ev[0] < 1e4
    m, L, seed, tol, k = 15, 60, 321, 1e-6, 12
    lml, grad, info = lgp.lgp_lml_and_grad(_dev(p.X), _dev(p.y), p, n_probes=m, lanczos_steps=L, seed=seed, tol=tol,
                                           max_iter=3000, precond_rank=k)
    est = go.estimator_precond_fp64(p.X, p.y, hyp, rank=k, n_probes=m, lanczos_steps=L, seed=seed, tol=tol,
                                    max_iter=3000)
    tg = go.precond_probe_targets(p.X, p.y, hyp, est["L"], est["Z"])
    plain = go.estimator_fp64(p.X, p.y, hyp, n_probes=m, lanczos_steps=L, seed=seed, tol=tol, max_iter=3000)
    exact = go.lml(p.X, p.y, hyp)
    print(f"kind={kind} kappa={ev[-1] / ev[0]:.1e}: lml gpu {lml:.6f} fp64-est {est['lml']:.6f} target "
          f"{tg['lml']:.6f} exact {exact:.6f}; iters gpu {info['iters_max']} fp64 {est['iters'].max()} "
          f"plain {plain['iters'].max()}")
    assert info["logdet_precond"] == pytest.approx(go.precond_logdet(est["L"], hyp.noise), rel=1e-9)
    assert info["quad"] == pytest.approx(tg["quad"], rel=1e-4)
    assert lml == pytest.approx(est["lml"], rel=1e-3)
    assert info["logdet"] == pytest.approx(est["logdet"], abs=1e-3 * abs(est["lml"]))
    scale = np.maximum(np.abs(tg["grad"]), 1e-2 * np.abs(tg["grad"]).max())
    eg_t = (np.abs(np.asarray(grad) - tg["grad"]) / scale).max()
    eg_e = (np.abs(np.asarray(grad) - est["grad"]) / scale).max()
    print(f"kind={kind}: grad err vs target {eg_t:.2e} vs fp64 estimator {eg_e:.2e}; "
          f"lml err {abs(lml - est['lml']) / abs(est['lml']):.2e}")
    assert eg_t <= 1e-3
    assert eg_e <= 1e-3


def test_preconditioned_prediction(lgp):
    p = wl.random_problem(1600, 2, wl.MATERN52, seed=970, log_noise=math.log(0.01))
    hyp = go.hyper_of(p)
    Xs = np.random.default_rng(971).uniform(0.0, 1.0, (40, 2)).astype(np.float32)
    mean, var, info, s = lgp.lgp_predict(_dev(p.X), _dev(p.y), p, _dev(Xs), tol=1e-7, max_iter=5000, precond_rank=16)
    assert s == lgp.LGP_OK
    m_ref, v_ref = go.predict_exact(p.X, p.y, Xs, hyp)
    Ky = go.noisy_kernel_matrix(p.X, hyp)
    ev = np.linalg.eigvalsh(Ky)
    gate = max(1e-5, 1e-7 * ev[-1] / ev[0])
    Ksf = go.cross_kernel(Xs, p.X, hyp)
    scale = np.abs(Ksf) @ np.abs(go.cholesky_solve(Ky, p.y.astype(np.float64)))
    assert np.max(np.abs(mean.cpu().numpy() - m_ref) / scale) <= gate
    assert np.abs(var.cpu().numpy() - v_ref).max() <= gate * hyp.s2


def test_preconditioner_argument_checks(lgp):
    p = wl.random_problem(400, 2, wl.RBF, seed=980)
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(_dev(p.X), p, _dev(wl.rhs_block(p.N, 2, seed=1)), precond_rank=33)
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(_dev(p.X), p, _dev(wl.rhs_block(p.N, 40, seed=1)), precond_rank=8)
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED
    # rank above the number of points: the extra columns stay zero and the solve still converges
    q = wl.random_problem(20, 2, wl.MATERN12, seed=981)
    x, it, rel, s = lgp.lgp_cg_solve(_dev(q.X), q, _dev(q.y[:, None]), tol=1e-6, precond_rank=32)
    ref = go.cholesky_solve(go.noisy_kernel_matrix(q.X, go.hyper_of(q)), q.y.astype(np.float64))
    assert s == lgp.LGP_OK and it[0] <= 3
    assert np.linalg.norm(x.cpu().numpy()[:, 0] - ref) / np.linalg.norm(ref) <= 1e-4


@pytest.mark.parametrize("rank", [0, 12])
def test_warm_start(lgp, rank):
    """A warm start from a nearby solution takes fewer iterations and reaches the same solution; from the
    converged solution itself, no column iterates."""
    p = wl.random_problem(2000, 3, wl.MATERN52, seed=990, log_noise=math.log(0.02))
    B = wl.rhs_block(p.N, 4, seed=990)
    hyp = go.hyper_of(p)
    ref = go.cholesky_solve(go.noisy_kernel_matrix(p.X, hyp), B.astype(np.float64))
    x_cold, it_cold, _, s = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=4000, precond_rank=rank)
    assert s == lgp.LGP_OK
    near = (ref * (1.0 + 1e-3 * np.random.default_rng(1).standard_normal(ref.shape))).astype(np.float32)
    x_warm, it_warm, rel, s = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=4000, precond_rank=rank,
                                               x0=_dev(near))
    assert s == lgp.LGP_OK and (rel <= 1e-6).all()
    assert it_warm.max() < it_cold.max()
    e_cold = np.linalg.norm(x_cold.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    e_warm = np.linalg.norm(x_warm.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    print(f"rank {rank}: iterations cold {it_cold.max()} warm {it_warm.max()}; err {e_cold.max():.2e} / {e_warm.max():.2e}")
    assert e_warm.max() <= max(2.0 * e_cold.max(), 1e-5)
    # the float32 true residual of the converged solution is well above its recursive 1e-6: use a tolerance
    # it meets
    x_same, it_same, _, s = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-2, max_iter=4000, precond_rank=rank,
                                             x0=x_cold)
    assert s == lgp.LGP_OK and it_same.max() == 0
    np.testing.assert_array_equal(x_same.cpu().numpy(), x_cold.cpu().numpy())
