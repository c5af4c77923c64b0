"""Posterior prediction (Sec. 2: mu_* = K_*f K_y^-1 y, var_* = diag(K_** - K_*f K_y^-1 K_f*)) through
lgp_predict, against the FP64 oracle.

Gates. The solves run float32 CG to relative residual tol = 1e-7, and a solve whose relative
residual is tol has a relative forward error up to kappa(K_y) tol. The gate is therefore
g = max(1e-5, kappa tol), with kappa from the oracle's eigenvalues:
- mean: |mu_i - mu*_i| <= g (|K_*f| |a*|)_i, the size of the terms that the mean sums
  (a* = K_y^-1 y), since a mean can be a small difference of large terms;
- variance: |var_i - var*_i| <= g s^2.
The probe variance is gated the same way against its probe-conditioned target (the value the
estimate takes for the same probes with exact solves); its distance to the exact variance is the
estimator's own sampling error and is only reported.
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


def _case(kind, N, M, D=3, seed=0, log_noise=math.log(0.1)):
    p = wl.random_problem(N, D, kind, seed=seed, log_noise=log_noise)
    Xs = np.random.default_rng(seed + 1).uniform(0.0, 1.0, (M, D)).astype(np.float32)
    hyp = go.hyper_of(p)
    Ky = go.noisy_kernel_matrix(p.X, hyp)
    ev = np.linalg.eigvalsh(Ky)
    return p, Xs, hyp, ev[-1] / ev[0]


TOL = 1e-7


def _gate(kappa):
    return max(1e-5, kappa * TOL)


def _mean_err(mean, X, y, Xs, hyp):
    """max_i |mu_i - mu*_i| / (|K_*f| |a*|)_i."""
    Ksf = go.cross_kernel(Xs, X, hyp)
    a = go.cholesky_solve(go.noisy_kernel_matrix(X, hyp), np.asarray(y, dtype=np.float64))
    m_ref = Ksf @ a
    scale = np.abs(Ksf) @ np.abs(a)
    diff = np.abs(np.asarray(mean, dtype=np.float64) - m_ref)
    # a test point with no kernel mass (far from every input) has mean 0 exactly: compare absolutely
    return float(np.max(np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)))


@pytest.mark.parametrize("M", [1, 7, 31, 32, 100])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52, wl.MATERN32, wl.MATERN12])
def test_predict_exact_variance(lgp, kind, M):
    p, Xs, hyp, kappa = _case(kind, 1200, M, seed=10 * kind + M)
    mean, var, info, s = lgp.lgp_predict(_dev(p.X), _dev(p.y), p, _dev(Xs), tol=TOL, max_iter=4000)
    assert s == lgp.LGP_OK
    m_ref, v_ref = go.predict_exact(p.X, p.y, Xs, hyp)
    mean, var = mean.cpu().numpy().astype(np.float64), var.cpu().numpy().astype(np.float64)
    em = _mean_err(mean, p.X, p.y, Xs, hyp)
    ev = np.abs(var - v_ref).max() / hyp.s2
    print(f"kind={kind} M={M} kappa={kappa:.0f} mean err {em:.2e} var err {ev:.2e} solves {info['solves']} "
          f"iters {info['iters_max']}")
    assert em <= _gate(kappa)
    assert ev <= _gate(kappa)
    assert info["solves"] == 1 + max(0, math.ceil((M - 31) / 32))
    assert info["var_probes"] == 0


@pytest.mark.parametrize("m", [15, 31])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN32])
def test_predict_probe_variance(lgp, kind, m):
    p, Xs, hyp, kappa = _case(kind, 1500, 200, seed=70 + m)
    seed = 1234
    mean, var, info, s = lgp.lgp_predict(_dev(p.X), _dev(p.y), p, _dev(Xs), n_probes=m, seed=seed, tol=TOL,
                                         max_iter=4000)
    assert s == lgp.LGP_OK and info["solves"] == 1 and info["var_probes"] == m
    Z = go.rademacher(seed, Xs.shape[0], m)
    target = go.predict_var_hutchinson_target(p.X, Xs, hyp, Z)
    m_ref, v_ref = go.predict_exact(p.X, p.y, Xs, hyp)
    mean, var = mean.cpu().numpy().astype(np.float64), var.cpu().numpy().astype(np.float64)
    assert _mean_err(mean, p.X, p.y, Xs, hyp) <= _gate(kappa)
    et = np.abs(var - target).max() / hyp.s2
    print(f"kind={kind} m={m}: vs probe target {et:.2e}, vs exact variance {np.abs(var - v_ref).max():.2e}")
    assert et <= _gate(kappa)


def test_predict_mean_only_and_limits(lgp):
    """var = NULL runs one single-column solve. A far test point gets the prior (mean 0, variance s^2);
    a test point on a training input gets a variance below the noise level."""
    p, Xs, hyp, kappa = _case(wl.MATERN52, 900, 3, seed=5)
    Xs[0] = 1e4
    Xs[1] = p.X[17]
    mean, var, info, s = lgp.lgp_predict(_dev(p.X), _dev(p.y), p, _dev(Xs), want_var=False, tol=TOL)
    assert var is None and info["solves"] == 1 and s == lgp.LGP_OK
    m_ref, v_ref = go.predict_exact(p.X, p.y, Xs, hyp)
    assert _mean_err(mean.cpu().numpy(), p.X, p.y, Xs, hyp) <= _gate(kappa)
    mean, var, info, s = lgp.lgp_predict(_dev(p.X), _dev(p.y), p, _dev(Xs), tol=TOL)
    var = var.cpu().numpy()
    assert abs(mean.cpu().numpy()[0]) < 1e-6
    assert var[0] == pytest.approx(hyp.s2, rel=1e-6)
    assert 0.0 <= v_ref[1] < hyp.noise and abs(var[1] - v_ref[1]) <= _gate(kappa) * hyp.s2


def test_predict_errors(lgp):
    import torch
    p, Xs, hyp, _ = _case(wl.RBF, 300, 4, seed=6)
    X, y, Xd = _dev(p.X), _dev(p.y), _dev(Xs)
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_predict(X, y, p, Xd, n_probes=32)
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_predict(X, y, p, Xd[:0])
    assert e.value.status == lgp.LGP_ERR_INVALID_ARG
    bad = Xs.copy()
    bad[2, 1] = np.nan
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_predict(X, y, p, _dev(bad))
    assert e.value.status == lgp.LGP_ERR_NONFINITE
    # the context stays usable
    mean, var, _, s = lgp.lgp_predict(X, y, p, Xd)
    torch.cuda.synchronize()
    assert s == lgp.LGP_OK and torch.isfinite(var).all()
