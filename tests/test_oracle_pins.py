"""Pins for the FP64 oracle: checks against facts fixed outside the oracle itself.

Each test compares an oracle routine with something it does not share code
with: a published constant or test vector (tests/golden), a library routine
computing the same quantity from another definition (SciPy densities, Bessel
functions, LAPACK log-determinants), a brute-force loop, a finite difference,
or an identity (Hadamard probes make Hutchinson exact; full-length Lanczos
makes Gauss quadrature exact).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as sp
import scipy.stats as st

import oracle
from oracle import gp_oracle as go
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hyp(kind, D, seed=0, los=0.3, ln=math.log(0.05)):
    rng = np.random.default_rng(seed)
    return go.Hyper(kind, np.log(rng.uniform(0.3, 2.0, D)), los, ln)


def _points(N, D, seed=0):
    return np.random.default_rng(seed + 100).uniform(0, 1, (N, D))


# ----------------------------------------------------------------------------- kernel entries

def test_kernel_closed_form_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "kernel_values.txt")) if l.strip() and l[0] != "#"]
    kinds = {"rbf": go.RBF, "m52": go.MATERN52, "m12": go.MATERN12, "m32": go.MATERN32}
    assert set(n for n, _, _ in rows) == set(kinds)
    for name, r, val in rows:
        kind = kinds[name]
        got = go.phi(kind, np.array([float(r) ** 2]))[0]
        assert got == pytest.approx(float(val), rel=1e-14, abs=1e-15), (name, r)


def test_rbf_is_gaussian_density_ratio():
    """ARD RBF = N(x; x', diag l^2) / N(x'; x', diag l^2) (SciPy's density, another definition)."""
    D = 3
    hyp = _hyp(go.RBF, D, seed=1, los=0.0)
    X = _points(6, D, seed=1)
    K = go.kernel_matrix(X, hyp)
    for i in range(6):
        mvn = st.multivariate_normal(mean=X[i], cov=np.diag(hyp.lengthscale ** 2))
        ref = mvn.pdf(X) / mvn.pdf(X[i])
        np.testing.assert_allclose(K[i], ref, rtol=1e-12)


@pytest.mark.parametrize("nu,kind", [(2.5, go.MATERN52), (1.5, go.MATERN32), (0.5, go.MATERN12)])
def test_matern_is_bessel_form(nu, kind):
    """Matern nu in {1/2, 3/2, 5/2} from the modified Bessel function K_nu (Rasmussen & Williams Eq. 4.14)."""
    r = np.linspace(0.01, 6.0, 200)
    z = math.sqrt(2 * nu) * r
    ref = 2 ** (1 - nu) / sp.gamma(nu) * z ** nu * sp.kv(nu, z)
    np.testing.assert_allclose(go.phi(kind, r * r), ref, rtol=1e-12)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_lengthscale_coefficient_is_a_derivative(kind):
    """d phi / d log l = c(r^2) r^2 for a 1-D problem (so r_d = r): central FD of phi(r^2 e^{-2u})."""
    r = np.linspace(0.05, 4.0, 60)
    h = 1e-6
    fd = (go.phi(kind, (r * math.exp(-h)) ** 2) - go.phi(kind, (r * math.exp(h)) ** 2)) / (2 * h)
    np.testing.assert_allclose(go.lengthscale_coef(kind, r * r) * r * r, fd, rtol=1e-7, atol=1e-10)
    assert go.lengthscale_coef(kind, np.array([0.0]))[0] >= 0.0  # finite (0 for M12) at r = 0


def test_ard_scaling_and_outputscale():
    hyp = go.Hyper(go.MATERN52, np.log([2.0, 0.5]), math.log(3.0), math.log(0.1))
    X = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 0.5]])
    K = go.kernel_matrix(X, hyp)
    # both off-diagonal pairs sit at ARD distance exactly 1; diagonal is s^2
    expect = 3.0 * (1 + math.sqrt(5) + 5 / 3) * math.exp(-math.sqrt(5))
    assert K[0, 1] == pytest.approx(expect, rel=1e-14)
    assert K[0, 2] == pytest.approx(expect, rel=1e-14)
    assert K[0, 0] == pytest.approx(3.0, rel=1e-15)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_symmetric_and_psd(kind):
    hyp = _hyp(kind, 4, seed=2)
    X = _points(120, 4, seed=2)
    Ky = go.noisy_kernel_matrix(X, hyp)
    assert np.array_equal(Ky, Ky.T)
    assert np.linalg.eigvalsh(Ky).min() >= hyp.noise * (1 - 1e-10)


# ----------------------------------------------------------------------------- products

@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_matvec_bruteforce_loop(kind):
    N, D, t = 23, 3, 2
    hyp = _hyp(kind, D, seed=3)
    X = _points(N, D, seed=3)
    V = np.random.default_rng(3).standard_normal((N, t))
    ls = hyp.lengthscale
    ref = np.zeros((N, t))
    for i in range(N):
        for j in range(N):
            r2 = sum(((X[i, d] - X[j, d]) / ls[d]) ** 2 for d in range(D))
            r = math.sqrt(r2)
            if kind == go.RBF:
                k = hyp.s2 * math.exp(-r2 / 2)
            elif kind == go.MATERN52:
                k = hyp.s2 * (1 + math.sqrt(5) * r + 5 * r2 / 3) * math.exp(-math.sqrt(5) * r)
            elif kind == go.MATERN32:
                k = hyp.s2 * (1 + math.sqrt(3) * r) * math.exp(-math.sqrt(3) * r)
            else:
                k = hyp.s2 * math.exp(-r)
            if i == j:
                k += hyp.noise
            for c in range(t):
                ref[i, c] += k * V[j, c]
    np.testing.assert_allclose(go.matvec(X, V, hyp, block=7), ref, rtol=1e-13, atol=1e-13)
    rows = [0, 5, 22]
    np.testing.assert_allclose(go.matvec_rows(X, V, hyp, rows), ref[rows], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_c_streaming_oracle_matches_dense(kind):
    N, D, t = 300, 5, 3
    hyp = _hyp(kind, D, seed=4)
    X = _points(N, D, seed=4).astype(np.float32)
    V = np.random.default_rng(4).standard_normal((N, t)).astype(np.float32)
    ref = go.matvec(X, V, hyp)
    got, used = oracle.kyv_rows_c(X, V, hyp)
    assert used >= 1
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    rows = np.array([299, 0, 17])
    got_r, _ = oracle.kyv_rows_c(X, V, hyp, rows=rows)
    np.testing.assert_allclose(got_r, ref[rows], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_dK_matvec_matches_finite_difference_of_K(kind):
    hyp = _hyp(kind, 2, seed=5)
    X = _points(30, 2, seed=5)
    W = np.random.default_rng(5).standard_normal((30, 2))
    G = go.dK_matvec(X, W, hyp)
    theta = np.concatenate([hyp.log_lengthscale, [hyp.log_outputscale, hyp.log_noise]])
    h = 1e-6
    for p in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        Kp = go.noisy_kernel_matrix(X, go.Hyper(hyp.kind, tp[:-2], tp[-2], tp[-1]))
        Km = go.noisy_kernel_matrix(X, go.Hyper(hyp.kind, tm[:-2], tm[-2], tm[-1]))
        np.testing.assert_allclose(G[p], (Kp - Km) @ W / (2 * h), rtol=1e-6, atol=1e-8)


# ----------------------------------------------------------------------------- exact inference

def test_cg_matches_cholesky_solve():
    hyp = _hyp(go.RBF, 3, seed=6, ln=math.log(0.1))
    X = _points(150, 3, seed=6)
    Ky = go.noisy_kernel_matrix(X, hyp)
    B = np.random.default_rng(6).standard_normal((150, 3))
    res = go.cg(lambda P: Ky @ P, B, 1e-12, 2000)
    ref = go.cholesky_solve(Ky, B)
    np.testing.assert_allclose(res.x, ref, rtol=1e-8, atol=1e-8)
    assert np.linalg.norm(B - Ky @ ref) <= 1e-10 * np.linalg.norm(B)
    assert (res.rel_resid <= 1e-12).all()


def test_logdet_three_ways():
    hyp = _hyp(go.MATERN52, 3, seed=7)
    Ky = go.noisy_kernel_matrix(_points(100, 3, seed=7), hyp)
    a = go.logdet(Ky)
    b = float(np.sum(np.log(np.linalg.eigvalsh(Ky))))
    sign, c = np.linalg.slogdet(Ky)
    assert sign == 1.0
    assert a == pytest.approx(b, rel=1e-10)
    assert a == pytest.approx(c, rel=1e-10)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_lml_is_gaussian_logpdf(kind):
    hyp = _hyp(kind, 2, seed=8)
    X = _points(60, 2, seed=8)
    y = np.random.default_rng(8).standard_normal(60)
    Ky = go.noisy_kernel_matrix(X, hyp)
    ref = st.multivariate_normal(mean=np.zeros(60), cov=Ky).logpdf(y)
    assert go.lml(X, y, hyp) == pytest.approx(ref, rel=1e-11)


def test_lml_single_point_closed_form():
    hyp = go.Hyper(go.RBF, np.array([0.3]), math.log(2.0), math.log(0.5))
    y = np.array([1.7])
    v = 2.0 + 0.5
    ref = -0.5 * (1.7 ** 2 / v + math.log(v) + math.log(2 * math.pi))
    assert go.lml(np.array([[0.4]]), y, hyp) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_gradient_matches_central_fd(kind):
    D = 3
    hyp = _hyp(kind, D, seed=9)
    X = _points(80, D, seed=9)
    y = np.sin(4 * X[:, 0]) + 0.1 * np.random.default_rng(9).standard_normal(80)
    g = go.grad_exact(X, y, hyp)
    theta = np.concatenate([hyp.log_lengthscale, [hyp.log_outputscale, hyp.log_noise]])
    h = 1e-5
    fd = []
    for p in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fp = go.lml(X, y, go.Hyper(kind, tp[:D], tp[D], tp[D + 1]))
        fm = go.lml(X, y, go.Hyper(kind, tm[:D], tm[D], tm[D + 1]))
        fd.append((fp - fm) / (2 * h))
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_noise_gradient_closed_form():
    hyp = _hyp(go.RBF, 2, seed=10)
    X = _points(50, 2, seed=10)
    y = np.random.default_rng(10).standard_normal(50)
    Ky = go.noisy_kernel_matrix(X, hyp)
    a = np.linalg.solve(Ky, y)
    ref = 0.5 * hyp.noise * (a @ a - np.trace(np.linalg.inv(Ky)))
    assert go.grad_exact(X, y, hyp)[-1] == pytest.approx(ref, rel=1e-10)


# ----------------------------------------------------------------------------- probes and estimators

def test_splitmix64_reference_vector():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.strip() and l[0] != "#"]
    state = 0
    for idx, hexval in rows:
        assert go.splitmix64(state) == int(hexval, 16), idx
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)


def test_rademacher_keying_and_balance():
    seed = 0x1234ABCD5678
    Z = go.rademacher(seed, 4096, 5)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    for (i, c) in [(0, 0), (4095, 4), (17, 3), (1000, 1)]:
        bit = go.splitmix64(seed ^ ((c << 32) | i)) >> 63
        assert Z[i, c] == 1.0 - 2.0 * bit
    assert abs(Z.mean()) < 0.03


def test_hadamard_probes_make_estimators_exact():
    """With all N Hadamard columns as probes, Hutchinson traces are exact (Z Z^T = N I)."""
    N = 64
    hyp = _hyp(go.MATERN52, 2, seed=11)
    X = _points(N, 2, seed=11)
    y = np.random.default_rng(11).standard_normal(N)
    H = sla.hadamard(N).astype(np.float64)
    tg = go.probe_conditioned_targets(X, y, hyp, H)
    assert tg["logdet"] == pytest.approx(tg["logdet_exact"], rel=1e-10)
    np.testing.assert_allclose(tg["grad"], go.grad_exact(X, y, hyp), rtol=1e-9, atol=1e-10)
    assert tg["lml"] == pytest.approx(go.lml(X, y, hyp), rel=1e-10)


def test_full_length_lanczos_quadrature_is_exact():
    """N Lanczos steps make Gauss quadrature exact: ||z||^2 e1^T log(T) e1 = z^T log(A) z."""
    N = 24
    hyp = _hyp(go.RBF, 2, seed=12, ln=math.log(0.5))
    Ky = go.noisy_kernel_matrix(_points(N, 2, seed=12), hyp)
    z = go.rademacher(99, N, 1)[:, 0]
    lam, Q = np.linalg.eigh(Ky)
    ref = float(np.sum((Q.T @ z) ** 2 * np.log(lam)))
    T = go.lanczos_full_reorth(Ky, z, N)
    assert go.quadrature_logdet(T, float(z @ z)) == pytest.approx(ref, rel=1e-9)
    res = go.cg(lambda P: Ky @ P, z, 1e-14, N)
    m = int(res.iters[0])
    Tc = go.lanczos_tridiag_from_cg(res.alphas[:, 0], res.betas[:, 0], m)
    assert go.quadrature_logdet(Tc, float(z @ z)) == pytest.approx(ref, rel=1e-7)


def test_cg_coefficients_give_the_lanczos_tridiagonal():
    """The tridiagonal from CG coefficients equals the one Lanczos builds directly.

    Checked over the first steps, before the Krylov space has captured the few
    large eigenvalues of K_y and the recurrences become dominated by rounding.
    """
    N, m = 200, 6
    hyp = _hyp(go.MATERN52, 3, seed=13, ln=math.log(0.2))
    Ky = go.noisy_kernel_matrix(_points(N, 3, seed=13), hyp)
    z = go.rademacher(5, N, 1)[:, 0]
    res = go.cg(lambda P: Ky @ P, z, 1e-14, m)
    Tc = go.lanczos_tridiag_from_cg(res.alphas[:, 0], res.betas[:, 0], m)
    Tl = go.lanczos_full_reorth(Ky, z, m)
    np.testing.assert_allclose(np.diag(Tc), np.diag(Tl), rtol=1e-8)
    np.testing.assert_allclose(np.abs(np.diag(Tc, 1)), np.abs(np.diag(Tl, 1)), rtol=1e-7)


def test_fp64_estimator_hits_probe_conditioned_targets():
    """Converged FP64 mBCG + SLQ with enough steps reproduces the probe-conditioned targets."""
    p = wl.cfg3(N=400, t=9, seed=14)
    hyp = go.hyper_of(p)
    est = go.estimator_fp64(p.X, p.y, hyp, n_probes=8, lanczos_steps=400, seed=77, tol=1e-12, max_iter=400)
    tg = go.probe_conditioned_targets(p.X, p.y, hyp, est["Z"])
    assert est["quad"] == pytest.approx(tg["quad"], rel=1e-8)
    assert est["logdet"] == pytest.approx(tg["logdet"], rel=1e-6)
    np.testing.assert_allclose(est["grad"], tg["grad"], rtol=1e-6, atol=1e-6 * np.abs(tg["grad"]).max())


@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_cross_product_bruteforce_loop(kind):
    """K(X*, X) V (the predictive-mean product) from the C oracle against a plain double loop."""
    N, M, D, t = 19, 5, 3, 2
    hyp = _hyp(kind, D, seed=6)
    X = _points(N, D, seed=6).astype(np.float32)
    Xs = _points(M, D, seed=16).astype(np.float32)
    V = np.random.default_rng(6).standard_normal((N, t)).astype(np.float32)
    ls = hyp.lengthscale
    ref = np.zeros((M, t))
    for i in range(M):
        for j in range(N):
            r2 = sum(((float(Xs[i, d]) - float(X[j, d])) / ls[d]) ** 2 for d in range(D))
            k = hyp.s2 * float(go.phi(kind, np.array([r2]))[0])
            for c in range(t):
                ref[i, c] += k * float(V[j, c])
    got, _ = oracle.kxv_c(Xs, X, V, hyp)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(go.cross_kernel(Xs, X, hyp) @ V.astype(np.float64), ref, rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------------------------- posterior prediction

@pytest.mark.parametrize("kind", [go.RBF, go.MATERN52, go.MATERN32, go.MATERN12])
def test_prediction_is_gaussian_conditioning_via_joint_precision(kind):
    """mu_* and var_* against Gaussian conditioning computed another way: from the precision
    matrix P of the joint covariance [[K_y, K_f*], [K_*f, K_**]], Cov(* | y) = inv(P_**) and
    E[* | y] = -inv(P_**) P_*f y (Schur-complement identities)."""
    N, M, D = 40, 9, 2
    hyp = _hyp(kind, D, seed=21)
    X = _points(N, D, seed=21)
    Xs = _points(M, D, seed=22)
    y = np.random.default_rng(21).standard_normal(N)
    A = np.vstack([X, Xs])
    C = go.kernel_matrix(A, hyp)
    C[:N, :N] += hyp.noise * np.eye(N)
    P = np.linalg.inv(C)
    cov = np.linalg.inv(P[N:, N:])
    mean_ref = -cov @ P[N:, :N] @ y
    mean, var = go.predict_exact(X, y, Xs, hyp)
    np.testing.assert_allclose(mean, mean_ref, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(var, np.diag(cov), rtol=1e-7, atol=1e-10)


def test_prediction_limits():
    """Far from the data the posterior is the prior (mean 0, variance s^2); at a training input with
    vanishing noise the mean interpolates y and the latent variance vanishes (Matern-1/2, so that K
    stays well conditioned at sigma^2 = 1e-9)."""
    hyp = _hyp(go.MATERN12, 2, seed=23, los=0.4, ln=math.log(1e-9))
    X = _points(12, 2, seed=23)
    y = np.random.default_rng(23).standard_normal(12)
    far = np.array([[1e3, 1e3]])
    mean, var = go.predict_exact(X, y, far, hyp)
    assert abs(mean[0]) < 1e-12
    assert var[0] == pytest.approx(math.exp(0.4), rel=1e-12)
    mean, var = go.predict_exact(X, y, X[:3], hyp)
    np.testing.assert_allclose(mean, y[:3], rtol=0, atol=1e-5)
    assert np.all(np.abs(var) < 1e-5)


def test_hadamard_probes_make_variance_estimate_exact():
    """With all M Hadamard columns as probes, the diagonal estimator is exact (Z Z^T = M I)."""
    M = 16
    hyp = _hyp(go.MATERN32, 3, seed=24)
    X = _points(50, 3, seed=24)
    Xs = _points(M, 3, seed=25)
    H = sla.hadamard(M).astype(np.float64)
    _, var = go.predict_exact(X, np.zeros(50), Xs, hyp)
    np.testing.assert_allclose(go.predict_var_hutchinson_target(X, Xs, hyp, H), var, rtol=1e-10, atol=1e-12)


def test_prediction_cg_route_reaches_the_exact_values():
    """The float64 CG route (exact-variance mode, and probe mode against its probe target)."""
    hyp = _hyp(go.MATERN52, 3, seed=26)
    X = _points(200, 3, seed=26)
    Xs = _points(21, 3, seed=27)
    y = np.random.default_rng(26).standard_normal(200)
    mean, var = go.predict_exact(X, y, Xs, hyp)
    ex = go.predict_fp64(X, y, Xs, hyp, n_probes=0, seed=0, tol=1e-12)
    np.testing.assert_allclose(ex["mean"], mean, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(ex["var"], var, rtol=1e-8, atol=1e-10)
    pr = go.predict_fp64(X, y, Xs, hyp, n_probes=8, seed=5, tol=1e-12)
    np.testing.assert_allclose(pr["var"], go.predict_var_hutchinson_target(X, Xs, hyp, pr["Z"]), rtol=1e-8,
                               atol=1e-10)


# ----------------------------------------------------------------------------- preconditioning

def test_pivoted_cholesky_full_rank_and_residual_trace():
    """Full rank reproduces K_ff; at lower rank the returned residual diagonal is diag(K - L L^T) and
    its trace falls with the rank (the pivoting rule picks the largest residual each step)."""
    hyp = _hyp(go.MATERN32, 2, seed=31)
    X = _points(18, 2, seed=31)
    K = go.kernel_matrix(X, hyp)
    L, piv, d = go.pivoted_cholesky(X, hyp, 18)
    np.testing.assert_allclose(L @ L.T, K, rtol=0, atol=1e-10)
    assert sorted(piv.tolist()) == list(range(18)) and piv[0] == 0
    prev = np.inf
    for k in (2, 5, 9):
        L, piv, d = go.pivoted_cholesky(X, hyp, k)
        np.testing.assert_allclose(d, np.diag(K - L @ L.T), rtol=0, atol=1e-12)
        assert np.all(d >= -1e-12) and d.sum() < prev
        prev = d.sum()


def test_woodbury_inverse_and_determinant_lemma():
    hyp = _hyp(go.RBF, 3, seed=32)
    X = _points(40, 3, seed=32)
    L, _, _ = go.pivoted_cholesky(X, hyp, 6)
    P = L @ L.T + hyp.noise * np.eye(40)
    R = np.random.default_rng(32).standard_normal((40, 3))
    np.testing.assert_allclose(go.precond_inverse(L, hyp.noise)(R), np.linalg.solve(P, R), rtol=1e-9, atol=1e-9)
    assert go.precond_logdet(L, hyp.noise) == pytest.approx(np.linalg.slogdet(P)[1], rel=1e-12)


def test_pcg_special_cases():
    """Identity preconditioner: the same iterates as CG. Exact preconditioner P = K_y: one step.
    Any preconditioner: the Cholesky solution."""
    hyp = _hyp(go.MATERN52, 2, seed=33)
    X = _points(60, 2, seed=33)
    Ky = go.noisy_kernel_matrix(X, hyp)
    B = np.random.default_rng(33).standard_normal((60, 2))
    a = go.cg(lambda P: Ky @ P, B, 1e-10, 200)
    b = go.pcg(lambda P: Ky @ P, lambda R: np.array(R, dtype=np.float64), B, 1e-10, 200)
    np.testing.assert_allclose(b.x, a.x, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(b.alphas, a.alphas, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b.betas, a.betas, rtol=1e-12, atol=1e-14)
    one = go.pcg(lambda P: Ky @ P, lambda R: np.linalg.solve(Ky, R), B, 1e-10, 200)
    assert one.iters.max() == 1
    L, _, _ = go.pivoted_cholesky(X, hyp, 8)
    pc = go.pcg(lambda P: Ky @ P, go.precond_inverse(L, hyp.noise), B, 1e-12, 500)
    np.testing.assert_allclose(pc.x, go.cholesky_solve(Ky, B), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(pc.rz0, np.sum(B * go.precond_inverse(L, hyp.noise)(B), axis=0), rtol=1e-12)


def test_full_length_preconditioned_quadrature_is_exact():
    """N PCG steps: (z^T P^{-1} z) e1^T log(T) e1 = w^T log(P^{-1/2} K_y P^{-1/2}) w, w = P^{-1/2} z."""
    N = 24
    hyp = _hyp(go.RBF, 2, seed=34, ln=math.log(0.5))
    X = _points(N, 2, seed=34)
    Ky = go.noisy_kernel_matrix(X, hyp)
    L, _, _ = go.pivoted_cholesky(X, hyp, 4)
    z = go.precond_probes(7, L, hyp.noise, 1)
    res = go.pcg(lambda P: Ky @ P, go.precond_inverse(L, hyp.noise), z, 0.0, N)
    T = go.lanczos_tridiag_from_cg(res.alphas[:N, 0], res.betas[:N, 0], N)
    P = L @ L.T + hyp.noise * np.eye(N)
    lam, Q = np.linalg.eigh(P)
    Pm12 = (Q / np.sqrt(lam)) @ Q.T
    mu, V = np.linalg.eigh(Pm12 @ Ky @ Pm12)
    w = Pm12 @ z[:, 0]
    ref = float(np.sum((V.T @ w) ** 2 * np.log(mu)))
    assert go.quadrature_logdet(T, float(res.rz0[0])) == pytest.approx(ref, rel=1e-8)


def test_hadamard_probes_make_preconditioned_estimators_exact():
    """z = [sigma I, L] e over all N + k Hadamard columns e: z z^T averages to P, so the probe targets
    are the exact log-determinant and gradient."""
    N, k = 58, 6
    hyp = _hyp(go.MATERN32, 2, seed=35)
    X = _points(N, 2, seed=35)
    y = np.random.default_rng(35).standard_normal(N)
    L, _, _ = go.pivoted_cholesky(X, hyp, k)
    H = sla.hadamard(N + k).astype(np.float64)
    Z = L @ H[N:] + math.sqrt(hyp.noise) * H[:N]
    tg = go.precond_probe_targets(X, y, hyp, L, Z)
    assert tg["logdet"] == pytest.approx(go.logdet(go.noisy_kernel_matrix(X, hyp)), rel=1e-10)
    np.testing.assert_allclose(tg["grad"], go.grad_exact(X, y, hyp), rtol=1e-8, atol=1e-9)


def test_preconditioned_fp64_estimator_hits_its_probe_targets():
    hyp = _hyp(go.RBF, 3, seed=36, ln=math.log(0.01))
    X = _points(150, 3, seed=36)
    y = np.random.default_rng(36).standard_normal(150)
    est = go.estimator_precond_fp64(X, y, hyp, rank=8, n_probes=6, lanczos_steps=150, seed=9, tol=1e-11,
                                    max_iter=2000)
    tg = go.precond_probe_targets(X, y, hyp, est["L"], est["Z"])
    assert est["logdet"] == pytest.approx(tg["logdet"], rel=1e-8)
    np.testing.assert_allclose(est["grad"], tg["grad"], rtol=1e-6, atol=1e-6 * np.abs(tg["grad"]).max())
