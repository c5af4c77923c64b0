"""FP64 CPU oracle for matrix-free GP inference (test infrastructure only).

This module is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the CUDA library never
does, and it shares no code, table or constant with the CUDA path. Inputs are
the float32 arrays handed to the GPU, promoted to float64, so input rounding is
not counted as error.

What it computes, in the paper's notation (Sec. 2 Background):

* ``K_y = K_ff + sigma_n^2 I`` and the product ``K_y V`` (the fused product of
  Sec. 3 "GPU backends" and Table 3, here written out as an explicit matrix).
* the exact solve ``K_y^{-1} B`` by Cholesky (Sec. 2 "Exact inference"),
* ``log|K_y|`` and the log marginal likelihood
  ``log p(y|X) = -1/2 [y^T K_y^{-1} y + log|K_y| + N log 2 pi]`` (Sec. 2),
* the exact hyperparameter gradient ``1/2 tr((a a^T - K_y^{-1}) dK/dtheta)``
  (the quantity the paper approximates by 2P+1 finite-difference fits, Sec. 5),
* textbook unpreconditioned CG from x0 = 0 (Sec. 3 "Inference", Sec. 5 "our
  simpler CG loop") with its coefficients, the Lanczos tridiagonal they define,
  and the stochastic Lanczos log-determinant over Rademacher probes
  (Sec. 3 "CG with stochastic Lanczos log-determinant", Sec. 4.3 probes),
* the probe-conditioned targets of the two stochastic estimators (the values
  the estimators converge to for the given probes as the Lanczos steps grow).

Readings of points the paper leaves open (the paper names the kernels in
Sec. 3 "Kernels" but prints no formula):

* RBF: ``k = s^2 exp(-r^2 / 2)``, ``r^2 = sum_d ((x_d - x'_d) / l_d)^2``.
* Matern-5/2: ``k = s^2 (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r)``.
* Matern-3/2: ``k = s^2 (1 + sqrt3 r) exp(-sqrt3 r)``.
* Matern-1/2: ``k = s^2 exp(-r)``.
  (The Matern family of Sec. 3 "Kernels", nu in {1/2, 3/2, 5/2}, in the standard
  half-integer closed forms of the Bessel definition, Rasmussen & Williams Eq. 4.14-4.17.)
* Hyperparameters live in log space in the order
  ``(log l_1..log l_D, log s^2, log sigma^2)``; zero prior mean.
* Probes: ``z[i, c] = +1`` if bit 63 of ``splitmix64(seed XOR (c * 2^32 + i))``
  is 0, else ``-1`` (splitmix64: Steele, Lea & Flood, OOPSLA 2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

RBF = 0
MATERN52 = 1
MATERN12 = 2
MATERN32 = 3
KINDS = (RBF, MATERN52, MATERN12, MATERN32)
SQRT5 = math.sqrt(5.0)
SQRT3 = math.sqrt(3.0)


@dataclass
class Hyper:
    kind: int
    log_lengthscale: np.ndarray
    log_outputscale: float
    log_noise: float

    @property
    def lengthscale(self) -> np.ndarray:
        return np.exp(np.asarray(self.log_lengthscale, dtype=np.float64))

    @property
    def s2(self) -> float:
        return math.exp(float(self.log_outputscale))

    @property
    def noise(self) -> float:
        return math.exp(float(self.log_noise))

    @property
    def P(self) -> int:
        return len(self.log_lengthscale) + 2


def hyper_of(p) -> Hyper:
    """Hyperparameters of any object with kind / log_lengthscale / log_outputscale / log_noise."""
    return Hyper(int(p.kind), np.asarray(p.log_lengthscale, dtype=np.float64).copy(),
                 float(p.log_outputscale), float(p.log_noise))


# --------------------------------------------------------------------------- kernel entries

def phi(kind: int, r2: np.ndarray) -> np.ndarray:
    """Unit-variance kernel profile as a function of the squared ARD distance r^2."""
    r2 = np.asarray(r2, dtype=np.float64)
    if kind == RBF:
        return np.exp(-0.5 * r2)
    if kind == MATERN52:
        r = np.sqrt(r2)
        return (1.0 + SQRT5 * r + (5.0 / 3.0) * r2) * np.exp(-SQRT5 * r)
    if kind == MATERN32:
        r = np.sqrt(r2)
        return (1.0 + SQRT3 * r) * np.exp(-SQRT3 * r)
    if kind == MATERN12:
        return np.exp(-np.sqrt(r2))
    raise ValueError(f"unknown kernel kind {kind}")


def lengthscale_coef(kind: int, r2: np.ndarray) -> np.ndarray:
    """c(r^2) with d phi / d log l_d = c(r^2) * ((x_d - x'_d) / l_d)^2, i.e. c = -2 d phi / d r^2.

    d r^2 / d log l_d = -2 ((x_d - x'_d) / l_d)^2, so c = -2 dphi/dr^2:
      RBF exp(-r^2/2); M52 (5/3)(1 + sqrt5 r) exp(-sqrt5 r); M32 3 exp(-sqrt3 r);
      M12 exp(-r) / r, which is unbounded at r = 0 where every ((x_d - x'_d)/l_d)^2 is 0 and the
      derivative is 0 (|(x_d - x'_d)/l_d|^2 / r <= r): c is set to 0 there.
    """
    r2 = np.asarray(r2, dtype=np.float64)
    if kind == MATERN12:
        r = np.sqrt(r2)
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(r > 0.0, np.exp(-r) / np.where(r > 0.0, r, 1.0), 0.0)
    return -2.0 * dphi_dr2(kind, r2)


def dphi_dr2(kind: int, r2: np.ndarray) -> np.ndarray:
    """Derivative of ``phi`` with respect to r^2 (chain rule for the lengthscale gradient)."""
    r2 = np.asarray(r2, dtype=np.float64)
    if kind == RBF:
        return -0.5 * np.exp(-0.5 * r2)
    if kind == MATERN52:
        # d phi / d r = -(5/3) r (1 + sqrt5 r) exp(-sqrt5 r);  d r / d r^2 = 1 / (2 r)
        r = np.sqrt(r2)
        return -(5.0 / 6.0) * (1.0 + SQRT5 * r) * np.exp(-SQRT5 * r)
    if kind == MATERN32:
        # d phi / d r = -3 r exp(-sqrt3 r)
        return -1.5 * np.exp(-SQRT3 * np.sqrt(r2))
    if kind == MATERN12:
        # d phi / d r = -exp(-r): unbounded in r^2 at r = 0 (see lengthscale_coef)
        r = np.sqrt(r2)
        return -np.exp(-r) / (2.0 * r)
    raise ValueError(f"unknown kernel kind {kind}")


def scaled_sqdist(Xa: np.ndarray, Xb: np.ndarray, lengthscale: np.ndarray) -> np.ndarray:
    """r^2[i, j] = sum_d ((Xa[i, d] - Xb[j, d]) / l_d)^2 in float64, one dimension at a time."""
    Xa = np.asarray(Xa, dtype=np.float64)
    Xb = np.asarray(Xb, dtype=np.float64)
    r2 = np.zeros((Xa.shape[0], Xb.shape[0]))
    for d in range(Xa.shape[1]):
        diff = (Xa[:, d][:, None] - Xb[:, d][None, :]) / lengthscale[d]
        r2 += diff * diff
    return r2


def cross_kernel(Xa, Xb, hyp: Hyper) -> np.ndarray:
    """K_ab[i, j] = s^2 phi(r^2(x_a,i, x_b,j)) (no noise)."""
    return hyp.s2 * phi(hyp.kind, scaled_sqdist(Xa, Xb, hyp.lengthscale))


def kernel_matrix(X, hyp: Hyper) -> np.ndarray:
    """K_ff for the training inputs (Sec. 2)."""
    return cross_kernel(X, X, hyp)


def noisy_kernel_matrix(X, hyp: Hyper) -> np.ndarray:
    """K_y = K_ff + sigma_n^2 I (Sec. 2)."""
    K = kernel_matrix(X, hyp)
    K[np.diag_indices_from(K)] += hyp.noise
    return K


# --------------------------------------------------------------------------- products

def matvec(X, V, hyp: Hyper, block: int = 2048) -> np.ndarray:
    """out = K_y V, the product of Table 3, row block by row block (memory O(block * N))."""
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    squeeze = V.ndim == 1
    V2 = V[:, None] if squeeze else V
    out = np.empty((X.shape[0], V2.shape[1]))
    for a in range(0, X.shape[0], block):
        b = min(a + block, X.shape[0])
        out[a:b] = cross_kernel(X[a:b], X, hyp) @ V2
    out += hyp.noise * V2
    return out[:, 0] if squeeze else out


def matvec_rows(X, V, hyp: Hyper, rows) -> np.ndarray:
    """Rows ``rows`` of K_y V, for spot checks at sizes where the full product is too slow."""
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    V2 = V[:, None] if V.ndim == 1 else V
    out = cross_kernel(X[rows], X, hyp) @ V2 + hyp.noise * V2[rows]
    return out[:, 0] if V.ndim == 1 else out


def dK_matrices(X, hyp: Hyper) -> list[np.ndarray]:
    """Explicit dK_y/dtheta_p for theta = (log l_1..log l_D, log s^2, log sigma^2).

    log l_d: s^2 dphi/dr^2 * dr^2/dlog l_d with dr^2/dlog l_d = -2 ((x_d - x'_d)/l_d)^2,
             i.e. s^2 lengthscale_coef(r^2) ((x_d - x'_d)/l_d)^2.
    log s^2: K_ff.   log sigma^2: sigma^2 I.
    """
    X = np.asarray(X, dtype=np.float64)
    ls = hyp.lengthscale
    r2 = scaled_sqdist(X, X, ls)
    g = hyp.s2 * lengthscale_coef(hyp.kind, r2)
    mats = []
    for d in range(X.shape[1]):
        rd2 = ((X[:, d][:, None] - X[:, d][None, :]) / ls[d]) ** 2
        mats.append(g * rd2)
    mats.append(hyp.s2 * phi(hyp.kind, r2))
    mats.append(hyp.noise * np.eye(X.shape[0]))
    return mats


def dK_matvec(X, W, hyp: Hyper) -> np.ndarray:
    """Derivative blocks G[p] = (dK_y/dtheta_p) W, shape [P, N, t]."""
    W = np.asarray(W, dtype=np.float64)
    W2 = W[:, None] if W.ndim == 1 else W
    return np.stack([M @ W2 for M in dK_matrices(X, hyp)])


# --------------------------------------------------------------------------- exact inference

def cholesky_solve(Ky: np.ndarray, B: np.ndarray) -> np.ndarray:
    """K_y^{-1} B by a Cholesky factor and two triangular solves (Sec. 2 exact inference)."""
    import scipy.linalg as sla
    L = np.linalg.cholesky(Ky)
    return sla.cho_solve((L, True), np.asarray(B, dtype=np.float64))


def logdet(Ky: np.ndarray) -> float:
    """log|K_y| = 2 sum log L_ii."""
    L = np.linalg.cholesky(Ky)
    return float(2.0 * np.sum(np.log(np.diag(L))))


def lml_from(Ky: np.ndarray, y: np.ndarray) -> float:
    """-1/2 [y^T K_y^{-1} y + log|K_y| + N log 2 pi] (Sec. 2)."""
    y = np.asarray(y, dtype=np.float64)
    a = cholesky_solve(Ky, y)
    return float(-0.5 * (y @ a + logdet(Ky) + y.shape[0] * math.log(2.0 * math.pi)))


def lml(X, y, hyp: Hyper) -> float:
    return lml_from(noisy_kernel_matrix(X, hyp), y)


def grad_exact(X, y, hyp: Hyper) -> np.ndarray:
    """d LML / d theta_p = 1/2 a^T dK_p a - 1/2 tr(K_y^{-1} dK_p), a = K_y^{-1} y."""
    Ky = noisy_kernel_matrix(X, hyp)
    a = cholesky_solve(Ky, np.asarray(y, dtype=np.float64))
    Kinv = cholesky_solve(Ky, np.eye(Ky.shape[0]))
    return np.array([0.5 * a @ M @ a - 0.5 * np.sum(Kinv * M) for M in dK_matrices(X, hyp)])


# --------------------------------------------------------------------------- probes

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of splitmix64 from state ``x`` (Steele, Lea & Flood 2014): advance, then mix."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def rademacher(seed: int, N: int, m: int) -> np.ndarray:
    """[N, m] float64 +-1 probes: z[i, c] = 1 - 2 * bit63(splitmix64(seed ^ (c << 32 | i))).

    Independent Rademacher probes are what the paper uses for its CG trace
    estimator (Sec. 4.3). Vectorised uint64 arithmetic wraps modulo 2^64 as the
    definition requires.
    """
    i = np.arange(N, dtype=np.uint64)[:, None]
    c = np.arange(m, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        key = np.uint64(seed & _M64) ^ ((c << np.uint64(32)) | i)
        z = key + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return 1.0 - 2.0 * (z >> np.uint64(63)).astype(np.float64)


# --------------------------------------------------------------------------- CG and Lanczos

@dataclass
class CGResult:
    x: np.ndarray          # [N, t]
    alphas: np.ndarray     # [max_iter, t] (0 after a column stops)
    betas: np.ndarray      # [max_iter, t]
    iters: np.ndarray      # [t] iterations taken per column
    rel_resid: np.ndarray  # [t] recursive ||r|| / ||b|| at stop


def cg(apply_A, B, tol: float, max_iter: int) -> CGResult:
    """Textbook CG from x0 = 0, no preconditioner, one independent recurrence per column.

    Column c stops when its recursive residual satisfies ||r||/||b|| <= tol (or
    at max_iter). alpha_k = r_k^T r_k / p_k^T A p_k, beta_k = r_{k+1}^T r_{k+1} / r_k^T r_k.
    """
    B = np.asarray(B, dtype=np.float64)
    B = B[:, None] if B.ndim == 1 else B
    N, t = B.shape
    x = np.zeros_like(B)
    r = B.copy()
    p = B.copy()
    rr = np.sum(r * r, axis=0)
    bnorm = np.sqrt(rr)
    active = bnorm > 0
    iters = np.zeros(t, dtype=np.int64)
    alphas = np.zeros((max_iter, t))
    betas = np.zeros((max_iter, t))
    for k in range(max_iter):
        if not active.any():
            break
        Ap = apply_A(p)
        pAp = np.sum(p * Ap, axis=0)
        alpha = np.where(active, rr / np.where(active, pAp, 1.0), 0.0)
        x += alpha * p
        r -= alpha * Ap
        rr_new = np.sum(r * r, axis=0)
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        alphas[k] = alpha
        betas[k] = beta
        iters += active
        p = np.where(active, r + beta * p, p)
        rr = np.where(active, rr_new, rr)
        active = active & (np.sqrt(rr) > tol * bnorm)
    rel = np.sqrt(rr) / np.where(bnorm > 0, bnorm, 1.0)
    return CGResult(x, alphas, betas, iters, rel)


def lanczos_tridiag_from_cg(alphas: np.ndarray, betas: np.ndarray, m: int) -> np.ndarray:
    """The m x m Lanczos tridiagonal that CG's coefficients define for one column.

    T[k, k] = 1/alpha_k + beta_{k-1}/alpha_{k-1} (second term absent for k = 0),
    T[k, k+1] = T[k+1, k] = sqrt(beta_k) / alpha_k
    (the CG-Lanczos relation; Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.7.3).
    """
    T = np.zeros((m, m))
    for k in range(m):
        T[k, k] = 1.0 / alphas[k] + (betas[k - 1] / alphas[k - 1] if k > 0 else 0.0)
        if k + 1 < m:
            T[k, k + 1] = T[k + 1, k] = math.sqrt(betas[k]) / alphas[k]
    return T


def quadrature_logdet(T: np.ndarray, znorm2: float) -> float:
    """||z||^2 e_1^T log(T) e_1 = ||z||^2 sum_j Q[0, j]^2 log(lambda_j) (Gauss quadrature)."""
    lam, Q = np.linalg.eigh(T)
    return float(znorm2 * np.sum(Q[0, :] ** 2 * np.log(lam)))


def lanczos_full_reorth(A: np.ndarray, z: np.ndarray, m: int) -> np.ndarray:
    """m steps of Lanczos on A from z/||z|| with full reorthogonalisation (Golub & Van Loan 10.1)."""
    N = A.shape[0]
    Qb = np.zeros((N, m))
    a = np.zeros(m)
    b = np.zeros(max(m - 1, 0))
    q = np.asarray(z, dtype=np.float64) / np.linalg.norm(z)
    for k in range(m):
        Qb[:, k] = q
        w = A @ q
        a[k] = q @ w
        w -= Qb[:, :k + 1] @ (Qb[:, :k + 1].T @ w)
        w -= Qb[:, :k + 1] @ (Qb[:, :k + 1].T @ w)
        if k + 1 < m:
            b[k] = np.linalg.norm(w)
            q = w / b[k]
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def slq_logdet_from_cg(res: CGResult, Z: np.ndarray, L: int, first_probe_col: int = 1) -> float:
    """Stochastic Lanczos log-det: mean over probe columns of ||z_i||^2 e_1^T log(T_i) e_1.

    T_i uses the first min(L, iterations of column i) CG steps of that column.
    """
    Z = np.asarray(Z, dtype=np.float64)
    vals = []
    for i in range(Z.shape[1]):
        c = first_probe_col + i
        m = int(min(L, res.iters[c]))
        T = lanczos_tridiag_from_cg(res.alphas[:, c], res.betas[:, c], m)
        vals.append(quadrature_logdet(T, float(Z[:, i] @ Z[:, i])))
    return float(np.mean(vals))


# --------------------------------------------------------------------------- estimators

def probe_conditioned_targets(X, y, hyp: Hyper, Z: np.ndarray) -> dict:
    """Exact values of the stochastic estimators for fixed probes Z ([N, m]).

    logdet_Z = mean_i z_i^T log(K_y) z_i (via eigh), tr_Z(M) = mean_i (K_y^{-1} z_i)^T M z_i,
    grad_Z[p] = 1/2 a^T dK_p a - 1/2 tr_Z(dK_p), lml_Z = -1/2 (y^T a + logdet_Z + N log 2 pi).
    """
    Ky = noisy_kernel_matrix(X, hyp)
    y = np.asarray(y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    lam, Q = np.linalg.eigh(Ky)
    W = Q.T @ Z
    logdet_Z = float(np.mean(np.sum(W * W * np.log(lam)[:, None], axis=0)))
    a = cholesky_solve(Ky, y)
    U = cholesky_solve(Ky, Z)
    grad = np.array([0.5 * a @ M @ a - 0.5 * np.mean(np.sum(U * (M @ Z), axis=0))
                     for M in dK_matrices(X, hyp)])
    N = y.shape[0]
    quad = float(y @ a)
    return {"logdet": logdet_Z, "quad": quad, "lml": -0.5 * (quad + logdet_Z + N * math.log(2 * math.pi)),
            "grad": grad, "logdet_exact": float(np.sum(np.log(lam)))}


def estimator_fp64(X, y, hyp: Hyper, n_probes: int, lanczos_steps: int, seed: int,
                   tol: float = 1e-6, max_iter: int | None = None) -> dict:
    """The mBCG / stochastic-Lanczos LML and Hutchinson gradient, run in float64.

    Batched CG on [y, z_1..z_m] gives a = K_y^{-1} y (quad term y^T a) and
    u_i = K_y^{-1} z_i; each probe's CG coefficients give a Lanczos tridiagonal
    for the log-det quadrature; the gradient is
    g_p = 1/2 a^T dK_p a - 1/2 mean_i u_i^T dK_p z_i.
    """
    X64 = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    Z = rademacher(seed, N, n_probes)
    B = np.concatenate([y[:, None], Z], axis=1)
    Ky = noisy_kernel_matrix(X64, hyp)
    res = cg(lambda P: Ky @ P, B, tol, max_iter or min(N, 1000))
    a = res.x[:, 0]
    U = res.x[:, 1:]
    ld = slq_logdet_from_cg(res, Z, lanczos_steps)
    quad = float(y @ a)
    grad = np.array([0.5 * a @ M @ a - 0.5 * np.mean(np.sum(U * (M @ Z), axis=0))
                     for M in dK_matrices(X64, hyp)])
    return {"logdet": ld, "quad": quad, "lml": -0.5 * (quad + ld + N * math.log(2 * math.pi)),
            "grad": grad, "iters": res.iters, "Z": Z, "cg": res}


# --------------------------------------------------------------------------- posterior prediction

def predict_exact(X, y, Xs, hyp: Hyper) -> tuple[np.ndarray, np.ndarray]:
    """Posterior predictive mean and latent variance at test points Xs (Sec. 2):
    mu_* = K_*f K_y^{-1} y,  var_* = diag(K_** - K_*f K_y^{-1} K_f*), by a Cholesky solve."""
    Ky = noisy_kernel_matrix(X, hyp)
    Ksf = cross_kernel(Xs, X, hyp)
    mean = Ksf @ cholesky_solve(Ky, np.asarray(y, dtype=np.float64))
    W = cholesky_solve(Ky, Ksf.T)
    kss = hyp.s2 * phi(hyp.kind, np.zeros(np.asarray(Xs).shape[0]))
    var = kss - np.sum(Ksf.T * W, axis=0)
    return mean, var


def predict_var_hutchinson_target(X, Xs, hyp: Hyper, Z: np.ndarray) -> np.ndarray:
    """What the probe estimate of the predictive variance converges to for given probes Z [M, m]
    (exact solves): var_i = k_ii - mean_c Z[i, c] (A Z)[i, c], A = K_*f K_y^{-1} K_f*
    (the diagonal estimator diag(A) ~ mean_c z_c * (A z_c); Bekas, Kokiopoulou & Saad 2007)."""
    Ky = noisy_kernel_matrix(X, hyp)
    Ksf = cross_kernel(Xs, X, hyp)
    AZ = Ksf @ cholesky_solve(Ky, Ksf.T @ np.asarray(Z, dtype=np.float64))
    kss = hyp.s2 * phi(hyp.kind, np.zeros(np.asarray(Xs).shape[0]))
    return kss - np.mean(np.asarray(Z, dtype=np.float64) * AZ, axis=1)


def predict_fp64(X, y, Xs, hyp: Hyper, n_probes: int, seed: int, tol: float = 1e-6,
                 max_iter: int | None = None) -> dict:
    """The CG prediction route in float64, step by step.

    One batched CG solve on [y, K_f* z_1 .. K_f* z_m] (textbook CG, as for the LML) gives
    a = K_y^{-1} y and w_c = K_y^{-1} K_f* z_c; then mu_* = K_*f a and
    var_i = k_ii - mean_c z_c[i] (K_*f w_c)[i], with probes z_c = rademacher(seed, M, m).
    n_probes = 0: exact variance, with columns K_f* e_j for every test point j instead of probes.
    """
    X64 = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    M = np.asarray(Xs).shape[0]
    Ky = noisy_kernel_matrix(X64, hyp)
    Ksf = cross_kernel(Xs, X64, hyp)
    Z = rademacher(seed, M, n_probes) if n_probes > 0 else np.eye(M)
    rhs = np.concatenate([y[:, None], Ksf.T @ Z], axis=1)
    res = cg(lambda P: Ky @ P, rhs, tol, max_iter or 10 * N)
    mean = Ksf @ res.x[:, 0]
    kss = hyp.s2 * phi(hyp.kind, np.zeros(M))
    Q = Ksf @ res.x[:, 1:]
    if n_probes > 0:
        var = kss - np.mean(Z * Q, axis=1)
    else:
        var = kss - np.diag(Q)
    return {"mean": mean, "var": var, "Z": Z, "iters": res.iters, "rel_resid": res.rel_resid}


# --------------------------------------------------------------------------- preconditioning
#
# Rank-k partial pivoted Cholesky of K_ff as the preconditioner P = L L^T + sigma^2 I of CG, the
# preconditioned stochastic Lanczos log-determinant and the matching gradient estimator. The
# paper names the missing preconditioner as a gap of its CG path (Sec. 5); this is the published
# construction of Gardner et al. (GPyTorch BBMM, 2018), with the pivoted Cholesky of Harbrecht,
# Peters & Schneider (2012).

def pivoted_cholesky(X, hyp: Hyper, rank: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Greedy partial pivoted Cholesky of K_ff: returns L [N, rank], the pivots and the final
    residual diagonal d = diag(K_ff - L L^T).

    Step m: i = argmax d (first index on ties); L[:, m] = (K[:, i] - L[:, :m] L[i, :m]) / sqrt(d_i);
    d -= L[:, m]^2. Once the largest remaining d is at most 1e-10 s^2 (K_ff is numerically reproduced),
    the remaining columns stay zero.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    L = np.zeros((N, rank))
    d = hyp.s2 * phi(hyp.kind, np.zeros(N))
    piv = []
    for m in range(rank):
        i = int(np.argmax(d))
        if not d[i] > 1e-10 * hyp.s2:
            break
        piv.append(i)
        row = cross_kernel(X[i:i + 1], X, hyp)[0]
        L[:, m] = (row - L[:, :m] @ L[i, :m]) / math.sqrt(d[i])
        d = d - L[:, m] ** 2
        d[i] = 0.0
    return L, np.asarray(piv, dtype=np.int64), d


def precond_inverse(L: np.ndarray, noise: float):
    """P^{-1} R for P = L L^T + sigma^2 I by the Woodbury identity:
    P^{-1} R = (R - L C^{-1} L^T R) / sigma^2, C = sigma^2 I_k + L^T L."""
    C = noise * np.eye(L.shape[1]) + L.T @ L

    def apply(R):
        R = np.asarray(R, dtype=np.float64)
        return (R - L @ np.linalg.solve(C, L.T @ R)) / noise
    return apply


def precond_logdet(L: np.ndarray, noise: float) -> float:
    """log|L L^T + sigma^2 I| = (N - k) log sigma^2 + log|sigma^2 I_k + L^T L| (determinant lemma)."""
    N, k = L.shape
    sign, ld = np.linalg.slogdet(noise * np.eye(k) + L.T @ L)
    return float((N - k) * math.log(noise) + ld)


@dataclass
class PCGResult:
    x: np.ndarray          # [N, t]
    alphas: np.ndarray     # [max_iter, t]
    betas: np.ndarray      # [max_iter, t]
    iters: np.ndarray      # [t]
    rel_resid: np.ndarray  # [t] recursive ||r|| / ||b||
    rz0: np.ndarray        # [t] b^T P^{-1} b (the quadrature weight)


def pcg(apply_A, apply_Pinv, B, tol: float, max_iter: int) -> PCGResult:
    """Textbook preconditioned CG from x0 = 0, one recurrence per column:
    z = P^{-1} r, alpha = r^T z / p^T A p, x += alpha p, r -= alpha A p, beta = r'^T z' / r^T z,
    p = z' + beta p; column c stops when ||r|| <= tol ||b|| (or at max_iter)."""
    B = np.asarray(B, dtype=np.float64)
    B = B[:, None] if B.ndim == 1 else B
    N, t = B.shape
    x = np.zeros_like(B)
    r = B.copy()
    z = apply_Pinv(r)
    p = z.copy()
    rz = np.sum(r * z, axis=0)
    rz0 = rz.copy()
    bb = np.sum(B * B, axis=0)
    active = bb > 0.0
    alphas = np.zeros((max_iter, t))
    betas = np.zeros((max_iter, t))
    iters = np.zeros(t, dtype=np.int64)
    rr = bb.copy()
    for k in range(max_iter):
        if not active.any():
            break
        Ap = apply_A(p)
        pAp = np.sum(p * Ap, axis=0)
        alpha = np.where(active, rz / np.where(active, pAp, 1.0), 0.0)
        x += alpha * p
        r -= alpha * Ap
        rr = np.sum(r * r, axis=0)
        z = apply_Pinv(r)
        rz_new = np.sum(r * z, axis=0)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        alphas[k] = alpha
        betas[k] = beta
        iters += active
        rz = np.where(active, rz_new, rz)
        p = np.where(active, z + beta * p, p)
        active = active & (np.sqrt(rr) > tol * np.sqrt(bb))
    rel = np.sqrt(rr / np.where(bb > 0, bb, 1.0))
    return PCGResult(x, alphas, betas, iters, rel, rz0)


def precond_probes(seed: int, L: np.ndarray, noise: float, m: int) -> np.ndarray:
    """Probes with covariance P = L L^T + sigma^2 I: z_c = L e1_c + sigma e2_c, where e = rademacher(seed,
    N + k, m) supplies e2 (rows 0..N-1) and e1 (rows N..N+k-1)."""
    N, k = L.shape
    E = rademacher(seed, N + k, m)
    return L @ E[N:] + math.sqrt(noise) * E[:N]


def estimator_precond_fp64(X, y, hyp: Hyper, rank: int, n_probes: int, lanczos_steps: int, seed: int,
                           tol: float = 1e-6, max_iter: int | None = None) -> dict:
    """The preconditioned mBCG / stochastic-Lanczos LML and gradient, run in float64:
    PCG on [y, z_1..z_m] with z_i ~ (0, P); logdet = log|P| + mean_i (z_i^T P^{-1} z_i) e1^T log(T_i) e1;
    g_p = 1/2 a^T dK_p a - 1/2 mean_i u_i^T dK_p P^{-1} z_i, u_i = K_y^{-1} z_i."""
    X64 = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    L, piv, _ = pivoted_cholesky(X64, hyp, rank)
    Pinv = precond_inverse(L, hyp.noise)
    Z = precond_probes(seed, L, hyp.noise, n_probes)
    Ky = noisy_kernel_matrix(X64, hyp)
    B = np.concatenate([y[:, None], Z], axis=1)
    res = pcg(lambda P: Ky @ P, Pinv, B, tol, max_iter or 10 * N)
    a = res.x[:, 0]
    U = res.x[:, 1:]
    gam = []
    for c in range(1, B.shape[1]):
        mm = min(lanczos_steps, int(res.iters[c]))
        T = lanczos_tridiag_from_cg(res.alphas[:mm, c], res.betas[:mm, c], mm)
        gam.append(quadrature_logdet(T, float(res.rz0[c])))
    logdet = precond_logdet(L, hyp.noise) + float(np.mean(gam))
    quad = float(y @ a)
    PZ = Pinv(Z)
    mats = dK_matrices(X64, hyp)
    grad = np.array([0.5 * a @ M @ a - 0.5 * np.mean(np.sum(U * (M @ PZ), axis=0)) for M in mats])
    lml_v = -0.5 * (quad + logdet + N * math.log(2.0 * math.pi))
    return {"lml": lml_v, "quad": quad, "logdet": logdet, "grad": grad, "Z": Z, "L": L, "piv": piv,
            "iters": res.iters, "rel_resid": res.rel_resid}


def precond_probe_targets(X, y, hyp: Hyper, L: np.ndarray, Z: np.ndarray) -> dict:
    """What the preconditioned estimators converge to for given P (from L) and probes Z, with exact solves
    and exact matrix functions: logdet = log|P| + mean_i w_i^T log(P^{-1/2} K_y P^{-1/2}) w_i,
    w_i = P^{-1/2} z_i; grad_p = 1/2 a^T dK_p a - 1/2 mean_i z_i^T K_y^{-1} dK_p P^{-1} z_i."""
    X64 = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    Ky = noisy_kernel_matrix(X64, hyp)
    P = L @ L.T + hyp.noise * np.eye(N)
    lam, Q = np.linalg.eigh(P)
    Pm12 = (Q / np.sqrt(lam)) @ Q.T
    mu, V = np.linalg.eigh(Pm12 @ Ky @ Pm12)
    W = Pm12 @ Z
    logdet = precond_logdet(L, hyp.noise) + float(np.mean(np.sum((V.T @ W) ** 2 * np.log(mu)[:, None], axis=0)))
    a = cholesky_solve(Ky, y)
    KZ = cholesky_solve(Ky, Z)
    PZ = np.linalg.solve(P, Z)
    grad = np.array([0.5 * a @ M @ a - 0.5 * np.mean(np.sum(KZ * (M @ PZ), axis=0)) for M in dK_matrices(X64, hyp)])
    quad = float(y @ a)
    return {"lml": -0.5 * (quad + logdet + N * math.log(2.0 * math.pi)), "quad": quad, "logdet": logdet,
            "grad": grad}
