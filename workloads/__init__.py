"""Seeded synthetic inputs for the matrix-free GP path.

This module only draws data: point sets X, targets y, right-hand-side blocks
and hyperparameter values. It holds none of the method's arithmetic (no kernel
function, no solve, no probe generator), so both the CUDA path and the FP64
oracle can take their inputs from it without sharing any computation.

Every generator uses NumPy's PCG64 ``default_rng`` with an explicit seed, draws
in float64 and casts the arrays handed to either side to float32.

Workload recipes (the paper gives no dataset for the matrix-free product, so
these stand in for its unspecified Table 3 data and for the problem sizes of
the CG / stochastic-Lanczos inference path of Sec. 3):

* ``cfg1``  N=1024, D=2, X~U[0,1]^2, y=sin(2 pi x1)+cos(2 pi x2)+0.1 eps,
            RBF, l=0.2, s^2=1, sigma^2=0.01, one right-hand side.
* ``cfg2``  N=20000, D=3, X~N(0,I), y=sum_d sin(pi x_d (d+1)/2)+0.05 eps,
            RBF or Matern-5/2, l=(0.3,0.775,2.0), s^2=1, sigma^2=0.01.
* ``cfg3``  N=100000, D=8, X~U[-1,1]^8, y=sum_d sin(pi x_d)+0.05 eps,
            Matern-5/2, l log-spaced over [0.3,2], s^2=1, sigma^2=0.01, t=32.
* ``cfg4``  as cfg3 but RBF and N=50000, t=16.
* ``cfg5``  64 independent GPs, N_g=round(exp(U[ln 500, ln 30000])),
            D_g~U{1..6}, X~U[0,1]^D_g, y as cfg2, RBF for even g and
            Matern-5/2 for odd g, l_g,d ~ logU[0.3,2], t=8; plus one large
            N=500000, D=2 RBF product with a N(0,1) block of t=32 columns.
* ``table3`` RBF, D=4, X~U[0,1]^4, l=0.5, s^2=1, sigma^2=0.01, t=1, any N.

Every config takes an optional ``N`` so the same distribution can be drawn at
a size the dense oracle handles in seconds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RBF = 0
MATERN52 = 1
MATERN12 = 2
MATERN32 = 3
KINDS = (RBF, MATERN52, MATERN12, MATERN32)


@dataclass
class Problem:
    """One GP problem: data, targets and log-space hyperparameters (float32)."""

    X: np.ndarray                    # [N, D] float32
    y: np.ndarray                    # [N] float32
    kind: int                        # RBF, MATERN52, MATERN12 or MATERN32
    log_lengthscale: np.ndarray      # [D] float32
    log_outputscale: float           # log s^2
    log_noise: float                 # log sigma^2
    t: int = 1                       # columns of the right-hand-side block
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def D(self) -> int:
        return int(self.X.shape[1])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _logspaced_lengthscales(D: int, lo: float = 0.3, hi: float = 2.0) -> np.ndarray:
    if D == 1:
        return np.array([math.sqrt(lo * hi)])
    return np.exp(np.linspace(math.log(lo), math.log(hi), D))


def _sinusoid_targets(rng, X64: np.ndarray, noise: float, freq_by_dim: bool) -> np.ndarray:
    D = X64.shape[1]
    y = np.zeros(X64.shape[0])
    for d in range(D):
        f = math.pi * (d + 2) / 2.0 if freq_by_dim else math.pi
        y += np.sin(f * X64[:, d])
    return y + noise * rng.standard_normal(X64.shape[0])


def cfg1(N: int = 1024, seed: int = 1) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, 2))
    y = np.sin(2 * math.pi * X[:, 0]) + np.cos(2 * math.pi * X[:, 1]) + 0.1 * rng.standard_normal(N)
    return Problem(_f32(X), _f32(y), RBF, _f32(np.log([0.2, 0.2])), 0.0, float(np.float32(math.log(0.01))),
                   t=1, name=f"cfg1-rbf-N{N}-D2")


def cfg2(N: int = 20000, kind: int = RBF, t: int = 1, seed: int = 2) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, 3))
    y = _sinusoid_targets(rng, X, 0.05, True)
    ls = np.array([0.3, 0.775, 2.0])
    kname = "rbf" if kind == RBF else "m52"
    return Problem(_f32(X), _f32(y), kind, _f32(np.log(ls)), 0.0, float(np.float32(math.log(0.01))),
                   t=t, name=f"cfg2-{kname}-N{N}-D3-t{t}")


def cfg3(N: int = 100000, t: int = 32, seed: int = 3, kind: int = MATERN52, D: int = 8) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(N, D))
    y = _sinusoid_targets(rng, X, 0.05, False)
    kname = "rbf" if kind == RBF else "m52"
    return Problem(_f32(X), _f32(y), kind, _f32(np.log(_logspaced_lengthscales(D))), 0.0,
                   float(np.float32(math.log(0.01))), t=t, name=f"cfg3-{kname}-N{N}-D{D}-t{t}")


def cfg4(N: int = 50000, t: int = 16, seed: int = 4) -> Problem:
    p = cfg3(N=N, t=t, seed=seed, kind=RBF)
    p.name = f"cfg4-rbf-N{N}-D8-t{t}"
    return p


def cfg5_batch(n_gp: int = 64, t: int = 8, seed: int = 5, n_lo: int = 500, n_hi: int = 30000) -> list[Problem]:
    rng = np.random.default_rng(seed)
    probs = []
    for g in range(n_gp):
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        D = int(rng.integers(1, 7))
        X = rng.uniform(0.0, 1.0, size=(N, D))
        y = _sinusoid_targets(rng, X, 0.05, True)
        ls = np.exp(rng.uniform(math.log(0.3), math.log(2.0), size=D))
        kind = RBF if g % 2 == 0 else MATERN52
        probs.append(Problem(_f32(X), _f32(y), kind, _f32(np.log(ls)), 0.0, float(np.float32(math.log(0.01))),
                             t=t, name=f"cfg5-gp{g}-N{N}-D{D}"))
    return probs


def cfg5_large(N: int = 500000, t: int = 32, seed: int = 55) -> tuple[Problem, np.ndarray]:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, 2))
    V = rng.standard_normal((N, t))
    p = Problem(_f32(X), _f32(V[:, 0]), RBF, _f32(np.log([0.2, 0.2])), 0.0, float(np.float32(math.log(0.01))),
                t=t, name=f"cfg5-large-rbf-N{N}-D2-t{t}")
    return p, _f32(V)


def table3(N: int, seed: int = 7) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, 4))
    y = rng.standard_normal(N)
    return Problem(_f32(X), _f32(y), RBF, _f32(np.log([0.5] * 4)), 0.0, float(np.float32(math.log(0.01))),
                   t=1, name=f"table3-rbf-N{N}-D4")


def rhs_block(N: int, t: int, seed: int, kind: str = "normal") -> np.ndarray:
    """A [N, t] float32 right-hand-side block: ``normal`` N(0,1) or ``sign`` +-1 entries."""
    rng = np.random.default_rng(seed)
    if kind == "sign":
        return _f32(np.where(rng.random((N, t)) < 0.5, -1.0, 1.0))
    return _f32(rng.standard_normal((N, t)))


def random_problem(N: int, D: int, kind: int, seed: int, lo: float = 0.3, hi: float = 2.0,
                   log_os: float | None = None, log_noise: float | None = None) -> Problem:
    """A generic problem for edge-case sweeps: X~U[0,1]^D, lengthscales logU[lo,hi]."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, D))
    y = rng.standard_normal(N)
    ls = np.exp(rng.uniform(math.log(lo), math.log(hi), size=D))
    los = float(rng.uniform(-0.5, 0.5)) if log_os is None else log_os
    ln = float(math.log(0.05)) if log_noise is None else log_noise
    return Problem(_f32(X), _f32(y), kind, _f32(np.log(ls)), float(np.float32(los)), float(np.float32(ln)),
                   t=1, name=f"rand-{kind}-N{N}-D{D}")
