"""CPU model of the symmetric product's dot-form distance, checking the limits it is gated on.

The GPU forms r^2 = a_i + a_j - 2 u_i . u_j from box-centred coordinates u. It splits them as
u = h + m in float16 and takes three Gram products (h h + m h + h m) together with the squared norms
a = sum(h^2 + 2 h m) (so that r^2_ii = 0 up to rounding) in one float32 tensor-core accumulation,
which returns -r^2 (the Matern square roots then take the absolute value of the rounded r^2). This model
repeats those roundings in NumPy (float16 splits, float32 sums: the Gram part, then each squared
norm, rounded in turn) on the same seeded data and compares the
resulting entries and products with the FP64 oracle. Three properties are checked:

- near each kernel's limit on max |u|^2 (RBF 97, Matern-3/2 134, Matern-5/2 403, prescaled
  units), the entry error stays below the ~1.6e-5 s^2 the limits are derived for, and the product
  meets the 1e-5 column gate;
- far above the limit the model's error is large, which is why such data takes the difference form;
- Matern-1/2 (not smooth in r^2 at 0) is outside the gate even at a small spread.
"""
import math

import numpy as np
import pytest

from oracle import gp_oracle as go
import workloads as wl

LIMIT = {wl.RBF: 97.0, wl.MATERN52: 403.0, wl.MATERN32: 134.0}
PRESCALE = {wl.RBF: math.sqrt(math.log2(math.e) / 2), wl.MATERN52: math.sqrt(5.0), wl.MATERN32: math.sqrt(3.0),
            wl.MATERN12: math.log2(math.e)}


def _prescaled(p):
    return (p.X.astype(np.float64) * PRESCALE[p.kind] / np.exp(p.log_lengthscale.astype(np.float64))).astype(np.float32)


def _dot_form_sq_dist(xs):
    """r^2 as the dot form rounds it: centred float32 u, float16 h + m, float32 Gram and norms."""
    xs = xs.astype(np.float32)
    c = (np.float32(0.5) * (xs.max(0) + xs.min(0))).astype(np.float32)
    u = (xs - c).astype(np.float32)
    h = u.astype(np.float16).astype(np.float64)
    m = (u - h.astype(np.float32)).astype(np.float16).astype(np.float64)
    g = (h @ h.T + m @ h.T + h @ m.T).astype(np.float32)
    a = (h * h + 2 * h * m).sum(1).astype(np.float32)
    d = (np.float32(2) * g - a[None, :]).astype(np.float32)  # the Gram value 2 u_i.u_j - a_j
    return (a[:, None] - d).astype(np.float32), float(((xs - c).astype(np.float64) ** 2).sum(1).max())


def _entries(kind, r2, s2):
    """k from prescaled squared distances (the oracle's forms on the prescaled coordinates). As on the GPU,
    the RBF exponent and the Matern-5/2 quadratic term take the rounded value as it is, and the Matern square
    roots its absolute value."""
    r2 = r2.astype(np.float64)
    if kind == wl.RBF:
        return s2 * np.exp2(-r2)
    r = np.sqrt(np.abs(r2))
    if kind == wl.MATERN52:
        # the quadratic term takes the signed r^2 (no absolute value there on the GPU either)
        return s2 * (1 + r + r2 / 3) * np.exp(-r)
    if kind == wl.MATERN32:
        return s2 * (1 + r) * np.exp(-r)
    return s2 * np.exp2(-r)


def _model(p, t=8, seed=0):
    hyp = go.hyper_of(p)
    xs = _prescaled(p)
    r2_dot, amax = _dot_form_sq_dist(xs)
    K_dot = _entries(p.kind, r2_dot, hyp.s2)
    K = go.kernel_matrix(p.X, hyp)
    V = np.random.default_rng(seed).choice([-1.0, 1.0], size=(p.N, t))
    ref = K @ V + hyp.noise * V
    got = K_dot @ V + hyp.noise * V
    col = (np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()
    return np.abs(K_dot - K).max() / hyp.s2, col, amax


def _scaled_to(p, target):
    """The problem with its lengthscales scaled so that max |u|^2 = target."""
    ls = np.exp(p.log_lengthscale.astype(np.float64))
    _, amax = _dot_form_sq_dist(_prescaled(p))
    p.log_lengthscale = np.log(ls * math.sqrt(amax / target)).astype(np.float32)
    return p


def test_entries_are_the_oracles_forms():
    """The model's entry forms reproduce the oracle's kernel matrix from exact distances."""
    for kind in wl.KINDS:
        p = wl.random_problem(60, 3, kind, seed=500 + kind)
        xs = _prescaled(p).astype(np.float64)
        r2 = ((xs[:, None, :] - xs[None, :, :]) ** 2).sum(-1)
        K = go.kernel_matrix(p.X, go.hyper_of(p))
        assert np.abs(_entries(kind, r2, go.hyper_of(p).s2) - K).max() <= 1e-5 * go.hyper_of(p).s2


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN32, wl.MATERN52])
def test_errors_near_the_limit_stay_within_the_bound(kind):
    p = _scaled_to(wl.cfg3(N=700, kind=kind), 0.9 * LIMIT[kind])
    ent, col, amax = _model(p)
    assert amax == pytest.approx(0.9 * LIMIT[kind], rel=1e-3)
    print(f"kind={kind}: max|u|^2 {amax:.1f}, entry error {ent:.2e} s^2, column error {col:.2e}")
    assert ent <= 1.6e-5
    assert col <= 1e-5


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN32, wl.MATERN52])
def test_box_filling_data_near_the_limit(kind, D):
    """Points that fill their box (X ~ U[0,1]^D, as in the low-dimensional workloads) with lengthscales
    set so that max |u|^2 is 90% of the limit: close pairs near the box's corners, where the Gram terms
    cancel most, lift single entries above the ~1.6e-5 s^2 the limits were derived for (up to ~4e-5 here,
    held within four times that bound), but the errors do not line up, and the product meets its 1e-5
    column gate (at most ~6e-6 over these draws)."""
    worst = 0.0
    for seed in range(3):
        p = _scaled_to(wl.random_problem(900, D, kind, seed=530 + 10 * D + kind + 100 * seed), 0.9 * LIMIT[kind])
        ent, col, amax = _model(p, t=8, seed=seed)
        assert amax == pytest.approx(0.9 * LIMIT[kind], rel=1e-3)
        print(f"kind={kind} D={D} seed={seed}: entry error {ent:.2e} s^2, column error {col:.2e}")
        assert ent <= 4 * 1.6e-5
        worst = max(worst, col)
    assert worst <= 1e-5


def test_one_dimension_is_outside_the_gate():
    """At D = 1 every point lies on one axis and close pairs at the far ends of the box are common: near
    the Matern-5/2 limit the model's product error exceeds the 1e-5 gate, which is why D = 1 takes the
    difference form."""
    worst = 0.0
    for seed in range(6):
        p = _scaled_to(wl.random_problem(900, 1, wl.MATERN52, seed=600 + 7 * seed + 1), 0.9 * LIMIT[wl.MATERN52])
        _, col, _ = _model(p, t=8, seed=seed)
        worst = max(worst, col)
    print(f"Matern-5/2, D = 1: worst column error {worst:.2e}")
    assert worst > 1e-5


@pytest.mark.parametrize("kind", [wl.RBF, wl.MATERN52])
def test_far_above_the_limit_the_dot_form_is_inaccurate(kind):
    """A spread 100x the limit, with close pairs far from the centre (two tight clusters at opposite
    ends of the box), makes the dot form's absolute rounding error visible, which is why such data
    takes the difference form."""
    rng = np.random.default_rng(510)
    X = rng.normal(0.0, 0.01, (400, 3))
    X[200:, 0] += 1.0
    p = wl.Problem(X.astype(np.float32), np.zeros(400, np.float32), kind, np.zeros(3, np.float32), 0.0,
                   float(np.float32(math.log(0.01))))
    p = _scaled_to(p, 100.0 * LIMIT[kind])
    ent, col, _ = _model(p)
    print(f"kind={kind}: entry error {ent:.2e} s^2, column error {col:.2e}")
    assert ent > 1e-4


def test_matern12_is_outside_the_gate():
    """Matern-1/2's dk/dr^2 is unbounded at r = 0: even a small spread gives entry errors above the
    bound, so it always takes the difference form."""
    p = wl.random_problem(600, 1, wl.MATERN12, seed=520)
    ent, _, amax = _model(p)
    print(f"Matern-1/2: max|u|^2 {amax:.2f}, entry error {ent:.2e} s^2")
    assert amax < 1.0 and ent > 1.6e-5
