"""Batched uneven-GP CG (lgp_batch_cg_solve) against the FP64 oracle.

Gates:
- Each problem's CG solution (run to relative residual 1e-6) is within max(1e-4, 2e-8 kappa) of its
  Cholesky solve. kappa(K_y) comes from the oracle's eigenvalues. The batch draws smooth kernels on
  small boxes, so kappa reaches 1e5 and a float32 solve carries about kappa times float32 rounding.
- At full batch size (64 problems, N up to 30000, kappa up to ~3e6), the componentwise backward
  error |b - K_y x|_i / ((K_y |x|)_i + |b_i|) is checked on sampled rows. The FP64 row oracle
  computes it, and it is valid because every kernel entry is positive. This is the property a
  float32 solve can meet at any conditioning; the plain relative residual cannot.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import gp_oracle as go
import workloads as wl

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _rhs(p, t, seed):
    B = wl.rhs_block(p.N, t, seed=seed, kind="sign")
    B[:, 0] = p.y
    return B


def test_batch_small_against_cholesky(lgp):
    probs = wl.cfg5_batch(n_gp=10, t=8, seed=11, n_lo=200, n_hi=2500)
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                 tol=1e-6, max_iter=3000)
    assert s == lgp.LGP_OK
    assert (rel <= 1e-6).all()
    for p, B, x in zip(probs, Bs, sols):
        Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
        ev = np.linalg.eigvalsh(Ky)
        gate = max(1e-4, 2e-8 * ev[-1] / ev[0])
        ref = go.cholesky_solve(Ky, B.astype(np.float64))
        err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= gate, (p.name, err.max(), gate)


def test_batch_cfg5_full_true_residual(lgp):
    """64 problems, N log-uniform in [500, 30000], D in 1..6, t=8, one call."""
    import torch
    probs = wl.cfg5_batch()
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                 tol=1e-6, max_iter=5000)
    assert s == lgp.LGP_OK
    assert (rel <= 1e-6).all()
    rng = np.random.default_rng(5)
    worst = 0.0
    for p, B, x in zip(probs, Bs, sols):
        rows = rng.choice(p.N, min(32, p.N), replace=False)
        xs = x.cpu().numpy()
        Kx, _ = oracle.kyv_rows_c(p.X, xs, go.hyper_of(p), rows=rows)
        Kabs, _ = oracle.kyv_rows_c(p.X, np.abs(xs), go.hyper_of(p), rows=rows)
        berr = np.abs(B[rows] - Kx) / (Kabs + np.abs(B[rows]))
        worst = max(worst, float(berr.max()))
    print(f"cfg5 batch: iterations {iters.min()}..{iters.max()}, worst componentwise backward error {worst:.2e}")
    assert worst <= 1e-5


def test_batch_matches_single_problem_solves(lgp):
    probs = wl.cfg5_batch(n_gp=6, t=8, seed=12, n_lo=300, n_hi=4000)
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    sols, _, _, _ = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs], tol=1e-6,
                                           max_iter=3000)
    for p, B, x in zip(probs, Bs, sols):
        y, _, _, _ = lgp.lgp_cg_solve(_dev(p.X), p, _dev(B), tol=1e-6, max_iter=3000, prec=lgp.LGP_PREC_FP32)
        ev = np.linalg.eigvalsh(go.noisy_kernel_matrix(p.X, go.hyper_of(p)))
        gate = max(1e-4, 4e-8 * ev[-1] / ev[0])  # two float32 solves, each within ~2e-8 kappa
        a = x.cpu().numpy().astype(np.float64)
        b = y.cpu().numpy().astype(np.float64)
        assert (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max() <= gate


def test_batch_edge_cases(lgp):
    # one problem with one point; a zero column; t = 1 and t = 3
    q = wl.random_problem(1, 3, wl.MATERN52, seed=13)
    sols, iters, _, s = lgp.lgp_batch_cg_solve([_dev(q.X)], [q], [_dev(np.array([[3.0]], np.float32))], tol=1e-6)
    assert s == lgp.LGP_OK
    v = math.exp(q.log_outputscale) + math.exp(q.log_noise)
    assert abs(float(sols[0].cpu()) - 3.0 / v) < 1e-6
    probs = [wl.random_problem(n, d, k, seed=n) for n, d, k in [(50, 1, wl.RBF), (700, 6, wl.MATERN52)]]
    Bs = [wl.rhs_block(p.N, 3, seed=1) for p in probs]
    Bs[1][:, 2] = 0.0
    sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs], tol=1e-6)
    assert s == lgp.LGP_OK and iters[1, 2] == 0 and np.all(sols[1].cpu().numpy()[:, 2] == 0)
    for p, B, x in zip(probs, Bs, sols):
        Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
        ev = np.linalg.eigvalsh(Ky)
        ref = go.cholesky_solve(Ky, B.astype(np.float64))
        keep = np.linalg.norm(ref, axis=0) > 0
        err = np.linalg.norm(x.cpu().numpy()[:, keep] - ref[:, keep], axis=0) / np.linalg.norm(ref[:, keep], axis=0)
        assert err.max() <= max(1e-4, 2e-8 * ev[-1] / ev[0])
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_batch_cg_solve([_dev(q.X)], [q], [_dev(np.ones((1, 17), np.float32))])
    assert e.value.status == lgp.LGP_ERR_UNSUPPORTED


def test_batch_routes_reach_the_same_backward_error(lgp):
    """Problems large enough for the tensor-core route (N >= 2048): the default call, whose route per shape
    is timed, and the same call with prec = FP32, which keeps every problem in the persistent batch launch,
    each reach a componentwise backward error below 1e-5 on sampled rows (FP64 row oracle), and the route
    diagnostic names a route for every shape after the call."""
    probs = wl.cfg5_batch(n_gp=6, t=8, seed=21, n_lo=2500, n_hi=9000)
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    ctx = lgp.Context(0)
    rng = np.random.default_rng(9)
    for prec in (lgp.LGP_PREC_AUTO, lgp.LGP_PREC_FP32):
        sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                     tol=1e-6, max_iter=6000, prec=prec, ctx=ctx)
        assert s == lgp.LGP_OK and (rel <= 1e-6).all()
        worst = 0.0
        for p, B, x in zip(probs, Bs, sols):
            rows = rng.choice(p.N, 32, replace=False)
            xs = x.cpu().numpy()
            Kx, _ = oracle.kyv_rows_c(p.X, xs, go.hyper_of(p), rows=rows)
            Kabs, _ = oracle.kyv_rows_c(p.X, np.abs(xs), go.hyper_of(p), rows=rows)
            worst = max(worst, float((np.abs(B[rows] - Kx) / (Kabs + np.abs(B[rows]))).max()))
        routes = [ctx.batch_route_choice(p.N, p.D, p.kind, 8) for p in probs]
        print(f"prec {prec}: routes {routes}, iterations {iters.max()}, worst backward error {worst:.2e}")
        assert worst <= 1e-5
        assert all(r in (lgp.LGP_BATCH_PERSISTENT, lgp.LGP_BATCH_TENSOR) for r in routes)
    assert ctx.batch_route_choice(100, 2, wl.RBF, 8) == lgp.LGP_BATCH_UNTUNED
    ctx.close()


def test_batch_split_counts_are_timed_and_both_choices_solve(lgp, monkeypatch):
    """The persistent launch's column-split count is chosen per problem shape by timing: after a batched
    solve every persistent-route problem has a count among the tuner's candidates (the fixed rule's count
    r and r/4, r/2, 2r, 4r, clamped to [1, 64-column tiles]); with LGP_AUTOTUNE=0 it is the rule's. Both
    solves meet the Cholesky gate of test_batch_small_against_cholesky."""
    probs = wl.cfg5_batch(n_gp=8, t=8, seed=31, n_lo=400, n_hi=3000)
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    refs = []
    for p, B in zip(probs, Bs):
        Ky = go.noisy_kernel_matrix(p.X, go.hyper_of(p))
        ev = np.linalg.eigvalsh(Ky)
        refs.append((go.cholesky_solve(Ky, B.astype(np.float64)), max(1e-4, 2e-8 * ev[-1] / ev[0])))
    for tuned in (True, False):
        if not tuned:
            monkeypatch.setenv("LGP_AUTOTUNE", "0")
        ctx = lgp.Context(0)
        sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                     tol=1e-6, max_iter=3000, ctx=ctx)
        assert s == lgp.LGP_OK and (rel <= 1e-6).all()
        for x, (ref, gate) in zip(sols, refs):
            err = np.linalg.norm(x.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
            assert err.max() <= gate
        chosen = []
        for p in probs:
            if ctx.batch_route_choice(p.N, p.D, p.kind, 8) != lgp.LGP_BATCH_PERSISTENT:
                continue
            S, r = ctx.batch_split_choice(p.N, p.D, p.kind, 8), ctx.batch_split_rule(p.N)
            tiles = (p.N + 63) // 64
            cands = {max(1, min(c, tiles)) for c in (r // 4, r // 2, r, 2 * r, 4 * r)}
            chosen.append((p.N, S, r))
            assert (S in cands) if tuned else (S == r), (p.N, S, r)
        print(f"{'timed' if tuned else 'rule'}: [N, split, rule] {sorted(chosen)}")
        assert chosen  # the persistent route is exercised
        assert ctx.batch_split_choice(100, 2, wl.RBF, 8) == 0
        ctx.close()


def test_batch_choices_persist_in_the_autotune_cache(lgp, monkeypatch, tmp_path):
    """LGP_AUTOTUNE_CACHE holds the batched solver's choices too: after one batched solve the file has a
    route line for every shape of at least 2048 rows and a split line for every persistent-route shape, and
    a fresh context reads the same route and split choices from it."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("LGP_AUTOTUNE_CACHE", str(path))
    probs = wl.cfg5_batch(n_gp=5, t=8, seed=41, n_lo=600, n_hi=5000)
    Bs = [_rhs(p, 8, g) for g, p in enumerate(probs)]
    choices = []
    for _ in range(2):
        ctx = lgp.Context(0)
        sols, iters, rel, s = lgp.lgp_batch_cg_solve([_dev(p.X) for p in probs], probs, [_dev(B) for B in Bs],
                                                     tol=1e-6, max_iter=3000, ctx=ctx)
        assert s == lgp.LGP_OK and (rel <= 1e-6).all()
        choices.append([(ctx.batch_route_choice(p.N, p.D, p.kind, 8), ctx.batch_split_choice(p.N, p.D, p.kind, 8))
                        for p in probs])
        ctx.close()
    assert choices[0] == choices[1]
    lines = path.read_text().splitlines()
    def shape(p):  # the cache key's shape: rows padded to 256, D, kernel
        return ((p.N + 255) // 256 * 256, p.D, p.kind)

    n_route = len({shape(p) for p in probs if p.N >= 2048})
    n_split = len({shape(p) for p, (r, _) in zip(probs, choices[0]) if r == lgp.LGP_BATCH_PERSISTENT})
    assert sum(1 for l in lines if "|route " in l) >= n_route
    assert sum(1 for l in lines if "|split " in l) >= n_split >= 1
