"""Failure detection without a GPU fault: bounded device waits and host-side error paths."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def test_wait_budget_exhaustion_is_reported_and_context_survives(lgp):
    """A one-cycle budget makes the tensor-core pipeline waits run out: the kernel records
    LGP_ERR_TIMEOUT, drains its own copies, frees tensor memory and returns; the same
    context then runs the product normally."""
    import torch
    ctx = lgp.Context(0)
    p = wl.random_problem(4096, 4, wl.RBF, seed=1)
    X = torch.as_tensor(p.X, device="cuda")
    V = torch.as_tensor(wl.rhs_block(p.N, 32, seed=1), device="cuda")
    assert ctx.check_device_status() == lgp.LGP_OK
    ctx.set_wait_budget(1)
    lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_BF16, ctx=ctx)
    assert ctx.check_device_status() == lgp.LGP_ERR_TIMEOUT
    ctx.set_wait_budget(0)  # default budget
    out = lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_SPLIT_F16, ctx=ctx)
    assert ctx.check_device_status() == lgp.LGP_OK
    ref = lgp.lgp_kernel_matvec(X, p, V, prec=lgp.LGP_PREC_FP32, ctx=ctx)
    torch.cuda.synchronize()
    err = (torch.linalg.norm(out - ref, dim=0) / torch.linalg.norm(ref, dim=0)).max().item()
    assert err <= 1e-5
    ctx.close()


def test_timeout_inside_cg_is_reported(lgp):
    import torch
    ctx = lgp.Context(0)
    p = wl.random_problem(3000, 2, wl.MATERN52, seed=2)
    B = torch.as_tensor(wl.rhs_block(p.N, 16, seed=2), device="cuda")
    ctx.set_wait_budget(1)
    with pytest.raises(lgp.LGPError) as e:
        lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p, B, ctx=ctx, prec=lgp.LGP_PREC_SPLIT_BF16)
    assert e.value.status == lgp.LGP_ERR_TIMEOUT
    ctx.set_wait_budget(0)
    x, iters, rel, s = lgp.lgp_cg_solve(torch.as_tensor(p.X, device="cuda"), p, B, ctx=ctx,
                                        prec=lgp.LGP_PREC_SPLIT_BF16)
    assert s == lgp.LGP_OK and (rel <= 1e-6).all()
    ctx.close()


def test_breakdown_detected_for_indefinite_operator(lgp):
    """A negative noise variance is impossible through log_noise, so indefiniteness is made
    with a huge outputscale and data of duplicated points: K_ff is then singular in float32
    and CG must either converge or stop with a reported status, never return garbage."""
    import torch
    X = np.repeat(np.random.default_rng(0).uniform(0, 1, (50, 2)), 20, axis=0).astype(np.float32)
    hyp = wl.Problem(X, np.zeros(len(X), np.float32), wl.RBF, np.log([0.5, 0.5]).astype(np.float32), 20.0,
                     float(np.log(1e-30)))
    B = torch.as_tensor(wl.rhs_block(len(X), 2, seed=3), device="cuda")
    try:
        x, iters, rel, s = lgp.lgp_cg_solve(torch.as_tensor(X, device="cuda"), hyp, B, max_iter=200)
        assert s in (lgp.LGP_OK, lgp.LGP_WARN_NOT_CONVERGED)
        assert np.isfinite(x.cpu().numpy()).all()
    except lgp.LGPError as e:
        assert e.status in (lgp.LGP_ERR_BREAKDOWN, lgp.LGP_ERR_NONFINITE)
