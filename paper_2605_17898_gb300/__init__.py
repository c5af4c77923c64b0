"""Python binding of the GB300 matrix-free GP library (liblgp.so, C ABI in include/lgp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. Tensors are passed as raw device pointers (``tensor.data_ptr()``) with
the current torch CUDA stream, so the binding does not depend on the torch C++
ABI. If the library is missing, ``load()`` raises: there is no CPU fallback.

Functions named ``lgp_*`` mirror the C entry points of the same name and take
torch tensors; ``Context`` owns an ``lgp_ctx``; ``LGPMarginalLikelihood`` is a
``torch.autograd.Function`` over ``lgp_lml_and_grad`` whose backward returns
the analytic gradient computed in the forward pass.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblgp.so")

LGP_OK = 0
LGP_WARN_NOT_CONVERGED = 1
LGP_ERR_INVALID_ARG = -1
LGP_ERR_UNSUPPORTED = -2
LGP_ERR_CUDA = -3
LGP_ERR_NONFINITE = -4
LGP_ERR_BREAKDOWN = -5
LGP_ERR_TIMEOUT = -6
LGP_ERR_WORKSPACE = -7

LGP_RBF = 0
LGP_MATERN52 = 1
LGP_MATERN12 = 2
LGP_MATERN32 = 3

LGP_PREC_AUTO = 0
LGP_PREC_FP32 = 1
LGP_PREC_SPLIT_BF16 = 2
LGP_PREC_SPLIT_F16 = 3
LGP_TC_UNTUNED = 0
LGP_TC_ROW = 1
LGP_TC_SYMMETRIC = 2
LGP_DIST_NONE = -1
LGP_DIST_DIFF = 0
LGP_DIST_DOT = 1
LGP_BATCH_UNTUNED = 0
LGP_BATCH_PERSISTENT = 1
LGP_BATCH_TENSOR = 2

EXPORTED = [
    "lgp_version", "lgp_status_string", "lgp_create", "lgp_destroy", "lgp_last_error_message",
    "lgp_workspace_bytes", "lgp_matvec_precision", "lgp_set_wait_budget", "lgp_check_device_status",
    "lgp_kernel_matvec", "lgp_kernel_matvec_grad", "lgp_cg_solve", "lgp_lml_and_grad",
    "lgp_rademacher_probes", "lgp_batch_cg_solve", "lgp_kernel_matvec_noalloc",
    "lgp_measure_pipe_peak", "lgp_tc_kernel_choice", "lgp_predict", "lgp_tc_distance_form",
    "lgp_kernel_matvec_noalloc_status", "lgp_batch_route_choice", "lgp_batch_split_choice", "lgp_batch_split_rule",
    "lgp_set_kernel_timing", "lgp_last_kernel_ms",
]


class lgp_hyper(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("D", ctypes.c_int32), ("log_lengthscale", ctypes.POINTER(ctypes.c_float)),
                ("log_outputscale", ctypes.c_float), ("log_noise", ctypes.c_float)]


class lgp_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
                ("n_probes", ctypes.c_int32), ("prec", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("precond_rank", ctypes.c_int32), ("flags", ctypes.c_int32)]


class lgp_lml_info(ctypes.Structure):
    _fields_ = [("lml", ctypes.c_double), ("quad", ctypes.c_double), ("logdet", ctypes.c_double),
                ("max_rel_resid", ctypes.c_double), ("iters_max", ctypes.c_int32), ("iters_min", ctypes.c_int32),
                ("t", ctypes.c_int32), ("prec_used", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("cg_chunks", ctypes.c_int32), ("logdet_precond", ctypes.c_double)]


class lgp_predict_info(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_int32), ("iters_max", ctypes.c_int32), ("max_rel_resid", ctypes.c_double),
                ("var_probes", ctypes.c_int32), ("prec_used", ctypes.c_int32)]


_lib = None


class LGPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblgp.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(p)
    c = ctypes
    vp = c.c_void_p
    sig = {
        "lgp_version": (c.c_int32, []),
        "lgp_status_string": (c.c_char_p, [c.c_int32]),
        "lgp_create": (c.c_int32, [c.POINTER(vp), c.c_int32]),
        "lgp_destroy": (None, [vp]),
        "lgp_last_error_message": (c.c_char_p, [vp]),
        "lgp_workspace_bytes": (c.c_int64, [vp]),
        "lgp_matvec_precision": (c.c_int32, [vp, c.c_int32, c.c_int32]),
        "lgp_set_wait_budget": (None, [vp, c.c_int64]),
        "lgp_check_device_status": (c.c_int32, [vp, vp]),
        "lgp_kernel_matvec": (c.c_int32, [vp, c.POINTER(lgp_hyper), vp, vp, vp, c.c_int64, c.c_int32, c.c_int32, vp]),
        "lgp_kernel_matvec_grad": (c.c_int32, [vp, c.POINTER(lgp_hyper), vp, vp, vp, c.c_int64, c.c_int32, vp]),
        "lgp_cg_solve": (c.c_int32, [vp, c.POINTER(lgp_hyper), vp, vp, vp, c.c_int64, c.c_int32,
                                     c.POINTER(lgp_options), vp, vp, vp]),
        "lgp_lml_and_grad": (c.c_int32, [vp, c.POINTER(lgp_hyper), vp, vp, c.c_int64, c.POINTER(lgp_options),
                                         vp, vp, c.POINTER(lgp_lml_info), vp]),
        "lgp_rademacher_probes": (c.c_int32, [vp, c.c_uint64, c.c_int64, c.c_int32, vp, c.c_int64, vp]),
        "lgp_batch_cg_solve": (c.c_int32, [vp, c.c_int32, c.POINTER(lgp_hyper), vp, vp, vp, vp, c.c_int32,
                                           c.POINTER(lgp_options), vp, vp, vp]),
        "lgp_measure_pipe_peak": (c.c_int32, [c.c_int32, c.POINTER(c.c_double), vp]),
        "lgp_tc_kernel_choice": (c.c_int32, [vp, c.c_int64, c.c_int32, c.c_int32, c.c_int32, c.c_int32]),
        "lgp_tc_distance_form": (c.c_int32, [vp, vp, vp, vp]),
        "lgp_predict": (c.c_int32, [vp, c.POINTER(lgp_hyper), vp, vp, c.c_int64, vp, c.c_int64,
                                    c.POINTER(lgp_options), vp, vp, c.POINTER(lgp_predict_info), vp]),
        "lgp_kernel_matvec_noalloc": (c.c_int32, [c.POINTER(lgp_hyper), vp, vp, vp, c.c_int64, c.c_int32, c.c_int32,
                                                  vp]),
        "lgp_kernel_matvec_noalloc_status": (c.c_int32, [vp]),
        "lgp_batch_route_choice": (c.c_int32, [vp, c.c_int64, c.c_int32, c.c_int32, c.c_int32]),
        "lgp_batch_split_choice": (c.c_int32, [vp, c.c_int64, c.c_int32, c.c_int32, c.c_int32]),
        "lgp_batch_split_rule": (c.c_int32, [vp, c.c_int64]),
        "lgp_set_kernel_timing": (c.c_int32, [vp, c.c_int32]),
        "lgp_last_kernel_ms": (c.c_int32, [vp, c.POINTER(c.c_float)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(s: int) -> str:
    try:
        return load().lgp_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


@dataclass
class Hyper:
    """Kernel kind and log-space hyperparameters (log l_d, log s^2, log sigma_n^2)."""
    kind: int
    log_lengthscale: np.ndarray
    log_outputscale: float
    log_noise: float

    @classmethod
    def of(cls, p) -> "Hyper":
        return cls(int(p.kind), np.asarray(p.log_lengthscale, dtype=np.float32).copy(), float(p.log_outputscale),
                   float(p.log_noise))

    def to_c(self) -> tuple[lgp_hyper, np.ndarray]:
        ls = np.ascontiguousarray(np.asarray(self.log_lengthscale, dtype=np.float32))
        h = lgp_hyper(int(self.kind), int(ls.shape[0]), ls.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                      float(self.log_outputscale), float(self.log_noise))
        return h, ls  # keep ls alive while h is used


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _f32_dev(a, device):
    import torch
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=torch.float32)
    else:
        t = torch.as_tensor(np.asarray(a, dtype=np.float32), device=device)
    return t.contiguous()


class Context:
    """Owns one lgp_ctx on a CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        self.lib = lib
        self.device = device
        h = ctypes.c_void_p()
        s = lib.lgp_create(ctypes.byref(h), int(device))
        if s != LGP_OK:
            raise LGPError(s, f"lgp_create(device={device}) failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.lgp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int, allow_warn: bool = True) -> int:
        if s < 0 or (s > 0 and not allow_warn):
            raise LGPError(s, self.lib.lgp_last_error_message(self.h).decode())
        return s

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.lgp_workspace_bytes(self.h))

    def matvec_precision(self, t: int, prec: int = LGP_PREC_AUTO) -> int:
        return int(self.lib.lgp_matvec_precision(self.h, int(t), int(prec)))

    def tc_kernel_choice(self, N: int, D: int, kind: int, t: int, prec: int = LGP_PREC_AUTO) -> int:
        """LGP_TC_UNTUNED / LGP_TC_ROW / LGP_TC_SYMMETRIC for that product shape (or a negative status)."""
        return int(self.lib.lgp_tc_kernel_choice(self.h, int(N), int(D), int(kind), int(t), int(prec)))

    def batch_route_choice(self, N: int, D: int, kind: int, t: int) -> int:
        """LGP_BATCH_UNTUNED / LGP_BATCH_PERSISTENT / LGP_BATCH_TENSOR for that batched-problem shape."""
        return int(self.lib.lgp_batch_route_choice(self.h, int(N), int(D), int(kind), int(t)))

    def batch_split_choice(self, N: int, D: int, kind: int, t: int) -> int:
        """Column splits the batched solver chose for that persistent-route problem shape (0: untuned)."""
        return int(self.lib.lgp_batch_split_choice(self.h, int(N), int(D), int(kind), int(t)))

    def set_kernel_timing(self, on: bool) -> None:
        """Record CUDA events around the product kernel of every uncaptured K_y V product."""
        self._check(self.lib.lgp_set_kernel_timing(self.h, 1 if on else 0))

    def last_kernel_ms(self) -> float:
        """Duration of the last timed product kernel (synchronises on its end event)."""
        ms = ctypes.c_float(0.0)
        self._check(self.lib.lgp_last_kernel_ms(self.h, ctypes.byref(ms)))
        return float(ms.value)

    def batch_split_rule(self, N: int) -> int:
        """The fixed rule's column-split count for a problem of N rows alone."""
        return int(self.lib.lgp_batch_split_rule(self.h, int(N)))

    def tc_distance_form(self, stream=None) -> tuple[int, float]:
        """(LGP_DIST_NONE / LGP_DIST_DIFF / LGP_DIST_DOT, max |u|^2 or -1) of the last symmetric product."""
        form = ctypes.c_int32(0)
        amax = ctypes.c_float(0.0)
        self._check(self.lib.lgp_tc_distance_form(self.h, _stream_ptr(stream), ctypes.byref(form), ctypes.byref(amax)))
        return int(form.value), float(amax.value)

    def set_wait_budget(self, cycles: int):
        self.lib.lgp_set_wait_budget(self.h, int(cycles))

    def check_device_status(self, stream=None) -> int:
        return int(self.lib.lgp_check_device_status(self.h, _stream_ptr(stream)))


_default_ctx: dict[int, Context] = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


# ---------------------------------------------------------------------------------------- entry points

def lgp_kernel_matvec(X, hyp, V, prec: int = LGP_PREC_AUTO, out=None, ctx: Context | None = None, stream=None,
                      check: bool = True):
    """out = (K_ff + sigma^2 I) V on the GPU; X [N, D], V [N, t] (or [N]) float32 CUDA tensors."""
    import torch
    ctx = ctx or default_context(X.device.index or 0)
    squeeze = V.dim() == 1
    V2 = V.reshape(-1, 1) if squeeze else V
    N, t = V2.shape
    if out is None:
        out = torch.empty((N, t), device=V.device, dtype=torch.float32)
    h, keep = Hyper.of(hyp).to_c()
    s = ctx.lib.lgp_kernel_matvec(ctx.h, ctypes.byref(h), _ptr(X), _ptr(V2), _ptr(out), int(N), int(t), int(prec),
                                  _stream_ptr(stream))
    if check:
        ctx._check(s)
    del keep
    return out.reshape(-1) if squeeze else out


def lgp_kernel_matvec_noalloc(X, hyp, V, out, prec: int = LGP_PREC_AUTO, stream=None) -> int:
    """K_y V into a caller-provided `out` with no device allocation (N <= 8192, t in {16, 32}).

    For callers that cannot allocate device memory (programs whose device memory belongs to
    another allocator, services under a fixed memory budget, latency-critical loops). Returns
    the lgp_status of the launch; device-side failures are read with
    lgp_kernel_matvec_noalloc_status. The scratch is a fixed array inside the library, so
    overlapping calls on different streams race.
    """
    N, t = V.shape
    h, keep = Hyper.of(hyp).to_c()
    s = load().lgp_kernel_matvec_noalloc(ctypes.byref(h), _ptr(X), _ptr(V), _ptr(out), int(N), int(t), int(prec),
                                         _stream_ptr(stream))
    del keep
    return int(s)


def lgp_kernel_matvec_noalloc_status(stream=None) -> int:
    """Synchronise `stream`, then read and clear the status words of the allocation-free product
    calls on the current device: LGP_OK, LGP_ERR_TIMEOUT or LGP_ERR_NONFINITE."""
    return int(load().lgp_kernel_matvec_noalloc_status(_stream_ptr(stream)))


PIPE_FFMA, PIPE_FFMA2, PIPE_MUFU_EX2, PIPE_MUFU_SQRT = 0, 1, 2, 3


def lgp_measure_pipe_peak(which: int, stream=None) -> float:
    """Measured results/s of one pipe on the current device (see include/lgp.h)."""
    v = ctypes.c_double(0.0)
    s = load().lgp_measure_pipe_peak(int(which), ctypes.byref(v), _stream_ptr(stream))
    if s != LGP_OK:
        raise LGPError(s, "lgp_measure_pipe_peak failed")
    return v.value


def lgp_kernel_matvec_grad(X, hyp, W, ctx: Context | None = None, stream=None):
    """G[p] = dK_y/dtheta_p W for theta = (log l_1..log l_D, log s^2, log sigma^2): [D+2, N, t]."""
    import torch
    ctx = ctx or default_context(X.device.index or 0)
    W2 = W.reshape(-1, 1) if W.dim() == 1 else W
    N, t = W2.shape
    D = X.shape[1]
    G = torch.empty((D + 2, N, t), device=W.device, dtype=torch.float32)
    h, keep = Hyper.of(hyp).to_c()
    ctx._check(ctx.lib.lgp_kernel_matvec_grad(ctx.h, ctypes.byref(h), _ptr(X), _ptr(W2), _ptr(G), int(N), int(t),
                                              _stream_ptr(stream)))
    del keep
    return G


LGP_OPT_WARM_START = 1
LGP_OPT_SINGLE_RHS = 2
LGP_MAX_LANCZOS_STEPS = 1024  # largest lanczos_steps accepted (include/lgp.h)


def _options(tol, max_iter, lanczos_steps=0, n_probes=0, prec=LGP_PREC_AUTO, seed=0, precond_rank=0,
             flags=0) -> lgp_options:
    return lgp_options(float(tol), int(max_iter), int(lanczos_steps), int(n_probes), int(prec),
                       int(seed) & ((1 << 64) - 1), int(precond_rank), int(flags))


def lgp_cg_solve(X, hyp, B, tol: float = 1e-6, max_iter: int = 1000, prec: int = LGP_PREC_AUTO,
                 ctx: Context | None = None, stream=None, out=None, precond_rank: int = 0, x0=None):
    """Solve K_y Xsol = B by batched CG. x0 (optional, [N, t] like B): warm start from that initial guess.
    Returns (Xsol, iters[t], rel_resid[t], status)."""
    import torch
    ctx = ctx or default_context(X.device.index or 0)
    squeeze = B.dim() == 1
    B2 = B.reshape(-1, 1) if squeeze else B
    N, t = B2.shape
    if out is None:
        out = torch.empty((N, t), device=B.device, dtype=torch.float32)
    if x0 is not None:
        out.copy_(x0.reshape(N, t))
    iters = np.zeros(t, dtype=np.int32)
    rel = np.zeros(t, dtype=np.float64)
    h, keep = Hyper.of(hyp).to_c()
    o = _options(tol, max_iter, prec=prec, precond_rank=precond_rank,
                 flags=LGP_OPT_WARM_START if x0 is not None else 0)
    s = ctx._check(ctx.lib.lgp_cg_solve(ctx.h, ctypes.byref(h), _ptr(X), _ptr(B2), _ptr(out), int(N), int(t),
                                        ctypes.byref(o), iters.ctypes.data_as(ctypes.c_void_p),
                                        rel.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    del keep
    return (out.reshape(-1) if squeeze else out), iters, rel, s


def lgp_lml_and_grad(X, y, hyp, n_probes: int = 15, lanczos_steps: int = LGP_MAX_LANCZOS_STEPS, seed: int = 0,
                     tol: float = 1e-4, max_iter: int = 1000, prec: int = LGP_PREC_AUTO, want_grad: bool = True,
                     ctx: Context | None = None, stream=None, precond_rank: int = 0, single_rhs: bool = False):
    """LML estimate, its gradient [D+2] (or None) and an info dict. single_rhs=True: the plain path that
    solves the columns one at a time with the float32 one-column product (LGP_OPT_SINGLE_RHS).

    lanczos_steps defaults to the largest accepted, so the log-determinant quadrature uses every CG step
    of each probe (up to 1024). Shorter tridiagonals truncate it: on a badly conditioned K_y (N=100000,
    D=8, Matern-5/2, noise 0.01) 50 steps move the LML estimate by about 20%. The quadrature's cost is
    negligible next to the solve at any length."""
    ctx = ctx or default_context(X.device.index or 0)
    N = int(y.shape[0])
    D = int(X.shape[1])
    lml = ctypes.c_double(0.0)
    grad = np.zeros(D + 2, dtype=np.float64)
    info = lgp_lml_info()
    h, keep = Hyper.of(hyp).to_c()
    o = _options(tol, max_iter, lanczos_steps, n_probes, prec, seed, precond_rank,
                 flags=LGP_OPT_SINGLE_RHS if single_rhs else 0)
    s = ctx._check(ctx.lib.lgp_lml_and_grad(ctx.h, ctypes.byref(h), _ptr(X), _ptr(y), N, ctypes.byref(o),
                                            ctypes.byref(lml), grad.ctypes.data_as(ctypes.c_void_p) if want_grad
                                            else None, ctypes.byref(info), _stream_ptr(stream)))
    del keep
    d = {k: getattr(info, k) for k, _ in lgp_lml_info._fields_}
    d["status"] = s
    return lml.value, (grad if want_grad else None), d


def lgp_predict(X, y, hyp, Xs, n_probes: int = 0, seed: int = 0, tol: float = 1e-6, max_iter: int = 1000,
                prec: int = LGP_PREC_AUTO, want_var: bool = True, ctx: Context | None = None, stream=None,
                precond_rank: int = 0):
    """Posterior predictive mean [M] and latent variance [M] (or None) at test points Xs [M, D].

    n_probes = 0: exact variance; 1..31: the Rademacher diagonal estimate with that many probes.
    Returns (mean, var, info dict, status)."""
    import torch
    ctx = ctx or default_context(X.device.index or 0)
    N = int(y.shape[0])
    M = int(Xs.shape[0])
    mean = torch.empty(M, device=X.device, dtype=torch.float32)
    var = torch.empty(M, device=X.device, dtype=torch.float32) if want_var else None
    info = lgp_predict_info()
    h, keep = Hyper.of(hyp).to_c()
    o = _options(tol, max_iter, 0, n_probes, prec, seed, precond_rank)
    s = ctx._check(ctx.lib.lgp_predict(ctx.h, ctypes.byref(h), _ptr(X), _ptr(y), N, _ptr(Xs), M, ctypes.byref(o),
                                       _ptr(mean), _ptr(var) if var is not None else None, ctypes.byref(info),
                                       _stream_ptr(stream)), allow_warn=True)
    del keep
    return mean, var, {k: getattr(info, k) for k, _ in info._fields_}, s


def lgp_rademacher_probes(seed: int, N: int, m: int, device: int = 0, ctx: Context | None = None, stream=None):
    """The probes lgp_lml_and_grad draws: [N, m] float32 +-1 on the GPU."""
    import torch
    ctx = ctx or default_context(device)
    Z = torch.empty((N, m), device=f"cuda:{device}", dtype=torch.float32)
    ctx._check(ctx.lib.lgp_rademacher_probes(ctx.h, int(seed) & ((1 << 64) - 1), int(N), int(m), _ptr(Z), int(m),
                                             _stream_ptr(stream)))
    return Z


def lgp_batch_cg_solve(Xs, hyps, Bs, tol: float = 1e-6, max_iter: int = 1000, prec: int = LGP_PREC_AUTO,
                       ctx: Context | None = None, stream=None):
    """Solve many independent GPs of uneven N in one call. Returns (sols, iters[n_gp, t], rel[n_gp, t], status)."""
    import torch
    n = len(Xs)
    ctx = ctx or default_context(Xs[0].device.index or 0)
    t = int(Bs[0].shape[1])
    sols = [torch.empty_like(B) for B in Bs]
    hs = (lgp_hyper * n)()
    keep = []
    for g, hp in enumerate(hyps):
        h, k = Hyper.of(hp).to_c()
        hs[g] = h
        keep.append(k)
    Xp = (ctypes.c_void_p * n)(*[X.data_ptr() for X in Xs])
    Bp = (ctypes.c_void_p * n)(*[B.data_ptr() for B in Bs])
    Sp = (ctypes.c_void_p * n)(*[S.data_ptr() for S in sols])
    Ns = np.array([int(B.shape[0]) for B in Bs], dtype=np.int64)
    iters = np.zeros((n, t), dtype=np.int32)
    rel = np.zeros((n, t), dtype=np.float64)
    o = _options(tol, max_iter, prec=prec)
    s = ctx._check(ctx.lib.lgp_batch_cg_solve(ctx.h, n, hs, ctypes.cast(Xp, ctypes.c_void_p),
                                              ctypes.cast(Bp, ctypes.c_void_p), ctypes.cast(Sp, ctypes.c_void_p),
                                              Ns.ctypes.data_as(ctypes.c_void_p), t, ctypes.byref(o),
                                              iters.ctypes.data_as(ctypes.c_void_p),
                                              rel.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    del keep
    return sols, iters, rel, s


# ---------------------------------------------------------------------------------------- autograd

def _autograd_function():
    import torch

    class LGPMarginalLikelihood(torch.autograd.Function):
        """LML(X, y; log l, log s^2, log sigma^2) with the analytic gradient of the adjoint pass.

        forward(X, y, log_lengthscale, log_outputscale, log_noise, kind, n_probes, lanczos_steps, seed, tol,
        max_iter, prec) -> scalar LML (float64 tensor). The gradient with respect to the three
        hyperparameter tensors is computed in the forward call and scaled by grad_output in backward.
        """

        @staticmethod
        def forward(ctx_, X, y, log_lengthscale, log_outputscale, log_noise, kind=LGP_RBF, n_probes=15,
                    lanczos_steps=LGP_MAX_LANCZOS_STEPS, seed=0, tol=1e-4, max_iter=1000, prec=LGP_PREC_AUTO):
            hyp = Hyper(int(kind), log_lengthscale.detach().cpu().numpy().astype(np.float32),
                        float(log_outputscale.detach().cpu()), float(log_noise.detach().cpu()))
            lml, grad, info = lgp_lml_and_grad(X.detach(), y.detach(), hyp, n_probes, lanczos_steps, seed, tol,
                                               max_iter, prec, want_grad=True)
            D = hyp.log_lengthscale.shape[0]
            g = torch.as_tensor(grad, dtype=torch.float64)
            ctx_.save_for_backward(g)
            ctx_.D = D
            ctx_.dev = log_lengthscale.device
            ctx_.dtypes = (log_lengthscale.dtype, log_outputscale.dtype, log_noise.dtype)
            return torch.tensor(lml, dtype=torch.float64, device=log_lengthscale.device)

        @staticmethod
        def backward(ctx_, grad_out):
            (g,) = ctx_.saved_tensors
            go = grad_out.detach().to("cpu", torch.float64)
            D = ctx_.D
            gl = (go * g[:D]).to(ctx_.dev, ctx_.dtypes[0])
            gs = (go * g[D]).to(ctx_.dev, ctx_.dtypes[1])
            gn = (go * g[D + 1]).to(ctx_.dev, ctx_.dtypes[2])
            return (None, None, gl, gs, gn) + (None,) * 7

    return LGPMarginalLikelihood


_LML_FN = None


def marginal_likelihood(X, y, log_lengthscale, log_outputscale, log_noise, kind=LGP_RBF, **kw):
    """Differentiable LML (see LGPMarginalLikelihood)."""
    global _LML_FN
    if _LML_FN is None:
        _LML_FN = _autograd_function()
    args = [kw.get("n_probes", 15), kw.get("lanczos_steps", LGP_MAX_LANCZOS_STEPS), kw.get("seed", 0), kw.get("tol", 1e-4),
            kw.get("max_iter", 1000), kw.get("prec", LGP_PREC_AUTO)]
    return _LML_FN.apply(X, y, log_lengthscale, log_outputscale, log_noise, kind, *args)


def __getattr__(name):
    if name == "LGPMarginalLikelihood":
        global _LML_FN
        if _LML_FN is None:
            _LML_FN = _autograd_function()
        return _LML_FN
    raise AttributeError(name)
