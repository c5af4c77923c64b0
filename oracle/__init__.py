"""CPU oracle for the matrix-free GP path: test infrastructure, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. ``gp_oracle`` is the float64 NumPy definition of every
quantity the CUDA path computes; ``oracle_mv.c`` is a float64 OpenMP row-streamed
product for problem sizes where an explicit matrix does not fit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .gp_oracle import *  # noqa: F401,F403
from . import gp_oracle

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle_mv.so")
_lib = None


def build_oracle_lib(force: bool = False) -> str:
    """Compile oracle_mv.c with gcc (-O2 -fopenmp, no host-specific flags)."""
    src = os.path.join(_HERE, "oracle_mv.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_oracle_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_kyv_rows.restype = ctypes.c_int
        lib.oracle_kyv_rows.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int32]
        lib.oracle_kxv_rows.restype = ctypes.c_int
        lib.oracle_kxv_rows.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]
        _lib = lib
    return _lib


def kyv_rows_c(X, V, hyp, rows=None, n_threads: int = 0):
    """Rows of K_y V in float64 from the C streaming oracle; returns (out, threads used)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float32)
    V2 = V[:, None] if V.ndim == 1 else V
    V2 = np.ascontiguousarray(V2)
    N, D = X.shape
    t = V2.shape[1]
    if t > 256 or D > 64:
        raise ValueError("oracle_kyv_rows supports t <= 256 and D <= 64")
    ls = np.ascontiguousarray(hyp.lengthscale, dtype=np.float64)
    if rows is None:
        nrows = N
        rows_arr = None
        rows_ptr = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = rows_arr.shape[0]
        rows_ptr = rows_arr.ctypes.data
    out = np.empty((nrows, t), dtype=np.float64)
    used = lib.oracle_kyv_rows(X.ctypes.data, N, D, ls.ctypes.data, hyp.s2, hyp.noise, int(hyp.kind),
                               V2.ctypes.data, t, rows_ptr, nrows, out.ctypes.data, int(n_threads))
    return (out[:, 0] if V.ndim == 1 else out), used


def kxv_c(Xr, X, V, hyp, n_threads: int = 0):
    """K(Xr, X) V in float64 (no noise term) from the C streaming oracle; returns (out, threads used)."""
    lib = _load()
    Xr = np.ascontiguousarray(Xr, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float32)
    V2 = np.ascontiguousarray(V[:, None] if V.ndim == 1 else V)
    N, D = X.shape
    Nr = Xr.shape[0]
    t = V2.shape[1]
    if t > 256 or D > 64 or Xr.shape[1] != D:
        raise ValueError("oracle_kxv_rows supports t <= 256, D <= 64 and matching dimensions")
    ls = np.ascontiguousarray(hyp.lengthscale, dtype=np.float64)
    out = np.empty((Nr, t), dtype=np.float64)
    used = lib.oracle_kxv_rows(Xr.ctypes.data, Nr, X.ctypes.data, N, D, ls.ctypes.data, hyp.s2, int(hyp.kind),
                               V2.ctypes.data, t, out.ctypes.data, int(n_threads))
    return (out[:, 0] if V.ndim == 1 else out), used
