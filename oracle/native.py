"""Build and call the plain C part of the oracle (gemm_ref.c) through ctypes.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "gemm_ref.c")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gemm_ref.c with gcc (no fused multiply-add, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            i64, dp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            l.oracle_dgemm.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, ip]
            l.oracle_dgemm.restype = None
            l.oracle_dot2_entries.argtypes = [i64, i64, i64, dp, i64, dp, i64, i64,
                                              dp, dp, dp, dp, ip]
            l.oracle_dot2_entries.restype = None
            _lib = l
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def _f64c(x):
    x = np.asarray(x, dtype=np.float64)
    return np.ascontiguousarray(x)


def dgemm(A: np.ndarray, B: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """C = A x B by the plain triple loop (k ascending per element)."""
    A, B = _f64c(A), _f64c(B)
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = np.empty((M, N), dtype=np.float64)
    lib().oracle_dgemm(M, N, K, A.ctypes.data, K, B.ctypes.data, N, C.ctypes.data,
                       N, nthreads or default_threads())
    return C


def dot2_entries(A: np.ndarray, B: np.ndarray, rows, cols,
                 nthreads: int | None = None):
    """Near-exact C_ij (Dot2) and (|A||B|)_ij at the listed entries."""
    A, B = _f64c(A), _f64c(B)
    M, K = A.shape
    _, N = B.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    if rows.shape != cols.shape:
        raise ValueError("rows and cols differ in shape")
    if rows.size and (rows.min() < 0 or rows.max() >= M or cols.min() < 0
                      or cols.max() >= N):
        raise ValueError("entry index out of range")
    c = np.empty(rows.size, dtype=np.float64)
    ab = np.empty(rows.size, dtype=np.float64)
    lib().oracle_dot2_entries(M, N, K, A.ctypes.data, K, B.ctypes.data, N, rows.size,
                              rows.ctypes.data, cols.ctypes.data, c.ctypes.data,
                              ab.ctypes.data, nthreads or default_threads())
    return c, ab


def dot2_full(A: np.ndarray, B: np.ndarray, nthreads: int | None = None):
    """Dot2 reference and |A||B| for every entry (small shapes only)."""
    M, N = A.shape[0], B.shape[1]
    ii, jj = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    c, ab = dot2_entries(A, B, ii.ravel(), jj.ravel(), nthreads)
    return c.reshape(M, N), ab.reshape(M, N)
