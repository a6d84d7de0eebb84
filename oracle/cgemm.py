"""ctypes harness of the plain-C DGEMM oracle (dgemm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the benchmark's
CPU-baseline leg.  It never touches the CUDA library and the CUDA library never
touches it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgemm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, p = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_dgemm.argtypes = [i64, i64, i64, dbl, p, i64, p, i64, dbl, p, i64]
            lib.oracle_dgemm.restype = None
            lib.oracle_dgemm_rows.argtypes = [i64, p, i64, i64, dbl, p, i64, p, i64, dbl, p, i64]
            lib.oracle_dgemm_rows.restype = None
            lib.oracle_dgemm_omp.argtypes = [i64, i64, i64, dbl, p, i64, p, i64, dbl, p, i64,
                                             ctypes.c_int, p]
            lib.oracle_dgemm_omp.restype = ctypes.c_int
            lib.oracle_dgemm_dd_rows.argtypes = [i64, p, i64, i64, p, i64, p, i64, p, p, i64]
            lib.oracle_dgemm_dd_rows.restype = None
            lib.oracle_daxpy.argtypes = [i64, dbl, p, p]
            lib.oracle_daxpy.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(a: np.ndarray, rows: int, cols: int, name: str) -> int:
    if a.dtype != np.float64 or a.ndim != 2 or not a.flags.c_contiguous:
        raise ValueError(f"{name} must be a C-contiguous float64 2-D array")
    if a.shape[0] < rows or a.shape[1] < cols:
        raise ValueError(f"{name} too small")
    return a.shape[1]


def dgemm(alpha: float, A: np.ndarray, B: np.ndarray, beta: float = 0.0,
          C: np.ndarray | None = None, m: int | None = None, n: int | None = None,
          k: int | None = None) -> np.ndarray:
    """C <- alpha*A*B + beta*C by the definition; returns C (a new array if None).

    A's, B's and C's second extents are their leading dimensions; m, n, k default
    to the logical shapes (A.shape[0], B.shape[1], A.shape[1])."""
    m = A.shape[0] if m is None else m
    k = A.shape[1] if k is None else k
    n = B.shape[1] if n is None else n
    lda = _check(A, m, k, "A")
    ldb = _check(B, k, n, "B")
    if C is None:
        C = np.zeros((m, n), dtype=np.float64)
    ldc = _check(C, m, n, "C")
    _load().oracle_dgemm(m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc)
    return C


def dgemm_rows(rows, alpha: float, A: np.ndarray, B: np.ndarray, beta: float = 0.0,
               C_rows: np.ndarray | None = None, n: int | None = None,
               k: int | None = None) -> np.ndarray:
    """Rows ``rows`` of alpha*A*B + beta*C; ``C_rows`` holds those rows of C."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    k = A.shape[1] if k is None else k
    n = B.shape[1] if n is None else n
    lda = _check(A, int(rows.max(initial=-1)) + 1, k, "A")
    ldb = _check(B, k, n, "B")
    if C_rows is None:
        C_rows = np.zeros((len(rows), n), dtype=np.float64)
    ldc = _check(C_rows, len(rows), n, "C_rows")
    _load().oracle_dgemm_rows(len(rows), _ptr(rows), n, k, alpha, _ptr(A), lda, _ptr(B), ldb,
                              beta, _ptr(C_rows), ldc)
    return C_rows


def dgemm_omp(alpha: float, A: np.ndarray, B: np.ndarray, beta: float = 0.0,
              C: np.ndarray | None = None, threads: int | None = None,
              m: int | None = None):
    """The definition over OpenMP threads (bit-identical to ``dgemm``).

    Returns (C, threads actually used)."""
    m = A.shape[0] if m is None else m
    k, n = A.shape[1], B.shape[1]
    lda = _check(A, m, k, "A")
    ldb = _check(B, k, n, "B")
    if C is None:
        C = np.zeros((m, n), dtype=np.float64)
    ldc = _check(C, m, n, "C")
    threads = os.cpu_count() if threads is None else threads
    work = np.empty(max(1, threads) * max(1, n), dtype=np.float64)
    used = _load().oracle_dgemm_omp(m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                                    _ptr(C), ldc, threads, _ptr(work))
    return C, used


def dgemm_dd_rows(A: np.ndarray, B: np.ndarray, rows=None, n: int | None = None,
                  k: int | None = None):
    """Double-double value (hi, lo) of A*B for the given rows (all when None)."""
    k = A.shape[1] if k is None else k
    n = B.shape[1] if n is None else n
    lda = _check(A, 1, k, "A")
    ldb = _check(B, k, n, "B")
    if rows is None:
        nrows, rp = A.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nrows, rp = len(rows), rows
    hi = np.empty((nrows, n), dtype=np.float64)
    lo = np.empty((nrows, n), dtype=np.float64)
    _load().oracle_dgemm_dd_rows(nrows, _ptr(rp), n, k, _ptr(A), lda, _ptr(B), ldb,
                                 _ptr(hi), _ptr(lo), n)
    return hi, lo


def daxpy(alpha: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """y <- fma(alpha, x, y) elementwise (in place on a float64 copy); returns y."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.array(y, dtype=np.float64, copy=True)
    if x.shape != y.shape:
        raise ValueError("x and y differ in shape")
    _load().oracle_daxpy(x.size, alpha, _ptr(x), _ptr(y))
    return y
