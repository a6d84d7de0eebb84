"""Exact and error-measuring references for C <- alpha*A*B + beta*C.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

* ``fraction_gemm``: the definition of Section 4.2 evaluated in exact rational
  arithmetic (Python ``fractions.Fraction``): every double is a dyadic rational,
  so this is the mathematically exact C* for tiny inputs.
* ``error_bound``: the accuracy contract for an FP64 GEMM of inner length k,
  |C - C*|_ij <= 2 (k + 2) u (|alpha| (|A||B|)_ij + |beta| |C0_ij|), u = 2^-53.
  With alpha = 1, beta = 0 this is the classical 2 k u (|A||B|)_ij dot-product
  bound (Higham, "Accuracy and Stability of Numerical Algorithms", 2nd ed., 3.1)
  up to the k + 2 that covers the alpha, beta scaling and the final sum.
* ``residual``: C_test - C* computed from the double-double value of A*B with
  error-free products and a correctly rounded sum (``math.fsum``), so the
  residual itself carries no rounding error of FP64 size.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

U = 2.0 ** -53


def fraction_gemm(alpha, A, B, beta=0.0, C0=None):
    """Exact rational alpha*A*B + beta*C0 for small dense 2-D arrays (lists of lists)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    n = B.shape[1]
    fa, fb = Fraction(alpha), Fraction(beta)
    out = [[Fraction(0)] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            s = Fraction(0)
            for l in range(k):
                s += Fraction(float(A[i, l])) * Fraction(float(B[l, j]))
            v = fa * s
            if beta != 0.0:
                v += fb * Fraction(float(C0[i, j]))
            out[i][j] = v
    return out


def error_bound(k: int, alpha: float, absAB: np.ndarray, beta: float = 0.0,
                C0: np.ndarray | None = None) -> np.ndarray:
    """2 (k + 2) u (|alpha| (|A||B|) + |beta| |C0|), elementwise."""
    b = abs(alpha) * absAB
    if beta != 0.0 and C0 is not None:
        b = b + abs(beta) * np.abs(C0)
    return 2.0 * (k + 2) * U * b


_SPLIT = 134217729.0  # 2^27 + 1, Veltkamp splitting constant


def two_prod(a: np.ndarray, b: np.ndarray):
    """Dekker's error-free product: a*b = p + e exactly (no overflow assumed)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = a * b
    ca = _SPLIT * a
    ah = ca - (ca - a)
    al = a - ah
    cb = _SPLIT * b
    bh = cb - (cb - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def residual(C_test: np.ndarray, alpha: float, hi: np.ndarray, lo: np.ndarray,
             beta: float = 0.0, C0: np.ndarray | None = None) -> np.ndarray:
    """C_test - (alpha*(hi + lo) + beta*C0), each entry rounded once."""
    C_test = np.asarray(C_test, dtype=np.float64)
    p1, e1 = two_prod(np.full_like(hi, alpha), hi)
    t1 = alpha * lo
    if beta != 0.0 and C0 is not None:
        p2, e2 = two_prod(np.full_like(hi, beta), C0)
    else:
        p2 = e2 = np.zeros_like(hi)
    out = np.empty_like(hi)
    ct, a1, b1, c1, a2, b2 = (x.ravel() for x in (C_test, p1, e1, t1, p2, e2))
    o = out.ravel()
    for idx in range(o.size):
        if not math.isfinite(ct[idx]):
            o[idx] = math.inf
            continue
        o[idx] = math.fsum((ct[idx], -a1[idx], -b1[idx], -c1[idx], -a2[idx], -b2[idx]))
    return out
