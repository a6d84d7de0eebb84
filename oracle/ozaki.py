"""CPU model of the split-precision (Ozaki-style) FP64 GEMM, step by step.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

The paper's method is the FP64 GEMM C <- alpha*A*B + beta*C (Section 4.2).  The
split-precision path reaches an approximation of that same result in four steps;
this module restates each one plainly, in FP64 and exact integers, so the CUDA
kernels can be compared with it step by step:

  e1  exponents: e_i = exponent of max_l |A[i,l]| (frexp convention, so
      max_l |A[i,l]| < 2^e_i), f_j = exponent of max_l |B[l,j]|.  A zero row
      gets 0.  A row or column holding a NaN or Inf is flagged.
  e2  slicing: x = A[i,l] * 2^-e_i lies in (-1, 1).  Signed digits by
      round-to-nearest-even: d_1 = rint(x * 2^b1), r_1 = x * 2^b1 - d_1, and for
      t >= 2  d_t = rint(r_{t-1} * 2^b), r_t = r_{t-1} * 2^b - d_t.  Every step is
      exact in FP64 (power-of-two scalings and the difference of two numbers
      within 1/2 of each other), so
          A[i,l] = 2^e_i ( sum_{t=1..s} d_t 2^-(b1 + b (t-1)) + r_s 2^-(b1 + b (s-1)) ),
      |r_s| <= 1/2.  B is sliced the same way per column j with exponent f_j.
      E4M3 digits: b1 = 4, b = 5, |d| <= 16 (every such integer is exact in E4M3).
  e3  level sums: S_g = sum_{p+q=g} DA_p DB_q over 2 <= g <= s+1 (pairs with
      p + q > s + 1 are dropped), exact integers.
  e4  recombination: the levels are summed exactly as one integer in units of
      the smallest level, T = sum_{g=2..s+1} S_g 2^(b (s+1-g)); the exact value
      T * 2^E, E = e_i + f_j - 2 b1 - b (s-1), is rounded once to FP64:
      t = RN(T * 2^E), round to nearest with ties to even, gradual underflow
      (subnormal results) and overflow to +-inf, as one IEEE operation on the
      exact value would round it.  Then C = alpha * t + beta * C0 with each
      product and the sum one IEEE rounding (beta = 0: C0 not read; alpha = 1
      and beta = 0: C = t).  Rows of A or columns of B flagged in e1 give NaN
      outputs.

BLAS conventions as for the FP64 oracle: alpha == 0 or k == 0 gives beta*C0
(0 when beta == 0); m == 0 or n == 0 is empty.
"""
from __future__ import annotations

import math

import numpy as np

#: digit formats: name -> (b1, b, max |digit|)
FORMATS = {
    "e4m3": (4, 5, 16),
    "bf16": (7, 8, 128),
}


def exponents(X: np.ndarray, axis: int):
    """e1: frexp exponent of max |X| along ``axis`` and a non-finite flag per line."""
    X = np.asarray(X, dtype=np.float64)
    finite = np.isfinite(X)
    bad = ~finite.all(axis=axis)
    mx = np.where(finite, np.abs(X), 0.0).max(axis=axis, initial=0.0)
    _, e = np.frexp(mx)
    e = e.astype(np.int64)
    e[bad] = 0
    return e, bad


def slice_digits(X: np.ndarray, e: np.ndarray, s: int, fmt: str = "e4m3", axis: int = 1,
                 bad: np.ndarray | None = None):
    """e2: signed digits of X scaled by 2^-e along ``axis`` (e per row: axis=1).

    Lines flagged ``bad`` (non-finite, from e1) get all-zero digits.
    Returns (digits of shape (s,) + X.shape, final remainders r_s); the digits
    are int8 for E4M3 (|d| <= 16) and int16 for BF16 (|d| <= 128 does not fit
    int8)."""
    b1, b, dmax = FORMATS[fmt]
    X = np.asarray(X, dtype=np.float64)
    eb = e[:, None] if axis == 1 else e[None, :]
    Xf = np.where(np.isfinite(X), X, 0.0)
    if bad is not None:
        Xf = np.where(bad[:, None] if axis == 1 else bad[None, :], 0.0, Xf)
    x = np.ldexp(Xf, -eb)
    dtype = np.int8 if dmax <= 127 else np.int16
    D = np.zeros((s,) + X.shape, dtype=dtype)
    y = x * float(2 ** b1)
    for t in range(s):
        if t > 0:
            y = r * float(2 ** b)
        d = np.rint(y)
        r = y - d
        assert np.abs(d).max(initial=0) <= dmax
        D[t] = d.astype(dtype)
    return D, r


def level_sums(DA: np.ndarray, DBt: np.ndarray, s: int) -> np.ndarray:
    """e3: S[g-2] = sum_{p+q=g} DA_p @ DBt_q^T for g = 2..s+1 (exact int64).

    DA: (s, m, k) digits of A's rows; DBt: (s, n, k) digits of B's columns.
    The products are formed by a float64 matrix multiply: every digit product
    is an integer of magnitude <= dmax^2 (256 for E4M3 digits, 2^14 for BF16
    digits) and every partial sum an integer far below 2^53, so the library
    matmul is exact whatever its summation order."""
    m, n = DA.shape[1], DBt.shape[1]
    S = np.zeros((s, m, n), dtype=np.int64)
    dmax = max(int(np.abs(DA).max(initial=0)), int(np.abs(DBt).max(initial=0)), 1)
    assert DA.shape[2] * s * dmax * dmax < 2 ** 53
    fa = [DA[p].astype(np.float64) for p in range(s)]
    for q in range(1, s + 1):
        fbq = DBt[q - 1].astype(np.float64).T      # one plane at a time (memory)
        for p in range(1, s + 2 - q):
            S[p + q - 2] += (fa[p - 1] @ fbq).astype(np.int64)
    return S


def round_scaled(T: int, E: int) -> float:
    """RN(T * 2^E) for a Python integer T and any integer E: the double nearest to
    the exact value (ties to even), subnormal when it lies below 2^-1022, +-inf
    when it rounds beyond the largest double.  Python's int -> float conversion
    and int / int true division are both correctly rounded, so the exact value
    is handed to one of them whole."""
    T, E = int(T), int(E)
    if T == 0:
        return 0.0
    try:
        return float(T << E) if E >= 0 else T / (1 << -E)
    except OverflowError:
        return math.copysign(math.inf, T)


def recombine(S: np.ndarray, e: np.ndarray, f: np.ndarray, alpha: float, beta: float = 0.0,
              C0: np.ndarray | None = None, fmt: str = "e4m3",
              bad_rows=None, bad_cols=None) -> np.ndarray:
    """e4: exact integer sum of the levels, T * 2^E rounded once to FP64, then
    alpha/beta."""
    b1, b, _ = FORMATS[fmt]
    s = S.shape[0]
    T = np.zeros(S.shape[1:], dtype=object)
    for g in range(2, s + 2):                   # Horner form of sum S_g 2^(b(s+1-g))
        T = T * (2 ** b) + S[g - 2].astype(object)
    E = e[:, None] + f[None, :] - (2 * b1 + b * (s - 1))
    t = (np.vectorize(round_scaled, otypes=[np.float64])(T, E) if T.size
         else np.zeros(T.shape))
    if alpha == 1.0 and beta == 0.0:
        out = t.copy()
    else:
        out = alpha * t
        if beta != 0.0:
            out = out + beta * np.asarray(C0, dtype=np.float64)
    if bad_rows is not None:
        out[np.asarray(bad_rows, dtype=np.int64), :] = np.nan
    if bad_cols is not None:
        out[:, np.asarray(bad_cols, dtype=np.int64)] = np.nan
    return out


def emulated_gemm(alpha: float, A: np.ndarray, B: np.ndarray, beta: float = 0.0,
                  C0: np.ndarray | None = None, s: int = 10, fmt: str = "e4m3",
                  rows=None, details: bool = False):
    """alpha*A*B + beta*C0 by steps e1-e4.  ``rows`` restricts the output rows
    (C0 then holds only those rows).  With ``details`` also returns the
    intermediate values of every step."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    n = B.shape[1]
    if rows is not None:
        A = A[np.asarray(rows)]
        m = A.shape[0]
    if m == 0 or n == 0:
        return np.zeros((m, n))
    if alpha == 0.0 or k == 0:
        out = np.zeros((m, n)) if beta == 0.0 else beta * np.asarray(C0, dtype=np.float64)
        return (out, {}) if details else out
    e, bad_r = exponents(A, axis=1)
    f, bad_c = exponents(B, axis=0)
    DA, _ = slice_digits(A, e, s, fmt, axis=1, bad=bad_r)
    DB, _ = slice_digits(B, f, s, fmt, axis=0, bad=bad_c)      # (s, k, n)
    DBt = np.ascontiguousarray(DB.transpose(0, 2, 1))  # (s, n, k)
    S = level_sums(DA, DBt, s)
    out = recombine(S, e, f, alpha, beta, C0, fmt, np.nonzero(bad_r)[0], np.nonzero(bad_c)[0])
    if details:
        return out, dict(e=e, f=f, DA=DA, DBt=DBt, S=S, bad_rows=bad_r, bad_cols=bad_c)
    return out


def reconstruct(D: np.ndarray, r: np.ndarray | None, e: np.ndarray, fmt: str = "e4m3",
                axis: int = 1):
    """Inverse of e2 in exact rationals' stead: returns the FP64 sum of the digit
    terms plus remainder (exact when it fits 53 bits), used by the pins."""
    b1, b, _ = FORMATS[fmt]
    s = D.shape[0]
    x = np.zeros(D.shape[1:])
    for t in range(s - 1, -1, -1):
        x = x + D[t].astype(np.float64) * 2.0 ** -(b1 + b * t)
    if r is not None:
        x = x + r * 2.0 ** -(b1 + b * (s - 1))
    eb = e[:, None] if axis == 1 else e[None, :]
    return np.ldexp(x, eb)
