"""CPU model of the FP64 GEMM by residue arithmetic (the Chinese-remainder form of
the split-precision GEMM), step by step.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

The method computes C <- alpha*A*B + beta*C (Section 4.2) from exact integer
products on low-precision tensor cores.  Instead of cutting each operand into
digit slices whose pair products are summed by level (oracle/ozaki.py), this
form scales each operand to integers once and multiplies the integers modulo
several small pairwise-coprime moduli; the Chinese remainder theorem then gives
the exact integer product back.  The steps, in order:

  c1  exponents: e_i = frexp exponent of max_l |A[i,l]| (max < 2^e_i), f_j of
      max_l |B[l,j]|, as in oracle/ozaki.exponents; NaN/Inf lines are flagged.
  c2  integer scaling: with N moduli m_1 .. m_N of product M and K = k, take the
      largest bit count b (1 <= b <= 62) with K * 2^(2b) <= M / 4, and
      A'[i,l] = rint(A[i,l] 2^(b - e_i)), B'[l,j] = rint(B[l,j] 2^(b - f_j))
      (round to nearest, ties to even; exact in FP64: a power-of-two scaling then
      one rounding), so |A'|, |B'| <= 2^b and |(A'B')[i,j]| <= M / 4.
  c3  residues: R^A_t = A' mod m_t in the symmetric representative: for
      u = |A'| mod m_t, sym(u) = u when 2u <= m_t, else u - m_t, with the sign
      of A' (every modulus is odd, so |R| <= (m_t - 1) / 2 <= 256, an integer
      exact in BF16).
  c4  residue products: P_t = R^A_t R^B_t, exact integers, reduced to
      c_t = sym(P_t mod m_t) (the sign of P_t kept as in c3).
  c5  reconstruction: the integer C' with C' = c_t (mod m_t) for every t and
      |C'| < M / 2, i.e. C' = (sum_t c_t w_t) mod M in the symmetric range, with
      w_t = (M / m_t) ((M / m_t)^-1 mod m_t); since |A'B'| <= M / 4, C' = A'B'.
  c6  C = alpha RN(C' 2^(e_i + f_j - 2b)) + beta C0: one rounding of the exact
      value (oracle/ozaki.round_scaled), then alpha / beta as in
      oracle/ozaki.recombine; flagged lines give NaN.

The only approximation is c2 (each operand rounded to b bits of its line's
scale); c3 - c6 are exact.  BLAS conventions as for the FP64 oracle.
"""
from __future__ import annotations

import numpy as np

from .ozaki import exponents, round_scaled

#: the moduli, largest first: the largest odd primes below 513, so that a
#: symmetric residue has |r| <= 256 and a product of two residues |r r'| <= 2^16
MODULI = (509, 503, 499, 491, 487, 479, 467, 463, 461, 457, 449, 443, 439, 433, 431, 421)

#: default number of moduli
DEFAULT_N = 13


def moduli(N: int) -> tuple:
    """The first N moduli."""
    if not 1 <= N <= len(MODULI):
        raise ValueError(f"1 <= N <= {len(MODULI)}")
    return MODULI[:N]


def modulus_product(N: int) -> int:
    M = 1
    for m in moduli(N):
        M *= m
    return M


def scale_bits(N: int, k: int) -> int:
    """c2: the largest b in [1, 62] with k 2^(2b) <= M / 4 (exact integers), or 0
    when even b = 1 violates it."""
    M = modulus_product(N)
    k = max(int(k), 1)
    b = 0
    for cand in range(1, 63):
        if 4 * k * (1 << (2 * cand)) <= M:
            b = cand
    return b


def scale_to_integers(X: np.ndarray, e: np.ndarray, b: int, axis: int = 1,
                      bad: np.ndarray | None = None) -> np.ndarray:
    """c2: rint(X 2^(b - e)) along lines (axis=1: rows of A, axis=0: columns of B)
    as int64; flagged lines give 0."""
    X = np.asarray(X, dtype=np.float64)
    eb = e[:, None] if axis == 1 else e[None, :]
    with np.errstate(over="ignore", invalid="ignore"):
        Y = np.rint(np.ldexp(np.where(np.isfinite(X), X, 0.0), b - eb))
    Y = Y.astype(np.int64)
    if bad is not None and bad.any():
        if axis == 1:
            Y[bad, :] = 0
        else:
            Y[:, bad] = 0
    return Y


def sym_mod(X, m: int):
    """c3: the symmetric residue of integers X (numpy int64 or object arrays, or
    Python ints) modulo odd m, with the sign of X: sign(X) sym(|X| mod m).
    int64 arrays (|X| < 2^63) are reduced with numpy's integer operations, other
    integers one by one; both are exact."""
    X = np.asarray(X)
    if X.dtype == np.int64:
        u = np.abs(X) % m
        s = np.where(2 * u <= m, u, u - m)
        return np.where(X < 0, -s, s).astype(np.int64)
    X = X.astype(object)
    u = np.vectorize(lambda x: abs(int(x)) % m, otypes=[object])(X) if X.size else X
    s = np.vectorize(lambda v: v if 2 * v <= m else v - m, otypes=[object])(u) if X.size else u
    sign = np.vectorize(lambda x: -1 if int(x) < 0 else 1, otypes=[object])(X) if X.size else X
    return (s * sign).astype(np.int64) if X.size else np.zeros(X.shape, dtype=np.int64)


def residues(Xi: np.ndarray, N: int) -> np.ndarray:
    """c3 for every modulus: (N, ...) int64 of symmetric residues."""
    return np.stack([sym_mod(Xi, m) for m in moduli(N)])


def residue_products(RA: np.ndarray, RB: np.ndarray, N: int) -> np.ndarray:
    """c4: c_t = sym(R^A_t R^B_t mod m_t), int64 (N, m, n).  The products are
    integers of magnitude at most k 256^2: below 2^53 (k < 2^37) every partial sum
    of an FP64 matrix product is an exactly representable integer, whatever its
    order, so the FP64 product is exact; longer K takes the int64 product."""
    k = RA.shape[-1]
    exact_fp64 = k * 256 * 256 < 2 ** 53
    out = []
    for t, m in enumerate(moduli(N)):
        if exact_fp64:
            P = (RA[t].astype(np.float64) @ RB[t].astype(np.float64)).astype(np.int64)
        else:
            P = RA[t].astype(np.int64) @ RB[t].astype(np.int64)
        out.append(sym_mod(P, m))
    return np.stack(out)


def crt(c: np.ndarray, N: int) -> np.ndarray:
    """c5: the integers (object array) congruent to c_t mod m_t with |C'| < M/2."""
    ms = moduli(N)
    M = modulus_product(N)
    w = []
    for m in ms:
        Mt = M // m
        w.append(Mt * pow(Mt % m, -1, m))
    S = np.zeros(c.shape[1:], dtype=object)
    for t in range(N):
        S = S + c[t].astype(object) * w[t]
    r = np.vectorize(lambda v: v % M, otypes=[object])(S) if S.size else S
    return np.vectorize(lambda v: v - M if 2 * v > M else v, otypes=[object])(r) if S.size else r


def finish(Cp: np.ndarray, e: np.ndarray, f: np.ndarray, b: int, alpha: float, beta: float,
           C0, bad_rows, bad_cols) -> np.ndarray:
    """c6: RN(C' 2^(e_i + f_j - 2b)), then alpha / beta; flagged lines NaN."""
    E = e[:, None] + f[None, :] - 2 * b
    t = (np.vectorize(round_scaled, otypes=[np.float64])(Cp, E) if Cp.size
         else np.zeros(Cp.shape))
    if alpha == 1.0 and beta == 0.0:
        out = t.copy()
    else:
        out = alpha * t
        if beta != 0.0:
            out = out + beta * np.asarray(C0, dtype=np.float64)
    out[np.asarray(bad_rows, dtype=np.int64), :] = np.nan
    out[:, np.asarray(bad_cols, dtype=np.int64)] = np.nan
    return out


def crt_gemm(alpha: float, A: np.ndarray, B: np.ndarray, beta: float = 0.0,
             C0: np.ndarray | None = None, N: int = DEFAULT_N, rows=None, cols=None,
             details: bool = False):
    """alpha*A*B + beta*C0 by steps c1-c6.  ``rows`` / ``cols`` restrict the output
    rows / columns (C0 then holds only those; each line's scaling depends on that
    line alone and b on k, so the selected outputs are those of the full product)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if rows is not None:
        A = A[np.asarray(rows)]
    if cols is not None:
        B = B[:, np.asarray(cols)]
    m, k = A.shape
    n = B.shape[1]
    if m == 0 or n == 0:
        return np.zeros((m, n))
    if alpha == 0.0 or k == 0:
        out = np.zeros((m, n)) if beta == 0.0 else beta * np.asarray(C0, dtype=np.float64)
        return (out, {}) if details else out
    b = scale_bits(N, k)
    if b == 0:
        raise ValueError("k too large for this number of moduli")
    e, bad_r = exponents(A, axis=1)
    f, bad_c = exponents(B, axis=0)
    Ai = scale_to_integers(A, e, b, axis=1, bad=bad_r)
    Bi = scale_to_integers(B, f, b, axis=0, bad=bad_c)
    RA = residues(Ai, N)
    RB = residues(Bi, N)
    c = residue_products(RA, RB, N)
    Cp = crt(c, N)
    out = finish(Cp, e, f, b, alpha, beta, C0, np.nonzero(bad_r)[0], np.nonzero(bad_c)[0])
    if details:
        return out, dict(b=b, e=e, f=f, Ai=Ai, Bi=Bi, RA=RA, RB=RB, c=c, Cp=Cp,
                         bad_rows=bad_r, bad_cols=bad_c)
    return out
