"""Shared helpers of the GPU parity tests (seeded inputs, oracle comparisons)."""
import numpy as np

from oracle import cgemm, exact
from synth import generators as g


def torch_mod():
    import torch
    return torch


def to_dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def inputs(kind, m, n, k, seed, with_c=True):
    A = g.matrix(kind, m, k, seed, g.STREAM_A)
    B = g.matrix(kind, k, n, seed, g.STREAM_B)
    C0 = g.matrix(kind, m, n, seed, g.STREAM_C) if with_c else np.zeros((m, n))
    return A, B, C0


def within_bound(C_test, alpha, A, B, beta, C0, rows=None):
    """max |C_test - C*| / bound over the given rows (all when None); C* from the
    double-double reference, exact residuals."""
    k = A.shape[1]
    if rows is None:
        hi, lo = cgemm.dgemm_dd_rows(A, B)
        absab = cgemm.dgemm(1.0, np.abs(A), np.abs(B))
        c0 = C0
    else:
        rows = np.asarray(rows)
        hi, lo = cgemm.dgemm_dd_rows(A, B, rows)
        absab = cgemm.dgemm_rows(rows, 1.0, np.abs(A), np.abs(B))
        c0 = C0[rows] if C0 is not None else None
    res = exact.residual(C_test, alpha, hi, lo, beta, c0)
    bound = exact.error_bound(k, alpha, absab, beta, c0)
    ratio = np.abs(res) / np.where(bound > 0, bound, np.inf)
    ratio = np.where((res == 0), 0.0, ratio)
    return float(np.max(ratio)) if ratio.size else 0.0


def e4m3_decode(b: np.ndarray) -> np.ndarray:
    """Value of E4M3 bytes (OCP FP8 E4M3: bias 7, 3 mantissa bits, no infinities)."""
    b = b.astype(np.int64)
    sign = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    mnt = b & 7
    val = np.where(e == 0, np.ldexp(mnt / 8.0, -6), np.ldexp(1.0 + mnt / 8.0, e - 7))
    return sign * val
