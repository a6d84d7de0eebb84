"""Counter-based seeded generators for the synthetic DGEMM workloads.

Every value is a pure function of (seed, stream id, element index), so a test
can regenerate any single row of a large matrix without producing the rest.

Generator: splitmix64 (Steele, Lea, Flood, OOPSLA 2014). Output number ``i``
(0-based) of the sequence started from ``seed`` is ``mix(seed + (i+1)*gamma)``
with ``gamma = 0x9E3779B97F4A7C15`` and the published finaliser

    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)

all modulo 2**64.  Stream ``sid`` of a seed uses counters starting at
``sid << 40``, so streams never overlap for matrices below 2**40 elements.

Value maps (the workload recipes; all bit-reproducible on any IEEE host since
they use integer operations, exact power-of-two scalings and one rounding):
  * uniform[-1, 1):   2 * ((x >> 11) * 2**-53) - 1
  * integers [-8, 8]: ((x >> 11) mod 17) - 8
  * hard set:         sign from bit 0, binade E = ((x >> 1) & 2047) mod 54 - 27,
                      significand 1 + (x >> 12) * 2**-52, value = +-(1+f) * 2**E;
                      magnitudes span [2**-27, 2**27) ~ [7.5e-9, 1.3e8], i.e. the
                      16 decades of the log-uniform [1e-8, 1e8] recipe with a
                      uniform binade and a uniform significand inside it.
  * log-uniform integers in [a, b]: round(exp(ln a + U ln(b/a))), U = (x>>11) 2**-53.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_SHIFT = 40

#: Base seed of every synthetic workload; workload ``c`` uses ``BASE_SEED + c``.
BASE_SEED = 1602084770

#: Stream ids of the operands of one GEMM.
STREAM_A, STREAM_B, STREAM_C = 0, 1, 2


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Outputs of splitmix64 started at ``seed``, at the given 0-based counters."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def raw_stream(seed: int, stream_id: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit draws of stream ``stream_id`` starting at ``offset``."""
    base = (int(stream_id) << _STREAM_SHIFT) + int(offset)
    counters = np.arange(count, dtype=np.uint64) + np.uint64(base)
    return splitmix64(seed, counters)


def _unit(x: np.ndarray) -> np.ndarray:
    """53-bit uniform in [0, 1)."""
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(x: np.ndarray) -> np.ndarray:
    return 2.0 * _unit(x) - 1.0


def integers_pm8(x: np.ndarray) -> np.ndarray:
    return ((x >> np.uint64(11)) % np.uint64(17)).astype(np.float64) - 8.0


def hard_magnitudes(x: np.ndarray) -> np.ndarray:
    sign = np.where((x & np.uint64(1)) == np.uint64(1), -1.0, 1.0)
    binade = (((x >> np.uint64(1)) & np.uint64(2047)) % np.uint64(54)).astype(np.int64) - 27
    frac = (x >> np.uint64(12)).astype(np.float64) * (2.0 ** -52)
    return sign * np.ldexp(1.0 + frac, binade)


_KINDS = {
    "uniform": uniform_pm1,
    "int8": integers_pm8,
    "hard": hard_magnitudes,
}


def log_uniform_ints(seed: int, stream_id: int, count: int, lo: int, hi: int) -> np.ndarray:
    u = _unit(raw_stream(seed, stream_id, count))
    v = np.rint(np.exp(np.log(float(lo)) + u * np.log(float(hi) / float(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


def matrix(kind: str, rows: int, cols: int, seed: int, stream_id: int,
           ld: int | None = None, row_indices: np.ndarray | None = None,
           pad_value: float = np.nan) -> np.ndarray:
    """A ``rows x cols`` row-major matrix of ``kind`` ("uniform", "int8", "hard").

    Element (i, j) is draw ``i * cols + j`` of the stream, independent of ``ld``.
    With ``ld > cols`` the result has shape (rows, ld) and the padding columns
    hold ``pad_value`` (NaN by default, so a kernel that reads padding is caught).
    With ``row_indices`` only those rows are produced (shape (len, ld)).
    """
    if kind not in _KINDS:
        raise ValueError(f"unknown kind {kind!r}")
    ld = cols if ld is None else ld
    if ld < cols:
        raise ValueError("ld < cols")
    fn = _KINDS[kind]
    if row_indices is None:
        vals = fn(raw_stream(seed, stream_id, rows * cols)).reshape(rows, cols)
    else:
        ri = np.asarray(row_indices, dtype=np.int64)
        counters = (ri[:, None] * cols + np.arange(cols, dtype=np.int64)[None, :]).astype(np.uint64)
        counters += np.uint64(int(stream_id) << _STREAM_SHIFT)
        vals = fn(splitmix64(seed, counters))
    if ld == cols:
        return np.ascontiguousarray(vals)
    out = np.full((vals.shape[0], ld), pad_value, dtype=np.float64)
    out[:, :cols] = vals
    return out


def grouped_problems(seed: int, count: int = 2048, lo: int = 16, hi: int = 512):
    """(m, n, k) int64 arrays of ``count`` problems, each log-uniform in [lo, hi]."""
    m = log_uniform_ints(seed, 10, count, lo, hi)
    n = log_uniform_ints(seed, 11, count, lo, hi)
    k = log_uniform_ints(seed, 12, count, lo, hi)
    return m, n, k


def poisson_gaps_ms(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Exponential inter-arrival gaps (ms) of a Poisson process of ``rate_per_s``."""
    u = _unit(raw_stream(seed, 20, count))
    return -np.log1p(-u) / rate_per_s * 1e3
