"""Writes the stored expected values under tests/golden/ from the oracle alone.

The paper prints no worked GEMM example, so the fixtures here are the definition
of Section 4.2 (C <- alpha A B + beta C) evaluated by the oracle on seeded
synthetic inputs, each checked against a second exact evaluation before it is
written:

* dgemm_int_n256.txt: the n = 256 configuration's integer variant
  (alpha = 1.5, beta = 0.5, A, B, C0 with integer entries in [-8, 8]).  Every
  partial sum is an integer below 2^53 and alpha, beta scale exactly, so C is
  unique: the plain-C oracle's result must equal exact integer arithmetic
  (Python ints).  Stored: the SHA-256 of C's little-endian float64 bytes, the
  exact sum of all entries and 64 sampled entries.
* dgemm_dyadic_5x7x3.txt: a 5 x 7 x 3 product of odd multiples of 2^-10
  (alpha = -0.75, beta = 0.25), whose exact value C* is stored entry by entry
  as a reduced fraction (exact rational arithmetic, oracle.exact.fraction_gemm).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import os
import sys
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import cgemm, exact  # noqa: E402
from synth import generators as g  # noqa: E402

INT_N = 256
INT_ALPHA, INT_BETA = 1.5, 0.5
INT_SEED = g.BASE_SEED + 100   # the integer variant of the n = 256 configuration
DY_M, DY_N, DY_K = 5, 7, 3
DY_ALPHA, DY_BETA = -0.75, 0.25
DY_SEED = 1602084771


def int_inputs():
    A = g.matrix("int8", INT_N, INT_N, INT_SEED, g.STREAM_A)
    B = g.matrix("int8", INT_N, INT_N, INT_SEED, g.STREAM_B)
    C0 = g.matrix("int8", INT_N, INT_N, INT_SEED, g.STREAM_C)
    return A, B, C0


def int_case():
    """(C from the C oracle, the same C in exact integer arithmetic) for the fixture."""
    A, B, C0 = int_inputs()
    C = cgemm.dgemm(INT_ALPHA, A, B, INT_BETA, C0.copy())
    Ai = [[int(v) for v in row] for row in A.astype(np.int64)]
    Bt = [[int(v) for v in col] for col in B.astype(np.int64).T]
    Ci = C0.astype(np.int64)
    exact_C = np.empty_like(C)
    for i in range(INT_N):
        for j in range(INT_N):
            s = sum(a * b for a, b in zip(Ai[i], Bt[j]))
            exact_C[i, j] = float(Fraction(3, 2) * s + Fraction(1, 2) * int(Ci[i, j]))
    return C, exact_C


def int_samples():
    rng = np.random.default_rng(INT_SEED)
    return [(int(i), int(j)) for i, j in zip(rng.integers(0, INT_N, 64), rng.integers(0, INT_N, 64))]


def dyadic_inputs():
    def odd_dyadic(rows, cols, sid):
        x = g.raw_stream(DY_SEED, sid, rows * cols)
        odd = (x % np.uint64(1023)).astype(np.int64) * 2 - 1021  # odd integers in [-1021, 1023]
        return (odd.astype(np.float64) * 2.0 ** -10).reshape(rows, cols)
    return odd_dyadic(DY_M, DY_K, 0), odd_dyadic(DY_K, DY_N, 1), odd_dyadic(DY_M, DY_N, 2)


def dyadic_case():
    A, B, C0 = dyadic_inputs()
    return exact.fraction_gemm(DY_ALPHA, A, B, DY_BETA, C0)


def sha256_of(C: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(C, dtype="<f8").tobytes()).hexdigest()


def int_text(C: np.ndarray) -> str:
    lines = ["# C = 1.5 A B + 0.5 C0, n = 256, A, B, C0 integer entries in [-8, 8]",
             "# (Section 4.2's definition; the integer variant of the n = 256 configuration)",
             f"# inputs: synth.generators.matrix('int8', 256, 256, {INT_SEED}, stream 0 / 1 / 2)",
             "# written by tests/golden/make_golden.py from the oracle; exact and unique",
             f"sha256 {sha256_of(C)}",
             f"sum {sum(Fraction(float(v)) for v in C.ravel())}"]
    lines += [f"entry {i} {j} {float(C[i, j])!r}" for i, j in int_samples()]
    return "\n".join(lines) + "\n"


def dyadic_text(Cs) -> str:
    lines = ["# C* = -0.75 A B + 0.25 C0 exactly (Section 4.2's definition), m, n, k = 5, 7, 3,",
             f"# entries odd multiples of 2^-10 from synth.generators.raw_stream({DY_SEED}, 0 / 1 / 2)",
             "# written by tests/golden/make_golden.py (exact rational arithmetic)"]
    for i, row in enumerate(Cs):
        for j, v in enumerate(row):
            lines.append(f"exact {i} {j} {v.numerator}/{v.denominator}")
    return "\n".join(lines) + "\n"


def main():
    C, exact_C = int_case()
    assert np.array_equal(C, exact_C), "oracle and exact integer arithmetic disagree"
    with open(os.path.join(HERE, "dgemm_int_n256.txt"), "w") as f:
        f.write(int_text(C))
    with open(os.path.join(HERE, "dgemm_dyadic_5x7x3.txt"), "w") as f:
        f.write(dyadic_text(dyadic_case()))
    print("wrote dgemm_int_n256.txt and dgemm_dyadic_5x7x3.txt")


if __name__ == "__main__":
    main()
