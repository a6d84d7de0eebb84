"""Pins of the CPU model of the split-precision FP64 GEMM (steps e1..e4).

(a) exact reconstruction of every input from its digits and remainder, checked in
    exact rationals; digit bounds; (b) level sums equal a brute-force integer
    triple loop; (c) the truncation-error closed form; (d) integer inputs are
    reproduced exactly; (e) an adversarial input whose digits are known by hand.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cgemm, exact, ozaki
from synth import generators as g


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("s", [1, 3, 8, 11])
def test_exact_reconstruction_rows(kind, s):
    b1, b, dmax = ozaki.FORMATS["e4m3"]
    A = g.matrix(kind, 6, 9, 21, 0)
    e, bad = ozaki.exponents(A, axis=1)
    assert not bad.any()
    mx = np.abs(A).max(axis=1)
    assert np.all(mx < np.ldexp(1.0, e)) and np.all(mx >= np.ldexp(0.5, e))
    D, r = ozaki.slice_digits(A, e, s, axis=1)
    assert np.abs(D).max() <= dmax and np.abs(r).max() <= 0.5
    for i in range(6):
        for l in range(9):
            v = sum(Fraction(int(D[t, i, l])) / 2 ** (b1 + b * t) for t in range(s))
            v += Fraction(float(r[i, l])) / 2 ** (b1 + b * (s - 1))
            assert v * Fraction(2) ** int(e[i]) == Fraction(float(A[i, l]))


def test_exact_reconstruction_columns_and_zero_line():
    B = g.matrix("uniform", 7, 5, 22, 1)
    B[:, 2] = 0.0
    f, _ = ozaki.exponents(B, axis=0)
    assert f[2] == 0
    D, r = ozaki.slice_digits(B, f, 12, axis=0)
    assert np.all(D[:, :, 2] == 0)
    assert np.array_equal(ozaki.reconstruct(D, r, f, axis=0), B)


def test_level_sums_match_bruteforce_integers():
    s, m, n, k = 4, 3, 4, 5
    rng = np.random.default_rng(3)
    DA = rng.integers(-16, 17, (s, m, k))
    DBt = rng.integers(-16, 17, (s, n, k))
    S = ozaki.level_sums(DA, DBt, s)
    for g_ in range(2, s + 2):
        for i in range(m):
            for j in range(n):
                ref = 0
                for p in range(1, s + 1):
                    q = g_ - p
                    if 1 <= q <= s:
                        ref += sum(int(DA[p - 1, i, l]) * int(DBt[q - 1, j, l]) for l in range(k))
                assert S[g_ - 2, i, j] == ref


def _truncation_bound(s, k, e, f, alpha, absC_emu, beta, C0):
    """|alpha| k 2^(e_i+f_j) tau_s + recombination rounding, the closed form of
    the error left by s digits and the dropped pairs p + q > s + 1."""
    b1, b, dmax = ozaki.FORMATS["e4m3"]
    eps = 0.5 * 2.0 ** -(b1 + b * (s - 1))
    dropped = sum((2 * s + 1 - gg) * 2.0 ** -(b * (gg - 2)) for gg in range(s + 2, 2 * s + 1))
    tau = dmax * dmax * 2.0 ** -(2 * b1) * dropped + 2 * (1 + eps) * eps + eps * eps
    scale = np.ldexp(1.0, e[:, None] + f[None, :])
    rounding = (s + 4) * exact.U * (absC_emu + abs(beta) * np.abs(C0))
    return abs(alpha) * k * scale * tau + rounding


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("s", [2, 5, 9, 13])
def test_truncation_error_closed_form(kind, s):
    m, n, k = 12, 10, 64
    A = g.matrix(kind, m, k, 30, 0)
    B = g.matrix(kind, k, n, 30, 1)
    C0 = g.matrix(kind, m, n, 30, 2)
    out, d = ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s, details=True)
    hi, lo = cgemm.dgemm_dd_rows(A, B)
    res = exact.residual(out, 1.5, hi, lo, 0.5, C0)
    bound = _truncation_bound(s, k, d["e"], d["f"], 1.5, np.abs(out), 0.5, C0)
    assert np.all(np.abs(res) <= bound)


def test_integer_inputs_reproduced_exactly():
    # integers in [-8, 8]: row max <= 8 gives x = a/16 and d_1 = a exactly, so
    # one digit suffices and the result is the exact rational C*.
    m, n, k = 5, 6, 256
    seed = g.BASE_SEED + 100
    A = g.matrix("int8", m, k, seed, 0)
    B = g.matrix("int8", k, n, seed, 1)
    C0 = g.matrix("int8", m, n, seed, 2)
    star = np.array([[float(v) for v in row] for row in exact.fraction_gemm(1.5, A, B, 0.5, C0)])
    for s in (1, 2, 7):
        assert np.array_equal(ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s), star)


def test_adversarial_max_digit_input():
    # x = 1 - 2^-20: e = 0, digits (16, 0, 0, 0, -16) exactly (rint(-0.5) = -0 by
    # ties-to-even).  x^2 = 1 - 2^-19 + 2^-40 where the 2^-40 term is the pair
    # (5, 5) of level g = 10: with s = 5 it is dropped by the triangular
    # truncation (p + q > s + 1) and C = k (1 - 2^-19); with s >= 9 it is kept
    # and C = k x^2 exactly.  S_2 = 256 k, the largest level-2 sum at this k.
    k = 8192
    v = 1.0 - 2.0 ** -20
    A = np.full((2, k), v)
    B = np.full((k, 3), v)
    out, d = ozaki.emulated_gemm(1.0, A, B, s=5, details=True)
    assert d["DA"][:, 0, 0].tolist() == [16, 0, 0, 0, -16]
    assert np.all(d["S"][0] == 256 * k)
    assert np.all(out == k * (1.0 - 2.0 ** -19))
    out9 = ozaki.emulated_gemm(1.0, A, B, s=9)
    assert np.all(out9 == k * (1.0 - 2.0 ** -19 + 2.0 ** -40))


def test_nonfinite_rows_and_columns_give_nan():
    A = g.matrix("uniform", 4, 8, 40, 0)
    B = g.matrix("uniform", 8, 5, 40, 1)
    A[1, 3] = np.inf
    B[6, 2] = np.nan
    out = ozaki.emulated_gemm(1.0, A, B, s=6)
    assert np.isnan(out[1]).all() and np.isnan(out[:, 2]).all()
    mask = np.ones_like(out, dtype=bool)
    mask[1] = False
    mask[:, 2] = False
    assert np.isfinite(out[mask]).all()


def test_bound_met_with_enough_digits_uniform():
    # the FP64 accuracy contract is met by the emulation at the default digit
    # counts chosen for uniform inputs (k = 256 is the tightest case here).
    for k, s in ((256, 10), (1024, 9)):
        A = g.matrix("uniform", 16, k, 50, 0)
        B = g.matrix("uniform", k, 16, 50, 1)
        out = ozaki.emulated_gemm(1.0, A, B, s=s)
        hi, lo = cgemm.dgemm_dd_rows(A, B)
        res = exact.residual(out, 1.0, hi, lo)
        bound = exact.error_bound(k, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)))
        assert np.all(np.abs(res) <= bound)


def test_short_k_needs_one_more_digit():
    # The FP64 bound 2 (k+2) u (|A||B|) grows like k^2 while the error left by the
    # truncated digits of a random-sign dot product grows only like sqrt(k): short
    # dot products need more digits.  Problem 36 of the grouped recipe (47 x 38,
    # k = 19, uniform inputs) exceeds the bound at s = 10 and meets it at s = 11,
    # the slice count of the grouped benchmark.
    ms, ns, ks = g.grouped_problems(g.BASE_SEED + 3, 40)
    m, n, k = int(ms[36]), int(ns[36]), int(ks[36])
    assert (m, n, k) == (47, 38, 19)
    A = g.matrix("uniform", m, k, 7100 + 36, 0)
    B = g.matrix("uniform", k, n, 7100 + 36, 1)
    hi, lo = cgemm.dgemm_dd_rows(A, B)
    bound = exact.error_bound(k, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)))
    ratio = {s: np.max(np.abs(exact.residual(ozaki.emulated_gemm(1.0, A, B, s=s), 1.0, hi, lo))
                       / bound) for s in (10, 11)}
    assert ratio[10] > 1.0 and ratio[11] <= 0.1
