"""Pins of the CPU model's BF16 digit format (8-bit signed digits, b1 = 7, b = 8).

The split-precision GEMM is the same four steps with wider digits: every digit d
has |d| <= 128, an integer that BF16 (8 significant bits) holds exactly, so a
digit product is an integer of at most 2^14.  Pinned here against exact
rationals, brute-force integer loops, digits worked out by hand and the FP64
bound; the E4M3 pins of the same steps are in test_ozaki_model.py.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cgemm, exact, ozaki
from synth import generators as g

from gpu_util import inputs, within_bound

B1, B, DMAX = ozaki.FORMATS["bf16"]


def test_format_constants():
    # 7 + 8 (s - 1) bits of a line's scale per s digits: 7 digits cover 55 bits
    assert (B1, B, DMAX) == (7, 8, 128)


def _bf16_exact(d: np.ndarray) -> bool:
    """Every value of d survives a round trip through BF16 (the high half of FP32)."""
    f = d.astype(np.float32)
    return bool(np.all((f.view(np.uint32) & 0xFFFF) == 0))


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("s", [1, 3, 5, 7])
def test_exact_reconstruction_rows(kind, s):
    A = g.matrix(kind, 6, 9, 121, 0)
    e, bad = ozaki.exponents(A, axis=1)
    assert not bad.any()
    D, r = ozaki.slice_digits(A, e, s, "bf16", axis=1)
    assert D.dtype == np.int16
    assert np.abs(D).max() <= DMAX and np.abs(r).max() <= 0.5
    assert _bf16_exact(D)
    for i in range(6):
        for l in range(9):
            v = sum(Fraction(int(D[t, i, l])) / 2 ** (B1 + B * t) for t in range(s))
            v += Fraction(float(r[i, l])) / 2 ** (B1 + B * (s - 1))
            assert v * Fraction(2) ** int(e[i]) == Fraction(float(A[i, l]))


def test_exact_reconstruction_columns_and_zero_line():
    Bm = g.matrix("hard", 7, 5, 122, 1)
    Bm[:, 3] = 0.0
    f, _ = ozaki.exponents(Bm, axis=0)
    assert f[3] == 0
    D, r = ozaki.slice_digits(Bm, f, 7, "bf16", axis=0)
    assert np.all(D[:, :, 3] == 0)
    assert np.array_equal(ozaki.reconstruct(D, r, f, "bf16", axis=0), Bm)


def test_digits_reach_plus_and_minus_128():
    # x = 127.5 / 128 rounds to the first digit 128 (tie, 128 even) and leaves
    # r = -1/2, which the second digit takes to -128: both ends of the range.
    x = np.array([[127.5 / 128, -127.5 / 128]])
    e, _ = ozaki.exponents(x, axis=1)
    assert e.tolist() == [0]
    D, r = ozaki.slice_digits(x, e, 3, "bf16", axis=1)
    assert D[:, 0, 0].tolist() == [128, -128, 0]
    assert D[:, 0, 1].tolist() == [-128, 128, 0]
    assert r[0, 0] == 0.0


def test_level_sums_match_bruteforce_integers():
    s, m, n, k = 4, 3, 4, 5
    rng = np.random.default_rng(13)
    DA = rng.integers(-128, 129, (s, m, k))
    DBt = rng.integers(-128, 129, (s, n, k))
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


def test_hand_digits_and_truncation():
    # x = 1 - 2^-20: e = 0, x 2^7 = 128 - 2^-13 -> d_1 = 128, r = -2^-13;
    # 256 r = -2^-5 -> d_2 = -0, r = -2^-5; 256 r = -8 -> d_3 = -8, r = 0.
    # x^2 = 1 - 2^-19 + 2^-40: the 2^-40 term is the pair (3, 3) of level g = 6,
    # dropped by the triangular truncation at s = 3 and 4 (p + q > s + 1), kept
    # from s = 5 on.  S_2 = 2^14 k is the largest level-2 sum at this k.
    k = 4096
    v = 1.0 - 2.0 ** -20
    A = np.full((2, k), v)
    Bm = np.full((k, 3), v)
    out, d = ozaki.emulated_gemm(1.0, A, Bm, s=3, fmt="bf16", details=True)
    assert d["DA"][:, 0, 0].tolist() == [128, 0, -8]
    assert np.all(d["S"][0] == 2 ** 14 * k)
    assert np.all(d["S"][1] == 0)
    assert np.all(d["S"][2] == 2 * 128 * -8 * k)
    assert np.all(out == k * (1.0 - 2.0 ** -19))
    assert np.all(ozaki.emulated_gemm(1.0, A, Bm, s=4, fmt="bf16") == k * (1.0 - 2.0 ** -19))
    out5 = ozaki.emulated_gemm(1.0, A, Bm, s=5, fmt="bf16")
    assert np.all(out5 == k * (1.0 - 2.0 ** -19 + 2.0 ** -40))


def test_integer_inputs_reproduced_exactly():
    # integers in [-8, 8]: row max <= 8 gives e <= 4, x = a / 2^e and d_1 =
    # a 2^(7-e) exactly, so one digit suffices and the result is the exact C*
    m, n, k = 5, 6, 256
    seed = g.BASE_SEED + 101
    A = g.matrix("int8", m, k, seed, 0)
    Bm = g.matrix("int8", k, n, seed, 1)
    C0 = g.matrix("int8", m, n, seed, 2)
    star = np.array([[float(v) for v in row] for row in exact.fraction_gemm(1.5, A, Bm, 0.5, C0)])
    for s in (1, 2, 7):
        assert np.array_equal(ozaki.emulated_gemm(1.5, A, Bm, 0.5, C0, s=s, fmt="bf16"), star)


def _truncation_bound(s, k, e, f, alpha, absC_emu, beta, C0):
    """|alpha| k 2^(e_i+f_j) tau_s + recombination rounding: the error left by s
    BF16 digits (|remainder| <= 1/2 ulp of the last digit) and the dropped pairs
    p + q > s + 1, each pair product at most 128^2 2^-(14 + 8 (g - 2))."""
    eps = 0.5 * 2.0 ** -(B1 + B * (s - 1))
    dropped = sum((2 * s + 1 - gg) * 2.0 ** -(B * (gg - 2)) for gg in range(s + 2, 2 * s + 1))
    tau = DMAX * DMAX * 2.0 ** -(2 * B1) * dropped + 2 * (1 + eps) * eps + eps * eps
    scale = np.ldexp(1.0, e[:, None] + f[None, :])
    rounding = (s + 4) * exact.U * (absC_emu + abs(beta) * np.abs(C0))
    return abs(alpha) * k * scale * tau + rounding


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("s", [2, 4, 6, 7])
def test_truncation_error_closed_form(kind, s):
    m, n, k = 12, 10, 64
    A = g.matrix(kind, m, k, 130, 0)
    Bm = g.matrix(kind, k, n, 130, 1)
    C0 = g.matrix(kind, m, n, 130, 2)
    out, d = ozaki.emulated_gemm(1.5, A, Bm, 0.5, C0, s=s, fmt="bf16", details=True)
    hi, lo = cgemm.dgemm_dd_rows(A, Bm)
    res = exact.residual(out, 1.5, hi, lo, 0.5, C0)
    bound = _truncation_bound(s, k, d["e"], d["f"], 1.5, np.abs(out), 0.5, C0)
    assert np.all(np.abs(res) <= bound)


@pytest.mark.parametrize("s", [3, 7])
def test_recombine_weights_are_8_bits_per_level(s):
    # random level sums and exponents: each output is the double nearest to
    # sum_g S_g 2^(8 (s+1-g)) 2^(e_i + f_j - 14 - 8 (s-1)), formed here term by
    # term in exact rationals (a model that used E4M3's 5-bit weights fails)
    rng = np.random.default_rng(70 + s)
    m, n = 5, 6
    S = rng.integers(-2 ** 30, 2 ** 30, (s, m, n), dtype=np.int64)
    e = rng.integers(-400, 400, m)
    f = rng.integers(-400, 400, n)
    out = ozaki.recombine(S, e, f, 1.0, fmt="bf16")
    for i in range(m):
        for j in range(n):
            T = sum(Fraction(int(S[g_ - 2, i, j])) * 2 ** (8 * (s + 1 - g_))
                    for g_ in range(2, s + 2))
            want = float(T * Fraction(2) ** (int(e[i]) + int(f[j]) - 14 - 8 * (s - 1)))
            assert out[i, j] == want


def test_seven_digits_meet_the_fp64_bound():
    # 7 BF16 digits (55 bits of each line's scale) meet the FP64 accuracy contract
    # on the uniform and the 16-decade hard inputs, 6 do not on the hard set
    for kind, k in (("uniform", 256), ("uniform", 1024), ("hard", 1024)):
        A = g.matrix(kind, 16, k, 150, 0)
        Bm = g.matrix(kind, k, 16, 150, 1)
        hi, lo = cgemm.dgemm_dd_rows(A, Bm)
        bound = exact.error_bound(k, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(Bm)))
        res = exact.residual(ozaki.emulated_gemm(1.0, A, Bm, s=7, fmt="bf16"), 1.0, hi, lo)
        assert np.all(np.abs(res) <= bound), kind
    A = g.matrix("hard", 16, 1024, 150, 0)
    Bm = g.matrix("hard", 1024, 16, 150, 1)
    hi, lo = cgemm.dgemm_dd_rows(A, Bm)
    bound = exact.error_bound(1024, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(Bm)))
    res6 = exact.residual(ozaki.emulated_gemm(1.0, A, Bm, s=6, fmt="bf16"), 1.0, hi, lo)
    assert np.any(np.abs(res6) > bound)


def test_e4m3_digits_unchanged_by_the_format_parameter():
    # the default format is E4M3 with int8 digits, as the GPU parity tests expect
    A = g.matrix("uniform", 3, 40, 160, 0)
    e, _ = ozaki.exponents(A, axis=1)
    D, _ = ozaki.slice_digits(A, e, 10, axis=1)
    D2, _ = ozaki.slice_digits(A, e, 10, "e4m3", axis=1)
    assert D.dtype == np.int8 and np.array_equal(D, D2)
    assert np.abs(D).max() <= 16


def test_short_k_hard_set_needs_eight_digits():
    # the FP64 bound shrinks with k faster than the truncation error does: on the
    # 16-decade hard set at n = k = 256 (C = 1.5 A B + 0.5 C) 7 BF16 digits miss
    # it, 8 meet it (E4M3 digits: 12 miss, 13 meet)
    A, Bm, C0 = inputs("hard", 256, 256, 256, g.BASE_SEED + 3)
    r = {s: within_bound(ozaki.emulated_gemm(1.5, A, Bm, 0.5, C0, s=s, fmt="bf16"),
                         1.5, A, Bm, 0.5, C0) for s in (7, 8)}
    assert r[7] > 1.0 and r[8] <= 1.0
