"""Pins of the model's recombination (step e4) over the whole exponent range.

The model rounds the exact value T * 2^E once (round to nearest, ties to even,
gradual underflow, overflow to +-inf).  These tests do not re-run that rule:
they check, with exact rationals, that each result is the double nearest to the
exact value (a property any correct rounding has and any truncation, double
rounding, dropped level or wrong weight violates), plus hand-derived values at
the edges of the double range, and the power-of-two scaling identities of the
whole split-precision GEMM on integer inputs whose exact product is known.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, ozaki
from synth import generators as g

DBL_MAX = Fraction(2 ** 1024 - 2 ** 971)
OVERFLOW_AT = Fraction(2 ** 1024 - 2 ** 970)  # midpoint of DBL_MAX and 2^1024


def _odd(r: float) -> bool:
    return struct.unpack("<q", struct.pack("<d", r))[0] & 1 == 1


def is_nearest_double(r: float, x: Fraction) -> bool:
    """r is the double nearest to x (ties to the even significand), +-inf when |x|
    reaches the overflow threshold, and a zero carries x's sign."""
    if math.isnan(r):
        return False
    if math.isinf(r):
        return (r > 0) == (x > 0) and abs(x) >= OVERFLOW_AT
    if abs(x) >= OVERFLOW_AT:
        return False
    if r == 0:
        if x == 0:
            return True
        if math.copysign(1.0, r) != (1.0 if x > 0 else -1.0):
            return False
    d = abs(x - Fraction(r))
    for nb in (math.nextafter(r, math.inf), math.nextafter(r, -math.inf)):
        fn = Fraction(2 ** 1024) * (1 if nb > 0 else -1) if math.isinf(nb) else Fraction(nb)
        dn = abs(x - fn)
        if dn < d:
            return False
        if dn == d and _odd(r):
            return False
    return True


def test_nearest_double_checker_rejects_wrong_roundings():
    # the checker itself: truncation, a one-ulp slip, a lost tie rule, a wrong sign
    x = Fraction(1) + Fraction(3, 2 ** 53)             # 1 + 1.5 ulp: nearest is 1 + 2 ulp
    assert is_nearest_double(1.0 + 2 * 2.0 ** -52, x)
    assert not is_nearest_double(1.0 + 2.0 ** -52, x)  # truncated
    t = Fraction(1) + Fraction(1, 2 ** 53)             # tie between 1 and 1 + ulp
    assert is_nearest_double(1.0, t) and not is_nearest_double(1.0 + 2.0 ** -52, t)
    assert not is_nearest_double(-1.0, Fraction(1))
    assert not is_nearest_double(0.0, Fraction(-1, 2 ** 1080))
    assert is_nearest_double(-0.0, Fraction(-1, 2 ** 1080))


@pytest.mark.parametrize("T,E,want", [
    (1, -1074, 5e-324),                      # the smallest subnormal
    (1, -1075, 0.0),                         # exactly half of it: tie to the even 0
    (3, -1075, 1e-323),                      # 1.5 units: tie to the even 2 units
    (5, -1076, 5e-324),                      # 1.25 units
    (-1, -2000, -0.0),                       # far below: a signed zero
    (2 ** 60 + 1, -1135, 5e-324),            # just above half a unit: up (rounding T
                                             # to 53 bits first would give the tie, 0)
    (2 ** 52, -1074, 2.0 ** -1022),          # 2^52 units: the smallest normal
    (2 ** 53 - 1, -1074, (2 ** 53 - 1) * 2.0 ** -1074),   # subnormal grid, exact
    (2 ** 53 - 1, 971, 1.7976931348623157e308),          # the largest double, exact
    (2 ** 54 - 1, 970, math.inf),            # rounds up to 2^1024: overflow
    (-(2 ** 127 - 1), 1000, -math.inf),
    ((2 ** 64 + 1) * 2 ** 60 + 3, -1200, float(Fraction((2 ** 64 + 1) * 2 ** 60 + 3, 2 ** 1200))),
])
def test_round_scaled_hand_values(T, E, want):
    got = ozaki.round_scaled(T, E)
    assert got == want and math.copysign(1.0, got) == math.copysign(1.0, want)
    assert is_nearest_double(got, Fraction(T) * Fraction(2) ** E)


def test_round_scaled_is_nearest_over_the_exponent_range():
    rng = np.random.default_rng(1602)
    for _ in range(3000):
        bits = int(rng.integers(1, 128))
        T = int(rng.integers(0, 2 ** 62)) << max(0, bits - 62) | int(rng.integers(0, 2 ** 20))
        T = T % (2 ** bits) or 1
        if rng.random() < 0.5:
            T = -T
        # exponents placing the result in every regime: deep underflow,
        # subnormal, normal, near and beyond overflow
        E = int(rng.choice([rng.integers(-1250, -1050), rng.integers(-1200, 1000),
                            rng.integers(850, 1030), rng.integers(-2400, -1150)]))
        if rng.random() < 0.2:
            # a value sitting exactly on a rounding boundary of the subnormal grid
            E = -1075 - max(0, T.bit_length() - 54)
        r = ozaki.round_scaled(T, E)
        assert is_nearest_double(r, Fraction(T) * Fraction(2) ** E), (T, E, r)


@pytest.mark.parametrize("s", [3, 10, 16])
def test_recombine_is_nearest_to_the_exact_level_sum(s):
    # random level sums (int64, far beyond what digits produce, so T spans many
    # bits) and exponents spread over every regime: each output must be the
    # double nearest to sum_g S_g 2^(5 (s+1-g)) * 2^(e_i + f_j - 8 - 5 (s-1)),
    # that sum formed here term by term in exact rationals
    rng = np.random.default_rng(s)
    m, n = 7, 9
    S = rng.integers(-2 ** 40, 2 ** 40, (s, m, n), dtype=np.int64)
    S[:, 0, 0] = 0                                   # T = 0
    S[:, 1, :] = 0
    S[0, 1, :] = 1                                   # T = 2^(5 (s-1)): powers of two
    e = rng.integers(-1100, 1030, m)
    f = rng.integers(-1100, 1030, n)
    e[2], f[3] = -1073, -1073                        # subnormal lines
    e[3], f[4] = 1024, 1024                          # lines at the top of the range
    e[4], f[5] = -540, -536                          # |T| ~ 2^(40 + 5 (s-1)): results
                                                     # near 2^-1044, subnormal
    out = ozaki.recombine(S, e, f, 1.0)
    for i in range(m):
        for j in range(n):
            T = sum(Fraction(int(S[g_ - 2, i, j])) * 2 ** (5 * (s + 1 - g_))
                    for g_ in range(2, s + 2))
            E = int(e[i]) + int(f[j]) - 8 - 5 * (s - 1)
            assert is_nearest_double(float(out[i, j]), T * Fraction(2) ** E), (i, j)
    # every regime was visited
    assert np.any(np.isinf(out)) and np.any(out == 0)
    tiny = np.abs(out[np.isfinite(out)])
    assert np.any((tiny > 0) & (tiny < 2.0 ** -1022))


@pytest.mark.parametrize("shift", [-1060, -1080, -1100, -1140, -2000, 0, 900, 1040, 1200])
def test_integer_inputs_exact_at_any_scale(shift):
    # integers in [-8, 8] are single digits, so the emulated product is the exact
    # integer C*; with A scaled by 2^a and B by 2^b (a + b = shift) the result
    # must be C* 2^shift rounded once: exact rationals give it independently
    m, n, k = 6, 5, 64
    seed = g.BASE_SEED + 100
    A = g.matrix("int8", m, k, seed, 0)
    B = g.matrix("int8", k, n, seed, 1)
    a = shift // 2
    b = shift - a
    As, Bs = np.ldexp(A, a), np.ldexp(B, b)
    # scaling the integers must itself be exact for the identity to hold
    assert np.array_equal(np.ldexp(As, -a), A) and np.array_equal(np.ldexp(Bs, -b), B)
    star = exact.fraction_gemm(1.0, A, B)
    got = ozaki.emulated_gemm(1.0, As, Bs, s=2)
    for i in range(m):
        for j in range(n):
            x = star[i][j] * Fraction(2) ** shift
            assert is_nearest_double(float(got[i, j]), x), (shift, i, j)


def test_power_of_two_scaling_commutes_in_the_normal_range():
    # digits depend on x / 2^e only, so scaling a row of A (column of B) by a power
    # of two shifts e_i (f_j) and leaves the digits: the result scales exactly
    A = g.matrix("hard", 8, 40, 61, 0)
    B = g.matrix("hard", 40, 6, 61, 1)
    base = ozaki.emulated_gemm(1.0, A, B, s=11)
    for a, b in ((500, -480), (-600, 590), (300, 300), (-500, -400)):
        got = ozaki.emulated_gemm(1.0, np.ldexp(A, a), np.ldexp(B, b), s=11)
        assert np.array_equal(got, np.ldexp(base, a + b))


def test_error_bound_hand_value():
    # 2 (k + 2) u (|alpha| (|A||B|) + |beta| |C0|) with k = 6, alpha = -2,
    # (|A||B|) = 1.5, beta = 0.25, C0 = -4:  2 * 8 * 2^-53 * (3 + 1) = 2^-47
    assert exact.error_bound(6, -2.0, np.array([[1.5]]), 0.25, np.array([[-4.0]]))[0, 0] == 2.0 ** -47
    # beta = 0: C0 is not read (a NaN there changes nothing): 2 * 8 * 2^-53 * 3
    assert exact.error_bound(6, -2.0, np.array([[1.5]]), 0.0, np.array([[np.nan]]))[0, 0] == 3 * 2.0 ** -49
