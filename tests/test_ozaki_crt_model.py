"""Pins of the CPU model of the residue (Chinese-remainder) form of the
split-precision GEMM (oracle/ozaki_crt.py), each against something other than
the model itself: number theory checked by brute force, exact rationals,
direct exact integer products, closed forms and the FP64 bound.  A dropped
term, a wrong sign or index, a wrong modulus or weight fails one of them."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import cgemm, exact
from oracle import ozaki_crt as crt
from synth import generators as g


def is_prime(p):
    return p > 1 and all(p % d for d in range(2, int(p ** 0.5) + 1))


def test_moduli_are_odd_primes_whose_residues_are_exact_in_bf16():
    ms = crt.MODULI
    assert len(set(ms)) == len(ms)
    assert all(is_prime(m) and m % 2 == 1 and m <= 513 for m in ms)
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(ms) for b in ms[i + 1:])
    # |r| <= 256 and every integer of magnitude <= 256 is exact in BF16 (8-bit
    # significand): 256 = 2^8, 255 = 0b11111111
    assert max((m - 1) // 2 for m in ms) <= 256
    for r in range(-256, 257):
        f = np.float32(r)
        bits = f.view(np.uint32) & 0xFFFF
        assert bits == 0, r   # the low half of the FP32 pattern is empty: exact in BF16


@pytest.mark.parametrize("N", [1, 4, 13, 16])
@pytest.mark.parametrize("k", [1, 2, 17, 256, 8192, 10240])
def test_scale_bits_is_the_largest_safe_b(N, k):
    M = math.prod(crt.MODULI[:N])
    b = crt.scale_bits(N, k)
    if b == 0:
        assert 4 * k * 4 > M
        return
    assert 1 <= b <= 62
    assert 4 * k * 2 ** (2 * b) <= M
    assert b == 62 or 4 * k * 2 ** (2 * b + 2) > M


def test_scale_bits_hand_values():
    # 13 moduli: M ~ 2^115.9; k = 8192: 2^(13 + 2 + 2b) <= M  ->  b = 50
    assert crt.scale_bits(13, 8192) == 50
    assert crt.scale_bits(13, 4096) == 50   # 2^(12 + 2 + 102) = 2^116 > M: still 50
    assert crt.scale_bits(14, 8192) == 54


def rne(fr):
    """Round a Fraction to the nearest integer, ties to even."""
    fl = math.floor(fr)
    d = fr - fl
    if d > Fraction(1, 2) or (d == Fraction(1, 2) and fl % 2 == 1):
        return fl + 1
    return fl


def test_scaling_is_round_to_nearest_even_of_the_exact_scaled_value():
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (7, 33))
    # planted ties: dyadic values whose scaled form ends in exactly one half
    X[0, :8] = np.array([0.5, -0.5, 1.5, -1.5, 2.5, 3.5, -2.5, 0.25]) * 2.0 ** -7
    X[1, :4] = [2.0 ** -60, -3 * 2.0 ** -61, 2.0 ** -1070, -(2.0 ** -1074)]
    e, bad = crt.exponents(X, axis=1)
    for b in (3, 8, 50, 62):
        Xi = crt.scale_to_integers(X, e, b, axis=1, bad=bad)
        for i in range(X.shape[0]):
            for l in range(X.shape[1]):
                want = rne(Fraction(float(X[i, l])) * Fraction(2) ** (b - int(e[i])))
                assert int(Xi[i, l]) == want
                assert abs(int(Xi[i, l])) <= 2 ** b


def test_symmetric_residues_by_brute_force():
    rnd = random.Random(5)
    vals = [0, 1, -1, 2 ** 62, -(2 ** 62), 2 ** 61 + 12345, -(2 ** 50) - 7]
    vals += [rnd.randrange(-(2 ** 62), 2 ** 62) for _ in range(300)]
    for m in crt.MODULI[:5] + crt.MODULI[-2:]:
        r = crt.sym_mod(np.array(vals, dtype=object), m)
        for x, rv in zip(vals, r):
            rv = int(rv)
            assert (x - rv) % m == 0
            assert abs(rv) <= (m - 1) // 2
            # the sign convention: the residue of -x is minus that of x
        r_neg = crt.sym_mod(np.array([-v for v in vals], dtype=object), m)
        assert [int(a) for a in r_neg] == [-int(a) for a in r]


@pytest.mark.parametrize("N", [1, 3, 13, 16])
def test_reconstruction_recovers_every_integer_below_half_the_product(N):
    M = math.prod(crt.MODULI[:N])
    rnd = random.Random(N)
    xs = [0, 1, -1, (M - 1) // 2, -((M - 1) // 2)] + [rnd.randrange(-(M // 2) + 1, M // 2)
                                                     for _ in range(200)]
    c = np.stack([np.array([((x % m) if 2 * (x % m) <= m else (x % m) - m) for x in xs],
                           dtype=np.int64) for m in crt.MODULI[:N]])
    got = crt.crt(c, N)
    assert [int(v) for v in got] == xs


@pytest.mark.parametrize("N, m, n, k", [(13, 5, 7, 33), (4, 6, 3, 9), (16, 3, 4, 130)])
def test_reconstructed_product_equals_the_direct_integer_product(N, m, n, k):
    rng = np.random.default_rng(m * n * k)
    A = rng.uniform(-1, 1, (m, k)) * 2.0 ** rng.integers(-20, 20, (m, 1))
    B = rng.uniform(-1, 1, (k, n)) * 2.0 ** rng.integers(-20, 20, (1, n))
    _, d = crt.crt_gemm(1.0, A, B, N=N, details=True)
    direct = d["Ai"].astype(object) @ d["Bi"].astype(object)
    assert all(int(x) == int(y) for x, y in zip(d["Cp"].ravel(), direct.ravel()))
    M = math.prod(crt.MODULI[:N])
    assert all(4 * abs(int(x)) <= M for x in direct.ravel())


def test_result_is_the_single_rounding_of_the_exact_scaled_product():
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (4, 21))
    B = rng.uniform(-1, 1, (21, 5))
    out, d = crt.crt_gemm(1.0, A, B, N=13, details=True)
    b = d["b"]
    for i in range(4):
        for j in range(5):
            exact_int = sum(int(d["Ai"][i, l]) * int(d["Bi"][l, j]) for l in range(21))
            val = Fraction(exact_int) * Fraction(2) ** (int(d["e"][i]) + int(d["f"][j]) - 2 * b)
            assert out[i, j] == float(val)   # Fraction -> float rounds to nearest even


def test_scaling_error_closed_form():
    # |C - A B| <= 2^(e_i + f_j - 2b) (sum_l (|A'| + |B'|) / 2 + k / 4) + half an ulp
    rng = np.random.default_rng(9)
    m, n, k = 5, 6, 40
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    for N in (5, 7, 13):
        out, d = crt.crt_gemm(1.0, A, B, N=N, details=True)
        b = d["b"]
        for i in range(m):
            for j in range(n):
                true = sum(Fraction(float(A[i, l])) * Fraction(float(B[l, j])) for l in range(k))
                scale = Fraction(2) ** (int(d["e"][i]) + int(d["f"][j]) - 2 * b)
                bnd = scale * (Fraction(sum(abs(int(d["Ai"][i, l])) + abs(int(d["Bi"][l, j]))
                                            for l in range(k)), 2) + Fraction(k, 4))
                err = abs(Fraction(float(out[i, j])) - true)
                assert err <= bnd + abs(Fraction(float(out[i, j]))) * Fraction(1, 2 ** 53)


def test_integer_configuration_is_bit_exact():
    # the n = 256 integer configuration, C = 1.5 A B + 0.5 C: every entry of A'
    # is the integer times a power of two (b bits hold it), so C' and C are exact
    n = 256
    seed = g.BASE_SEED + 100
    A = g.matrix("int8", n, n, seed, g.STREAM_A)
    B = g.matrix("int8", n, n, seed, g.STREAM_B)
    C0 = g.matrix("int8", n, n, seed, g.STREAM_C)
    want = 1.5 * (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64) + 0.5 * C0
    got = crt.crt_gemm(1.5, A, B, 0.5, C0.copy(), N=13)
    assert np.array_equal(got, want)


def test_uniform_inputs_within_the_fp64_bound_at_13_moduli():
    n = 192
    seed = g.BASE_SEED + 2
    A = g.matrix("uniform", n, n, seed, g.STREAM_A)
    B = g.matrix("uniform", n, n, seed, g.STREAM_B)
    got = crt.crt_gemm(1.0, A, B, N=13)
    rows = np.arange(0, n, 7)
    hi, lo = cgemm.dgemm_dd_rows(A, B, rows)
    res = exact.residual(got[rows], 1.0, hi, lo)
    bound = exact.error_bound(n, 1.0, cgemm.dgemm_rows(rows, 1.0, np.abs(A), np.abs(B)))
    rho = float(np.max(np.abs(res) / bound))
    assert rho <= 1.0
    # and too few moduli is visibly worse (the pins see the scaling)
    got5 = crt.crt_gemm(1.0, A, B, N=5)
    res5 = exact.residual(got5[rows], 1.0, hi, lo)
    assert float(np.max(np.abs(res5) / bound)) > 100 * rho


def test_special_cases():
    A = np.ones((3, 4))
    B = np.ones((4, 2))
    C0 = np.full((3, 2), 2.0)
    assert np.array_equal(crt.crt_gemm(0.0, A, B, 0.5, C0), 0.5 * C0)
    assert np.array_equal(crt.crt_gemm(1.0, A[:, :0], B[:0], 0.5, C0), 0.5 * C0)
    assert crt.crt_gemm(1.0, A[:0], B).shape == (0, 2)
    A2 = A.copy()
    A2[1, 2] = np.nan
    out = crt.crt_gemm(1.0, A2, B)
    assert np.isnan(out[1]).all() and np.array_equal(out[[0, 2]], np.full((2, 2), 4.0))
    B2 = B.copy()
    B2[0, 1] = np.inf
    out = crt.crt_gemm(1.0, A, B2)
    assert np.isnan(out[:, 1]).all() and np.array_equal(out[:, 0], np.full(3, 4.0))
