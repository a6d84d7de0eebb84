"""Pins of the CPU DGEMM oracle against what mathematics fixes (Section 4.2 DGEMM).

Each test is chosen so that a plausible slip in the oracle fails at least one:
a dropped term (all-ones gives k-1), a transposed operand or swapped index
(non-symmetric permutation), a wrong alpha/beta handling (exact integer
alpha=1.5, beta=0.5 case), reading padding (NaN-poisoned ld > cols), reading C
when beta == 0 (NaN in C), wrong summation (bound vs double-double / exact).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

rng = np.random.default_rng(1602)


def test_identity_gives_B_bit_exact():
    n = 37
    B = g.matrix("uniform", n, 29, seed=1, stream_id=1)
    C = cgemm.dgemm(1.0, np.eye(n), B)
    assert np.array_equal(C, B)


def test_permutation_gives_row_permuted_B():
    n = 41
    perm = rng.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0           # (P B)[i] = B[perm[i]]
    assert not np.array_equal(P, P.T)     # a transposed operand would fail
    B = g.matrix("uniform", n, 23, seed=2, stream_id=1)
    assert np.array_equal(cgemm.dgemm(1.0, P, B), B[perm])
    # and B = I gives P itself (column side of the index map)
    assert np.array_equal(cgemm.dgemm(1.0, P, np.eye(n)), P)


@pytest.mark.parametrize("k", [1, 2, 17, 256, 1000])
def test_all_ones_gives_k(k):
    C = cgemm.dgemm(1.0, np.ones((5, k)), np.ones((k, 7)))
    assert np.all(C == float(k))


def test_rank_one_integer_outer_product():
    m, n, k = 13, 11, 64
    u = rng.integers(-9, 10, m).astype(float)
    v = rng.integers(-9, 10, n).astype(float)
    x = rng.integers(-9, 10, k).astype(float)
    y = rng.integers(-9, 10, k).astype(float)
    A = np.outer(u, x)
    B = np.outer(y, v)
    xy = float(int(np.dot(x.astype(np.int64), y.astype(np.int64))))
    assert np.array_equal(cgemm.dgemm(1.0, A, B), np.outer(u, v) * xy)


def _to_float(fr):
    return np.array([[float(v) for v in row] for row in fr])


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 2), (8, 8, 8), (7, 3, 6)])
def test_bruteforce_exact_rationals_dyadic(m, n, k):
    # odd multiples of 2^-10 with varied exponents: products are exact dyadics,
    # sums are not always exact in FP64, so check the bound against exact C*.
    A = (2 * rng.integers(-500, 500, (m, k)) + 1) * 2.0 ** -10 * 2.0 ** rng.integers(-20, 20, (m, k))
    B = (2 * rng.integers(-500, 500, (k, n)) + 1) * 2.0 ** -10 * 2.0 ** rng.integers(-20, 20, (k, n))
    C0 = rng.standard_normal((m, n))
    alpha, beta = 1.5, -0.75
    star = exact.fraction_gemm(alpha, A, B, beta, C0)
    C = cgemm.dgemm(alpha, A, B, beta, C0.copy())
    absAB = cgemm.dgemm(1.0, np.abs(A), np.abs(B))
    bound = exact.error_bound(k, alpha, absAB, beta, C0)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(float(C[i, j])) - star[i][j])
            assert err <= Fraction(float(bound[i, j]))


def test_integer_config_bit_exact_alpha_beta():
    # C = 1.5 A B + 0.5 C with integer entries in [-8, 8], k = 256: every partial
    # sum is an integer below 2^14, 1.5*s and 0.5*c are exact, so the result is
    # unique and equals the rational C* exactly.
    m, n, k = 6, 5, 256
    seed = g.BASE_SEED + 100
    A = g.matrix("int8", m, k, seed, g.STREAM_A)
    B = g.matrix("int8", k, n, seed, g.STREAM_B)
    C0 = g.matrix("int8", m, n, seed, g.STREAM_C)
    star = _to_float(exact.fraction_gemm(1.5, A, B, 0.5, C0))
    assert np.array_equal(cgemm.dgemm(1.5, A, B, 0.5, C0.copy()), star)


def test_double_double_reference_matches_exact():
    m, n, k = 4, 3, 50
    A = g.matrix("hard", m, k, 5, 0)
    B = g.matrix("hard", k, n, 5, 1)
    hi, lo = cgemm.dgemm_dd_rows(A, B)
    star = exact.fraction_gemm(1.0, A, B)
    for i in range(m):
        for j in range(n):
            scale = sum(abs(Fraction(float(A[i, l])) * Fraction(float(B[l, j]))) for l in range(k))
            err = abs(Fraction(float(hi[i, j])) + Fraction(float(lo[i, j])) - star[i][j])
            assert err <= scale * Fraction(1, 2 ** 100)


@pytest.mark.parametrize("kind", ["uniform", "hard"])
def test_oracle_within_bound_against_double_double(kind):
    n = 96
    A = g.matrix(kind, n, n, 17, 0)
    B = g.matrix(kind, n, n, 17, 1)
    C0 = g.matrix(kind, n, n, 17, 2)
    C = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    hi, lo = cgemm.dgemm_dd_rows(A, B)
    res = exact.residual(C, 1.5, hi, lo, 0.5, C0)
    bound = exact.error_bound(n, 1.5, cgemm.dgemm(1.0, np.abs(A), np.abs(B)), 0.5, C0)
    assert np.all(np.abs(res) <= bound)
    # the bound is not vacuous: the oracle's error is a visible fraction of it
    assert np.max(np.abs(res) / bound) > 1e-4


def test_beta_zero_does_not_read_C_and_alpha_zero_does_not_read_AB():
    A = g.matrix("uniform", 4, 6, 3, 0)
    B = g.matrix("uniform", 6, 5, 3, 1)
    C = np.full((4, 5), np.nan)
    out = cgemm.dgemm(2.0, A, B, 0.0, C)
    assert np.isfinite(out).all()
    An = np.full((4, 6), np.nan)
    Bn = np.full((6, 5), np.nan)
    C0 = g.matrix("uniform", 4, 5, 3, 2)
    out = cgemm.dgemm(0.0, An, Bn, 0.5, C0.copy())
    assert np.array_equal(out, 0.5 * C0)
    out = cgemm.dgemm(0.0, An, Bn, 0.0, np.full((4, 5), np.nan))
    assert np.array_equal(out, np.zeros((4, 5)))


def test_k_zero_and_empty():
    C0 = g.matrix("uniform", 3, 4, 3, 2)
    out = cgemm.dgemm(1.0, np.zeros((3, 1)), np.zeros((1, 4)), 0.25, C0.copy(), k=0)
    assert np.array_equal(out, 0.25 * C0)
    out = cgemm.dgemm(1.0, np.zeros((1, 3)), np.zeros((3, 4)), 0.0, np.zeros((1, 4)), m=0)
    assert np.array_equal(out, np.zeros((1, 4)))


def test_leading_dimensions_with_poisoned_padding():
    m, n, k = 9, 7, 13
    A = g.matrix("uniform", m, k, 8, 0, ld=16)
    B = g.matrix("uniform", k, n, 8, 1, ld=10)
    C = np.full((m, 12), np.nan)
    C[:, :n] = 0.0
    cgemm.dgemm(1.0, A, B, 0.0, C, m=m, n=n, k=k)
    assert np.isfinite(C[:, :n]).all() and np.isnan(C[:, n:]).all()
    ref = cgemm.dgemm(1.0, np.ascontiguousarray(A[:, :k]), np.ascontiguousarray(B[:, :n]))
    assert np.array_equal(C[:, :n], ref)


def test_power_of_two_alpha_commutes_exactly():
    A = g.matrix("uniform", 20, 30, 4, 0)
    B = g.matrix("uniform", 30, 10, 4, 1)
    assert np.array_equal(cgemm.dgemm(0.25, A, B), 0.25 * cgemm.dgemm(1.0, A, B))


def test_row_and_column_permutation_equivariance():
    A = g.matrix("uniform", 20, 30, 4, 0)
    B = g.matrix("uniform", 30, 10, 4, 1)
    C = cgemm.dgemm(1.0, A, B)
    pr, pc = rng.permutation(20), rng.permutation(10)
    assert np.array_equal(cgemm.dgemm(1.0, A[pr], B), C[pr])
    assert np.array_equal(cgemm.dgemm(1.0, A, np.ascontiguousarray(B[:, pc])), C[:, pc])


def test_transpose_identity_within_bound():
    A = g.matrix("uniform", 24, 40, 6, 0)
    B = g.matrix("uniform", 40, 16, 6, 1)
    C = cgemm.dgemm(1.0, A, B)
    Ct = cgemm.dgemm(1.0, np.ascontiguousarray(B.T), np.ascontiguousarray(A.T))
    bound = exact.error_bound(40, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)))
    assert np.all(np.abs(C - Ct.T) <= 2 * bound)


def test_rows_and_openmp_forms_bit_identical():
    m, n, k = 33, 21, 45
    A = g.matrix("uniform", m, k, 12, 0)
    B = g.matrix("uniform", k, n, 12, 1)
    C0 = g.matrix("uniform", m, n, 12, 2)
    full = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    rows = np.array([32, 0, 17])
    part = cgemm.dgemm_rows(rows, 1.5, A, B, 0.5, np.ascontiguousarray(C0[rows]))
    assert np.array_equal(part, full[rows])
    omp, used = cgemm.dgemm_omp(1.5, A, B, 0.5, C0.copy(), threads=4)
    assert used >= 1
    assert np.array_equal(omp, full)


def test_daxpy_oracle_pins():
    # exact cases: integers, a power-of-two alpha, alpha = 0 leaves y
    x = np.arange(-50, 50, dtype=np.float64)
    y = np.arange(100, dtype=np.float64) * 3.0
    assert np.array_equal(cgemm.daxpy(2.0, x, y), 2.0 * x + y)
    assert np.array_equal(cgemm.daxpy(0.0, np.full(5, np.nan), np.ones(5)), np.ones(5))
    # one rounding: fma(a, x, y) equals the exact rational rounded once
    a = 1.0 / 3.0
    xs = g.uniform_pm1(g.raw_stream(3, 0, 200))
    ys = g.uniform_pm1(g.raw_stream(3, 1, 200))
    got = cgemm.daxpy(a, xs, ys)
    for i in range(200):
        exact_v = Fraction(a) * Fraction(float(xs[i])) + Fraction(float(ys[i]))
        assert got[i] == float(exact_v)  # float(Fraction) rounds to nearest even
