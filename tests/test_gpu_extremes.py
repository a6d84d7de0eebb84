"""GPU parity at the edges of the FP64 exponent range.

Rows of A and columns of B are scaled by powers of two from 2^-1074 (subnormal
entries) to 2^+1000, so the products of the split-precision path land in every
regime of the final rounding: deep underflow to a signed zero, subnormal
results, normal results and overflow to +-Inf.  The emulated path (single GEMM
and grouped) must equal the CPU model of steps e1..e4 bit for bit, the model
rounding the exact T 2^E once.  The native kernels are checked where IEEE
arithmetic fixes one answer whatever the summation order or FMA contraction:
integer-valued inputs scaled into the subnormal range (every product and sum
exact), sign-definite overflow (+-Inf), and, for rounded subnormal products,
the FP64 bound widened by the absolute underflow error of k + 2 roundings.
"""
import numpy as np
import pytest

from oracle import cgemm, exact, ozaki
from synth import generators as g

from gpu_util import to_dev

pytestmark = pytest.mark.gpu

ROW_SCALES = [0, -540, -1000, -1060, -1074, 500, 600, -300, 1000, -20]
COL_SCALES = [0, -536, -20, 510, -1000, 24, 1000, -1074]


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def scaled_inputs(m, n, k, seed, kind="uniform"):
    """A with row i scaled by 2^ROW_SCALES[i % 10], B with column j scaled by
    2^COL_SCALES[j % 8] (np.ldexp rounds the subnormal ones; the rounded values
    are the inputs)."""
    A = g.matrix(kind, m, k, seed, g.STREAM_A)
    B = g.matrix(kind, k, n, seed, g.STREAM_B)
    ra = np.array([ROW_SCALES[i % len(ROW_SCALES)] for i in range(m)])
    cb = np.array([COL_SCALES[j % len(COL_SCALES)] for j in range(n)])
    return np.ldexp(A, ra[:, None]), np.ldexp(B, cb[None, :])


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def emulate(gb, A, B, C0, alpha, beta, s):
    import torch
    dC = to_dev(C0)
    gb.dgemm(to_dev(A), to_dev(B), dC, alpha, beta, precision="emulated", slices=s)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("s,alpha,beta", [(10, 1.0, 0.0), (11, 1.5, 0.5), (13, -0.75, 2.0),
                                          (16, 1.0, 0.0), (3, 1.0, 0.0)])
def test_emulated_bit_exact_across_the_exponent_range(gb, s, alpha, beta):
    m, n, k = 150, 70, 96
    A, B = scaled_inputs(m, n, k, 71)
    C0 = g.matrix("uniform", m, n, 71, g.STREAM_C)
    got = emulate(gb, A, B, C0, alpha, beta, s)
    want = ozaki.emulated_gemm(alpha, A, B, beta, C0, s=s)
    assert np.array_equal(bits(got), bits(want))
    if alpha == 1.0 and beta == 0.0:
        # every regime is present: infinities, zeros, subnormal and normal results
        fin = np.abs(want[np.isfinite(want)])
        assert np.isinf(want).any() and (want == 0).any()
        assert ((fin > 0) & (fin < 2.0 ** -1022)).any() and (fin >= 2.0 ** -1022).any()


def test_emulated_integer_inputs_exact_in_the_subnormal_range(gb):
    # single-digit integers scaled by 2^-540 and 2^-541: C* 2^-1081 rounded once
    m, n, k = 130, 40, 64
    seed = g.BASE_SEED + 100
    A = np.ldexp(g.matrix("int8", m, k, seed, 0), -540)
    B = np.ldexp(g.matrix("int8", k, n, seed, 1), -541)
    got = emulate(gb, A, B, np.zeros((m, n)), 1.0, 0.0, 2)
    Ci = cgemm.dgemm(1.0, np.ldexp(A, 540), np.ldexp(B, 541))   # exact integers
    want = np.array([[float(int(v)) for v in row] for row in Ci])
    from fractions import Fraction
    exp = np.array([[float(Fraction(int(v)) / 2 ** 1081) for v in row] for row in want])
    assert np.array_equal(bits(got), bits(exp))


def test_grouped_emulated_bit_exact_across_the_exponent_range(gb):
    import torch
    probs, host = [], []
    shapes = [(150, 70, 96), (33, 200, 17), (128, 48, 300), (7, 9, 5), (260, 31, 64)]
    for i, (m, n, k) in enumerate(shapes):
        A, B = scaled_inputs(m, n, k, 81 + i)
        C0 = g.matrix("uniform", m, n, 81 + i, g.STREAM_C)
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=1.5, beta=0.5,
                          precision="emulated", slices=11))
        host.append((A, B, C0))
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    for p, (A, B, C0) in zip(probs, host):
        want = ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=11)
        assert np.array_equal(bits(p["C"].cpu().numpy()), bits(want))
    plan.close()


@pytest.mark.parametrize("kernel", ["auto", "naive", "tiled", "dfma", "dmma"])
def test_native_exact_subnormal_results(gb, kernel):
    # integers in [-8, 8] times 2^-530: every product is an integer times 2^-1060,
    # a multiple of the smallest subnormal, and every sum too, so each kernel's
    # result is exact (C* 2^-1060 with alpha = 1.5, beta = 0.5) whatever its order
    import torch
    m, n, k = 97, 75, 256
    seed = g.BASE_SEED + 100
    Ai = g.matrix("int8", m, k, seed, 0)
    Bi = g.matrix("int8", k, n, seed, 1)
    Ci = g.matrix("int8", m, n, seed, 2)
    A, B, C0 = np.ldexp(Ai, -530), np.ldexp(Bi, -530), np.ldexp(Ci, -1060)
    dC = to_dev(C0)
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.5, 0.5, kernel=kernel)
    torch.cuda.synchronize()
    want = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    exact_int = 1.5 * cgemm.dgemm(1.0, Ai, Bi) + 0.5 * Ci          # integers, exact
    assert np.array_equal(want, np.ldexp(exact_int, -1060))
    assert np.array_equal(bits(dC.cpu().numpy()), bits(want))


@pytest.mark.parametrize("kernel", ["auto", "naive", "tiled", "dfma", "dmma"])
def test_native_overflow_to_signed_infinity(gb, kernel):
    # sign-definite rows of A at 2^600 against positive columns of B at 2^500:
    # every such entry is beyond the double range (+Inf or -Inf by the row's sign)
    # in any summation order; the other entries are finite and within the bound
    import torch
    m, n, k = 70, 50, 64
    A = np.abs(g.matrix("uniform", m, k, 91, 0)) + 0.25
    B = np.abs(g.matrix("uniform", k, n, 91, 1)) + 0.25
    A[1::2] *= -1.0
    big_r = np.arange(m) % 3 == 0
    big_c = np.arange(n) % 4 == 0
    A[big_r] = np.ldexp(A[big_r], 600)
    B[:, big_c] = np.ldexp(B[:, big_c], 500)
    dC = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.0, 0.0, kernel=kernel)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    want = cgemm.dgemm(1.0, A, B)
    over = big_r[:, None] & big_c[None, :]
    assert np.all(np.isinf(want[over])) and np.array_equal(got[over], want[over])
    fin = ~over
    assert np.all(np.isfinite(got[fin]))
    absab = cgemm.dgemm(1.0, np.abs(A), np.abs(B))
    bound = exact.error_bound(k, 1.0, absab)
    assert np.all(np.abs(got[fin] - want[fin]) <= 2 * bound[fin])


@pytest.mark.parametrize("kernel", ["auto", "naive", "tiled", "dfma", "dmma"])
def test_native_rounded_subnormal_products_within_widened_bound(gb, kernel):
    # uniform rows at 2^-530 against columns at 2^-532: products near 2^-1064 are
    # rounded to the subnormal grid (absolute error up to 2^-1075 each), so the
    # relative FP64 bound is widened by (k + 2) 2^-1074 for the kernel and the
    # oracle alike
    import torch
    m, n, k = 80, 60, 128
    A = np.ldexp(g.matrix("uniform", m, k, 95, 0), -530)
    B = np.ldexp(g.matrix("uniform", k, n, 95, 1), -532)
    dC = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.0, 0.0, kernel=kernel)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    want = cgemm.dgemm(1.0, A, B)
    tol = 2 * (exact.error_bound(k, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)))
               + (k + 2) * 2.0 ** -1074)
    assert np.all(np.abs(got - want) <= tol)
    assert np.any((np.abs(got) > 0) & (np.abs(got) < 2.0 ** -1022))
