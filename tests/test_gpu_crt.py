"""GPU parity of the residue (Chinese-remainder) form of the emulated FP64 GEMM
against the CPU model (oracle/ozaki_crt.py), bit for bit: the scaled integers
and their residues are exact, the residue products and the reconstruction are
exact, and the single rounding is the same, so every output must match the
model's bits; plus the FP64 bound against the double-double reference, the
integer configuration, the exponent extremes, NaN/Inf and argument errors.
"""
import numpy as np
import pytest

from oracle import cgemm, ozaki_crt
from synth import generators as g

from gpu_util import inputs, to_dev, within_bound

pytestmark = pytest.mark.gpu

PREC = "emulated_crt"


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def run(gb, A, B, C0, alpha, beta, N, workspace=None):
    import torch
    dC = to_dev(C0) if C0 is not None else torch.zeros((A.shape[0], B.shape[1]),
                                                         dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, alpha, beta if C0 is not None else 0.0, precision=PREC,
             slices=N, workspace=workspace)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("N,k", [(13, 333), (14, 200), (7, 129), (3, 17), (1, 5)])
def test_bit_exact_against_model(gb, N, k):
    # 300 x 260: three tile rows and three tile columns of 128, ragged in both
    m, n = 300, 260
    A, B, C0 = inputs("uniform", m, n, k, 901 + N)
    want = ozaki_crt.crt_gemm(1.5, A, B, 0.5, C0, N=N)
    got = run(gb, A, B, C0, 1.5, 0.5, N)
    assert np.array_equal(bits(got), bits(want))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1000), (1, 513, 33), (257, 1, 300), (2, 3, 1),
                                   (129, 255, 513)])
def test_degenerate_and_single_line_shapes(gb, m, n, k):
    # one row and/or one column (a single partly filled tile), K of one element,
    # and K one past a whole unit of 256 (the padded K extent then holds a second,
    # almost empty unit of zero residues)
    A, B, C0 = inputs("uniform", m, n, k, 903 + m + n)
    want = ozaki_crt.crt_gemm(0.5, A, B, -1.0, C0, N=13)
    assert np.array_equal(bits(run(gb, A, B, C0, 0.5, -1.0, 13)), bits(want))


@pytest.mark.parametrize("k", [256, 257, 4000, 17000])
def test_long_k_exact_units(gb, k):
    # K in units of 256 (FP32 sums exact), the int32 totals reduced every 64 units
    # (k = 17000: 67 units), the hard set's 16 decades
    A, B, C0 = inputs("hard", 130, 70, k, 902)
    want = ozaki_crt.crt_gemm(-0.75, A, B, 2.0, C0, N=14)
    assert np.array_equal(bits(run(gb, A, B, C0, -0.75, 2.0, 14)), bits(want))


def test_largest_residue_products(gb):
    # every element equal: the scaled integers 2^b - ..., residues of the largest
    # magnitudes, K = 8192 (the FP32 unit sums reach ~256 * 254^2)
    k = 8192
    v = 0.999999999999
    A = np.full((130, k), v)
    A[1::2] = -v
    B = np.full((k, 150), -v)
    B[:, ::3] = v
    want = ozaki_crt.crt_gemm(1.0, A, B, N=13)
    assert np.array_equal(bits(run(gb, A, B, None, 1.0, 0.0, 13)), bits(want))


def test_integer_configuration_is_exact(gb):
    A, B, C0 = inputs("int8", 256, 256, 256, g.BASE_SEED + 100)
    want = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    assert np.array_equal(run(gb, A, B, C0, 1.5, 0.5, 13), want)


def test_config0_within_fp64_bound(gb):
    A, B, C0 = inputs("uniform", 256, 256, 256, g.BASE_SEED)
    got = run(gb, A, B, C0, 1.5, 0.5, 13)
    assert np.array_equal(bits(got), bits(ozaki_crt.crt_gemm(1.5, A, B, 0.5, C0, N=13)))
    assert within_bound(got, 1.5, A, B, 0.5, C0) <= 1.0


def test_hard_set_at_short_k_is_bit_exact_but_beyond_the_bound(gb):
    # the 16-decade hard set at n = 256: each line keeps b bits of its largest
    # element (b = 52 at 13 moduli, 57 at 14, the most the 128-bit reconstruction
    # allows), and with 16 decades in a line that is not enough for the FP64
    # bound at this short K; the result is still the model's, bit for bit, and
    # the error falls by 2^5 with the five extra bits
    A, B, C0 = inputs("hard", 256, 256, 256, g.BASE_SEED + 3)
    got13 = run(gb, A, B, C0, 1.5, 0.5, 13)
    got14 = run(gb, A, B, C0, 1.5, 0.5, 14)
    assert np.array_equal(bits(got13), bits(ozaki_crt.crt_gemm(1.5, A, B, 0.5, C0, N=13)))
    assert np.array_equal(bits(got14), bits(ozaki_crt.crt_gemm(1.5, A, B, 0.5, C0, N=14)))
    r13 = within_bound(got13, 1.5, A, B, 0.5, C0)
    r14 = within_bound(got14, 1.5, A, B, 0.5, C0)
    assert r13 > 1.0 and 8 * r14 < r13


ROW_SCALES = [0, -540, -1000, -1060, -1074, 500, 600, -300, 1000, -20]
COL_SCALES = [0, -536, -20, 510, -1000, 24, 1000, -1074]


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (1.5, 0.5)])
def test_bit_exact_across_the_exponent_range(gb, alpha, beta):
    # rows of A and columns of B scaled from 2^-1074 (subnormal entries) to
    # 2^1000: results in every regime of the single rounding
    m, n, k = 150, 70, 96
    A = g.matrix("uniform", m, k, 171, g.STREAM_A)
    B = g.matrix("uniform", k, n, 171, g.STREAM_B)
    A = np.ldexp(A, np.array([ROW_SCALES[i % 10] for i in range(m)])[:, None])
    B = np.ldexp(B, np.array([COL_SCALES[j % 8] for j in range(n)])[None, :])
    C0 = g.matrix("uniform", m, n, 171, g.STREAM_C)
    got = run(gb, A, B, C0, alpha, beta, 13)
    want = ozaki_crt.crt_gemm(alpha, A, B, beta, C0, N=13)
    assert np.array_equal(bits(got), bits(want))
    if alpha == 1.0 and beta == 0.0:
        fin = np.abs(want[np.isfinite(want)])
        assert np.isinf(want).any() and (want == 0).any()
        assert ((fin > 0) & (fin < 2.0 ** -1022)).any() and (fin >= 2.0 ** -1022).any()


def test_nonfinite_rows_and_columns(gb):
    import torch
    k = 3000
    A, B, _ = inputs("uniform", 70, 50, k, 903, with_c=False)
    A[4, 7] = np.inf
    B[9, 13] = np.nan
    B[k - 3, 40] = -np.inf
    q = gb.Queue(gb.Device(0), torch.cuda.current_stream())
    dC = torch.zeros((70, 50), dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.0, 0.0, precision=PREC, slices=13, queue=q)
    with pytest.raises(gb.GbError, match="GB_ERR_NONFINITE"):
        q.wait()
    got = dC.cpu().numpy()
    want = ozaki_crt.crt_gemm(1.0, A, B, N=13)
    assert np.all(np.isnan(got[4, :])) and np.all(np.isnan(got[:, 13]))
    assert np.all(np.isnan(got[:, 40]))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert np.array_equal(got[fin], want[fin])


def test_writes_only_c_and_takes_wide_leading_dimensions(gb):
    import torch
    m, n, k = 200, 97, 150
    A, B, C0 = inputs("uniform", m, n, k, 904)
    canary = -12345.678
    big = np.full((m + 3, n + 7), canary)
    big[1:1 + m, 2:2 + n] = C0
    dbig = to_dev(big)
    Aw = np.full((m, k + 5), np.nan)
    Aw[:, :k] = A
    dA = to_dev(Aw)[:, :k]
    gb.dgemm(dA, to_dev(B), dbig[1:1 + m, 2:2 + n], 1.5, 0.5, precision=PREC, slices=13)
    torch.cuda.synchronize()
    out = dbig.cpu().numpy()
    mask = np.ones_like(out, dtype=bool)
    mask[1:1 + m, 2:2 + n] = False
    assert np.all(out[mask] == canary)
    want = ozaki_crt.crt_gemm(1.5, A, B, 0.5, C0, N=13)
    assert np.array_equal(bits(out[1:1 + m, 2:2 + n]), bits(want))


def test_argument_errors_and_other_entry_points(gb):
    import torch
    A, B, C0 = inputs("uniform", 16, 16, 16, 905)
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.dgemm(dA, dB, dC, precision=PREC, slices=15)
    with pytest.raises(gb.GbError, match="GB_ERR_WORKSPACE"):
        gb.dgemm(dA, dB, dC, precision=PREC, slices=13,
                 workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
    # one modulus holds the exact product only for very short K
    a = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    b = torch.zeros((64, 1), dtype=torch.float64, device="cuda")
    c = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
        gb.dgemm(a, b, c, precision=PREC, slices=1,
                 workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.host_workspace_size(PREC, 15, 16, 16, 16)
    with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
        gb.GroupedPlan([dict(A=dA, B=dB, C=dC, precision=PREC, slices=13)])


def test_two_calls_reuse_the_workspace(gb):
    import torch
    A, B, C0 = inputs("uniform", 129, 131, 300, 906)
    ws = gb.alloc_workspace(gb.workspace_size(PREC, 13, 129, 131, 300))
    first = run(gb, A, B, C0, 1.0, 1.0, 13, workspace=ws)
    A2, B2, _ = inputs("hard", 129, 131, 300, 907)
    second = run(gb, A2, B2, None, 1.0, 0.0, 13, workspace=ws)
    assert np.array_equal(bits(first), bits(ozaki_crt.crt_gemm(1.0, A, B, 1.0, C0, N=13)))
    assert np.array_equal(bits(second), bits(ozaki_crt.crt_gemm(1.0, A2, B2, N=13)))
    del ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,kind,N", [(4096, "uniform", 13), (8192, "uniform", 13),
                                      (8192, "hard", 14)])
def test_full_size_sampled_rows(gb, n, kind, N):
    # square sizes of the emulated workload: sampled rows x sampled columns against
    # the model (bit-exact) and whole sampled rows against the double-double
    # reference (FP64 bound)
    A, B, _ = inputs(kind, n, n, n, g.BASE_SEED + (2 if kind == "uniform" else 3), with_c=False)
    got = run(gb, A, B, None, 1.0, 0.0, N)
    rng = np.random.default_rng(n + N)
    rows = rng.choice(n, 4, replace=False)
    cols = np.sort(rng.choice(n, 96, replace=False))
    want = ozaki_crt.crt_gemm(1.0, A, B, N=N, rows=rows, cols=cols)
    assert np.array_equal(bits(got[np.ix_(rows, cols)]), bits(want))
    assert within_bound(got[rows], 1.0, A, B, 0.0, None, rows=rows) <= 1.0


@pytest.mark.parametrize("m,n,k,beta", [(300, 700, 333, 0.0), (1100, 1300, 500, 0.5),
                                        (129, 257, 17, 1.0), (2048, 3000, 256, 0.5)])
def test_host_buffers_bit_identical_to_device_call(gb, m, n, k, beta):
    # A, B, C in pinned host memory: bands of A, blocks of B and pieces of C
    # pipelined with the copies; every piece's result is the device call's (the
    # last case runs four bands, four blocks of B and a last band in two launches)
    import torch
    A, B, C0 = inputs("uniform", m, n, k, 908)
    want = run(gb, A, B, C0, 1.25, beta, 13)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.from_numpy(C0.copy()).pin_memory()
    gb.dgemm_host(hA, hB, hC, 1.25, beta, precision=PREC, slices=13)
    torch.cuda.synchronize()
    assert np.array_equal(bits(hC.numpy()), bits(want))


def test_host_buffers_full_size_sampled(gb):
    import torch
    n = 8192
    A, B, _ = inputs("uniform", n, n, n, g.BASE_SEED + 2, with_c=False)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((n, n), dtype=torch.float64).pin_memory()
    gb.dgemm_host(hA, hB, hC, 1.0, 0.0, precision=PREC, slices=13)
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    rows = rng.choice(n, 4, replace=False)
    cols = np.sort(rng.choice(n, 96, replace=False))
    want = ozaki_crt.crt_gemm(1.0, A, B, N=13, rows=rows, cols=cols)
    assert np.array_equal(bits(hC.numpy()[np.ix_(rows, cols)]), bits(want))


def test_steps_one_at_a_time_equal_the_single_call(gb):
    import torch
    m, n, k = 300, 520, 700
    A, B, C0 = inputs("uniform", m, n, k, 909)
    want = run(gb, A, B, C0, -1.5, 0.25, 13)
    ws = gb.alloc_workspace(gb.workspace_size(PREC, 13, m, n, k))
    dC = to_dev(C0)
    gb.emulated_crt_steps(to_dev(A), to_dev(B), dC, -1.5, 0.25, 13, ws)
    torch.cuda.synchronize()
    assert np.array_equal(bits(dC.cpu().numpy()), bits(want))
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.emulated_crt_steps(to_dev(A), to_dev(B), dC, 1.0, 0.0, 15, ws)
