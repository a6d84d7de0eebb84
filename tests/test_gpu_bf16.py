"""GPU parity of the BF16-digit emulated FP64 path against the CPU model.

The same four steps as the E4M3 path with 8-bit digits (b1 = 7, b = 8): the split
kernels' exponents and BF16 digit planes bit-exact against the model; the
kind::f16 products, whose level sums are read out of tensor memory every
1024 / s K indices and added exactly, and the recombination, bit-exact against
the model over many read-out units, both level sets, K streamed in both
directions and the edges of the exponent range; the FP64 bound at 7 digits
(uniform) and 8 (the hard set);
integer inputs exact; NaN/Inf; argument errors and the entry points that do not
take this precision.
"""
import numpy as np
import pytest

from oracle import cgemm, ozaki
from synth import generators as g

from gpu_util import inputs, to_dev, within_bound

pytestmark = pytest.mark.gpu

PREC = "emulated_bf16"


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def emulate(gb, A, B, C0, alpha, beta, s, workspace=None):
    import torch
    dC = to_dev(C0) if C0 is not None else torch.zeros((A.shape[0], B.shape[1]),
                                                         dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, alpha, beta if C0 is not None else 0.0, precision=PREC,
             slices=s, workspace=workspace)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def layout(s, m, n, k):
    """Offsets of the BF16 workspace as gb_gemm.h documents them."""
    up = lambda x: (x + 1023) // 1024 * 1024
    kp = max(16, -(-k // 16) * 16)
    mp, np_ = -(-m // 128) * 128, -(-n // 32) * 32
    a_dig = 0
    b_dig = up(2 * s * mp * kp)
    a_exp = up(b_dig + 2 * s * np_ * kp)
    b_exp = up(a_exp + 4 * m)
    return dict(kp=kp, a_digits=a_dig, b_digits=b_dig, a_exp=a_exp, b_exp=b_exp)


def untile16(raw, base, s, lines, kp, R):
    """BF16 digit values (s, lines_padded, kp) from the tiled layout: tiles of R
    lines x 32 bytes (16 digits), slices consecutive per K step, 16-byte chunk c
    of line r stored at chunk c ^ ((r // 4) & 1)."""
    lp = -(-lines // R) * R
    nks = kp // 16
    buf = raw[base:base + 2 * s * lp * kp].reshape(lp // R, nks, s, R, 2, 16)
    swz = (np.arange(R) // 4) & 1
    logical = np.empty_like(buf)
    logical[:, :, :, swz == 0] = buf[:, :, :, swz == 0]
    logical[:, :, :, swz == 1] = buf[:, :, :, swz == 1][:, :, :, :, ::-1]
    codes = np.ascontiguousarray(logical.transpose(2, 0, 3, 1, 4, 5)).reshape(s, lp, kp * 2)
    u16 = codes.view(np.uint16).astype(np.uint32) << 16
    return u16.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("m,n,k,s", [(37, 45, 70, 7), (128, 64, 256, 6), (5, 300, 33, 1),
                                     (200, 3, 129, 4), (130, 97, 64, 8), (3, 49, 40, 5)])
def test_split_digits_and_exponents_bit_exact(gb, kind, m, n, k, s):
    import torch
    A, B, _ = inputs(kind, m, n, k, 131, with_c=False)
    ws = gb.alloc_workspace(gb.workspace_size(PREC, s, m, n, k))
    ws.fill_(0xAB)  # poison: every digit byte the layout defines must be written
    emulate(gb, A, B, None, 1.0, 0.0, s, workspace=ws)
    raw = ws.cpu().numpy()
    lay = layout(s, m, n, k)
    kp = lay["kp"]
    da = untile16(raw, lay["a_digits"], s, m, kp, 128)
    db = untile16(raw, lay["b_digits"], s, n, kp, 32)
    ea = raw[lay["a_exp"]:lay["a_exp"] + 4 * m].view(np.int32)
    fb = raw[lay["b_exp"]:lay["b_exp"] + 4 * n].view(np.int32)
    e, _ = ozaki.exponents(A, axis=1)
    f, _ = ozaki.exponents(B, axis=0)
    assert np.array_equal(ea, e) and np.array_equal(fb, f)
    DA, _ = ozaki.slice_digits(A, e, s, "bf16", axis=1)
    DB, _ = ozaki.slice_digits(B, f, s, "bf16", axis=0)
    assert np.array_equal(da[:, :m, :k], DA.astype(np.float64))
    assert np.array_equal(db[:, :n, :k], DB.transpose(0, 2, 1).astype(np.float64))
    # padding lines and K indices hold zero digits
    assert not da[:, m:, :].any() and not da[:, :, k:].any()
    assert not db[:, n:, :].any() and not db[:, :, k:].any()


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6, 7, 8])
def test_products_bit_exact_against_model(gb, s):
    # k = 129: 9 K steps, two read-out units at s = 7 and 8 (both level sets)
    m, n, k = 300, 200, 129
    A, B, C0 = inputs("uniform", m, n, k, 132)
    want = ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s, fmt="bf16")
    got = emulate(gb, A, B, C0, 1.5, 0.5, s)
    assert np.array_equal(bits(got), bits(want))


@pytest.mark.parametrize("s,k", [(7, 3000), (7, 8200), (8, 8200), (5, 4100), (3, 6000),
                                 (6, 1)])
def test_long_k_read_out_units(gb, s, k):
    # K spans many read-out units (21 and 57 at s = 7): the units' exact sums must
    # add up to the model's level sums, which are exact in FP64
    A, B, C0 = inputs("hard", 130, 40, k, 134)
    want = ozaki.emulated_gemm(-0.5, A, B, 2.0, C0, s=s, fmt="bf16")
    assert np.array_equal(bits(emulate(gb, A, B, C0, -0.5, 2.0, s)), bits(want))


def test_second_wave_streams_k_backwards(gb):
    # 10 x 20 = 200 output tiles: the CTAs' second tiles stream K from its end, so
    # their read-out units cut K elsewhere; sampled rows of every tile row
    m, n, k = 1280, 640, 1000
    A, B, C0 = inputs("uniform", m, n, k, 135)
    got = emulate(gb, A, B, C0, 1.0, 1.0, 7)
    rows = np.arange(5, m, 53)
    want = ozaki.emulated_gemm(1.0, A, B, 1.0, C0[rows], s=7, fmt="bf16", rows=rows)
    assert np.array_equal(bits(got[rows]), bits(want))


@pytest.mark.parametrize("kind,s", [("uniform", 7), ("hard", 8)])
def test_config0_within_fp64_bound(gb, kind, s):
    # C = 1.5 A B + 0.5 C at n = 256 meets the FP64 contract with 7 BF16 digits on
    # uniform inputs and 8 on the 16-decade hard set (short K needs the extra digit)
    A, B, C0 = inputs(kind, 256, 256, 256, g.BASE_SEED + (0 if kind == "uniform" else 3))
    got = emulate(gb, A, B, C0, 1.5, 0.5, s)
    assert np.array_equal(bits(got), bits(ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s,
                                                                fmt="bf16")))
    assert within_bound(got, 1.5, A, B, 0.5, C0) <= 1.0


@pytest.mark.parametrize("s", [1, 2, 7])
def test_integer_inputs_exact(gb, s):
    A, B, C0 = inputs("int8", 256, 256, 256, g.BASE_SEED + 100)
    want = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    assert np.array_equal(emulate(gb, A, B, C0, 1.5, 0.5, s), want)


def test_largest_digits(gb):
    # every element 127.5 / 128 or its negative: digits (+-128, -+128), pair
    # products of magnitude 2^14 in levels 2 .. 4, the first level 2^14 k at k = 8192
    k = 8192
    v = 127.5 / 128
    A = np.full((130, k), v)
    A[1::2] = -v
    B = np.full((k, 70), v)
    B[:, ::3] = -v
    want = ozaki.emulated_gemm(1.0, A, B, s=3, fmt="bf16")
    assert np.array_equal(bits(emulate(gb, A, B, None, 1.0, 0.0, 3)), bits(want))
    assert np.all(np.abs(want) == k * v * v)


ROW_SCALES = [0, -540, -1000, -1060, -1074, 500, 600, -300, 1000, -20]
COL_SCALES = [0, -536, -20, 510, -1000, 24, 1000, -1074]


@pytest.mark.parametrize("s,alpha,beta", [(7, 1.0, 0.0), (8, 1.0, 0.0), (6, 1.5, 0.5),
                                          (3, -0.75, 2.0)])
def test_bit_exact_across_the_exponent_range(gb, s, alpha, beta):
    # rows of A and columns of B scaled from 2^-1074 (subnormal entries) to
    # 2^1000: results in every regime of the single rounding (signed zeros,
    # subnormals, normals, +-Inf)
    m, n, k = 150, 70, 96
    A = g.matrix("uniform", m, k, 171, g.STREAM_A)
    B = g.matrix("uniform", k, n, 171, g.STREAM_B)
    A = np.ldexp(A, np.array([ROW_SCALES[i % 10] for i in range(m)])[:, None])
    B = np.ldexp(B, np.array([COL_SCALES[j % 8] for j in range(n)])[None, :])
    C0 = g.matrix("uniform", m, n, 171, g.STREAM_C)
    got = emulate(gb, A, B, C0, alpha, beta, s)
    want = ozaki.emulated_gemm(alpha, A, B, beta, C0, s=s, fmt="bf16")
    assert np.array_equal(bits(got), bits(want))
    if alpha == 1.0 and beta == 0.0:
        fin = np.abs(want[np.isfinite(want)])
        assert np.isinf(want).any() and (want == 0).any()
        assert ((fin > 0) & (fin < 2.0 ** -1022)).any() and (fin >= 2.0 ** -1022).any()


def test_nonfinite_rows_and_columns(gb):
    import torch
    k = 3000
    A, B, _ = inputs("uniform", 70, 50, k, 133, with_c=False)
    A[4, 7] = np.inf
    B[9, 13] = np.nan
    B[k - 3, 40] = -np.inf
    q = gb.Queue(gb.Device(0), torch.cuda.current_stream())
    dC = torch.zeros((70, 50), dtype=torch.float64, device="cuda")
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.0, 0.0, precision=PREC, slices=7, queue=q)
    with pytest.raises(gb.GbError, match="GB_ERR_NONFINITE"):
        q.wait()
    got = dC.cpu().numpy()
    want = ozaki.emulated_gemm(1.0, A, B, s=7, fmt="bf16")
    assert np.all(np.isnan(got[4, :])) and np.all(np.isnan(got[:, 13]))
    assert np.all(np.isnan(got[:, 40]))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert np.array_equal(got[fin], want[fin])


def test_writes_only_c(gb):
    import torch
    m, n, k = 200, 97, 150
    A, B, C0 = inputs("uniform", m, n, k, 136)
    canary = -12345.678
    big = np.full((m + 3, n + 7), canary)
    big[1:1 + m, 2:2 + n] = C0
    dbig = to_dev(big)
    gb.dgemm(to_dev(A), to_dev(B), dbig[1:1 + m, 2:2 + n], 1.5, 0.5, precision=PREC, slices=7)
    torch.cuda.synchronize()
    out = dbig.cpu().numpy()
    mask = np.ones_like(out, dtype=bool)
    mask[1:1 + m, 2:2 + n] = False
    assert np.all(out[mask] == canary)
    want = ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=7, fmt="bf16")
    assert np.array_equal(bits(out[1:1 + m, 2:2 + n]), bits(want))


def test_argument_errors_and_other_entry_points(gb):
    import torch
    A, B, C0 = inputs("uniform", 16, 16, 16, 137)
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.dgemm(dA, dB, dC, precision=PREC, slices=9)
    with pytest.raises(gb.GbError, match="GB_ERR_WORKSPACE"):
        gb.dgemm(dA, dB, dC, precision=PREC, slices=7,
                 workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_WORKDIV"):
        wd, _ = gb.workdiv_suggest("dfma", 16, 16, 16)
        gb.dgemm(dA, dB, dC, precision=PREC, slices=7, workdiv=wd)
    with pytest.raises(ValueError):
        gb.dgemm(dA, dB, dC, precision="bf16")
    # k beyond 2^22: refused on the host before any workspace is needed
    k = (1 << 22) + 16
    a = torch.zeros((1, k), dtype=torch.float64, device="cuda")
    b = torch.zeros((k, 1), dtype=torch.float64, device="cuda")
    c = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
        gb.dgemm(a, b, c, precision=PREC, slices=7, workspace=torch.empty(
            256, dtype=torch.uint8, device="cuda"))
    # the host-buffer, grouped and serving calls take native or E4M3 digits
    with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
        gb.host_workspace_size(PREC, 7, 16, 16, 16)
    with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
        gb.GroupedPlan([dict(A=dA, B=dB, C=dC, precision=PREC, slices=7)])
    srv = gb.Server(1 << 30)
    try:
        with pytest.raises(gb.GbError, match="GB_ERR_UNSUPPORTED"):
            srv.submit(16, 16, 16, precision=PREC, slices=7)
    finally:
        srv.close()


@pytest.mark.parametrize("n,kind,s", [(4096, "uniform", 7), (8192, "uniform", 7),
                                      (8192, "hard", 7), (8192, "hard", 8)])
def test_full_size_sampled_rows(gb, n, kind, s):
    # square sizes of the emulated workload: 8 sampled rows against the model
    # (bit-exact) and the double-double reference (FP64 bound)
    A, B, _ = inputs(kind, n, n, n, g.BASE_SEED + (2 if kind == "uniform" else 3), with_c=False)
    got = emulate(gb, A, B, None, 1.0, 0.0, s)
    rows = np.random.default_rng(n + s).choice(n, 8, replace=False)
    want = ozaki.emulated_gemm(1.0, A, B, s=s, fmt="bf16", rows=rows)
    assert np.array_equal(bits(got[rows]), bits(want))
    assert within_bound(got[rows], 1.0, A, B, 0.0, None, rows=rows) <= 1.0
