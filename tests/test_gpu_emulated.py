"""GPU parity of the split-precision (emulated FP64) path against the CPU model of
steps e1..e4 and the FP64 oracle.

Step by step: exponents and E4M3 digit bytes of the split kernels bit-exact
against the model; the tensor-core products + recombination bit-exact against
the model (every level sum below 2^24 is exact in FP32 tensor memory); the full
result within the FP64 bound against the double-double reference; integer
inputs exact; an adversarial input with the largest level-2 sums; NaN/Inf
handling and its queue status.
"""
import numpy as np
import pytest

from oracle import cgemm, ozaki
from synth import generators as g

from gpu_util import e4m3_decode, inputs, to_dev, within_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def emulate(gb, A, B, C0, alpha, beta, s):
    import torch
    dA, dB = to_dev(A), to_dev(B)
    dC = to_dev(C0) if C0 is not None else torch.zeros((A.shape[0], B.shape[1]),
                                                         dtype=torch.float64, device="cuda")
    gb.dgemm(dA, dB, dC, alpha, beta if C0 is not None else 0.0, precision="emulated", slices=s)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def untile(raw, base, s, lines, kp, R):
    """Digit planes (s, lines_padded, kp) from the tiled workspace layout: tiles of R
    lines x 32 bytes, slices consecutive per K block, 16-byte chunk c of row r
    stored at chunk c ^ ((r // 4) & 1)."""
    lp = -(-lines // R) * R
    nkb = kp // 32
    buf = raw[base:base + s * lp * kp].reshape(lp // R, nkb, s, R, 2, 16)
    swz = (np.arange(R) // 4) & 1
    logical = np.empty_like(buf)
    logical[:, :, :, swz == 0] = buf[:, :, :, swz == 0]
    logical[:, :, :, swz == 1] = buf[:, :, :, swz == 1][:, :, :, :, ::-1]
    return logical.transpose(2, 0, 3, 1, 4, 5).reshape(s, lp, kp)


def split_on_gpu(gb, A, B, s):
    import torch
    m, k = A.shape
    n = B.shape[1]
    lay = gb.emulated_layout(s, m, n, k)
    ws = gb.alloc_workspace(lay.total)
    ws.fill_(0xAB)  # poison: every byte the layout defines must be written
    dA, dB = to_dev(A), to_dev(B)
    dC = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    gb.emulated_steps(dA, dB, dC, 1.0, 0.0, s, ws, steps=("split_a", "split_b"))
    torch.cuda.synchronize()
    raw = ws.cpu().numpy()
    kp = lay.kp
    assert lay.a_tile_rows == 128 and lay.b_tile_rows == (48 if s <= 10 else 32)
    da = untile(raw, lay.a_digits, s, m, kp, lay.a_tile_rows)
    db = untile(raw, lay.b_digits, s, n, kp, lay.b_tile_rows)
    ea = raw[lay.a_exp:lay.a_exp + 4 * m].view(np.int32)
    fb = raw[lay.b_exp:lay.b_exp + 4 * n].view(np.int32)
    return da, db, ea, fb, kp


@pytest.mark.parametrize("kind", ["uniform", "hard"])
@pytest.mark.parametrize("m,n,k,s", [(37, 45, 70, 11), (128, 64, 256, 16), (5, 300, 33, 1),
                                     (200, 3, 129, 7), (130, 97, 64, 10), (3, 49, 40, 9)])
def test_split_digits_and_exponents_bit_exact(gb, kind, m, n, k, s):
    A, B, _ = inputs(kind, m, n, k, 31, with_c=False)
    da, db, ea, fb, kp = split_on_gpu(gb, A, B, s)
    e, _ = ozaki.exponents(A, axis=1)
    f, _ = ozaki.exponents(B, axis=0)
    assert np.array_equal(ea, e) and np.array_equal(fb, f)
    DA, _ = ozaki.slice_digits(A, e, s, axis=1)
    DB, _ = ozaki.slice_digits(B, f, s, axis=0)
    vals_a = e4m3_decode(da)
    vals_b = e4m3_decode(db)
    assert np.array_equal(vals_a[:, :m, :k], DA.astype(np.float64))
    assert np.array_equal(vals_b[:, :n, :k], DB.transpose(0, 2, 1).astype(np.float64))
    # K padding and line padding hold zero digits
    assert np.all(vals_a[:, :, k:] == 0) and np.all(vals_b[:, :, k:] == 0)
    assert np.all(vals_a[:, m:, :] == 0) and np.all(vals_b[:, n:, :] == 0)


@pytest.mark.parametrize("s", [1, 2, 4, 8, 9, 11, 13, 16])
def test_products_bit_exact_against_model(gb, s):
    m, n, k = 300, 200, 129
    A, B, C0 = inputs("uniform", m, n, k, 32)
    want = ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s)
    got = emulate(gb, A, B, C0, 1.5, 0.5, s)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind,s", [("uniform", 11), ("hard", 13)])
def test_config0_within_fp64_bound(gb, kind, s):
    # C = 1.5 A B + 0.5 C at n = 256: the emulated result meets the FP64 contract
    A, B, C0 = inputs(kind, 256, 256, 256, g.BASE_SEED + (0 if kind == "uniform" else 3))
    got = emulate(gb, A, B, C0, 1.5, 0.5, s)
    assert np.array_equal(got, ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s))
    assert within_bound(got, 1.5, A, B, 0.5, C0) <= 1.0


@pytest.mark.parametrize("s", [1, 2, 11])
def test_integer_variant_bit_exact(gb, s):
    A, B, C0 = inputs("int8", 256, 256, 256, g.BASE_SEED + 100)
    want = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    assert np.array_equal(emulate(gb, A, B, C0, 1.5, 0.5, s), want)


@pytest.mark.parametrize("s,k", [(16, 4200), (10, 6600), (10, 13100), (12, 6600)])
def test_long_k_accumulates_in_exact_chunks(gb, s, k):
    # K beyond (2^24 / (256 s)) runs in several tensor-memory chunks whose exact
    # 128-bit sums are added (one and two chunk boundaries at s = 16 and s = 10,
    # 48-column tiles at s = 10), or, at s = 12 with 32-column tiles, in two sets
    # of level accumulators; bit-exact against the model, whose level sums are
    # exact in FP64.
    A, B, C0 = inputs("hard", 130, 40, k, 34)
    want = ozaki.emulated_gemm(-0.5, A, B, 2.0, C0, s=s)
    assert np.array_equal(emulate(gb, A, B, C0, -0.5, 2.0, s), want)


def test_largest_level_sums_exact_in_tensor_memory(gb):
    # every digit of A and B is (16, 0, 0, 0, -16): S_2 = 256 k = 2^21 at k = 8192,
    # the largest exact level-2 sum; the result k (1 - 2^-20)^2 is exact (s = 9).
    k = 8192
    v = 1.0 - 2.0 ** -20
    A = np.full((130, k), v)
    B = np.full((k, 70), v)
    got = emulate(gb, A, B, None, 1.0, 0.0, 9)
    assert np.all(got == k * (1.0 - 2.0 ** -19 + 2.0 ** -40))
    got5 = emulate(gb, A, B, None, 1.0, 0.0, 5)
    assert np.all(got5 == k * (1.0 - 2.0 ** -19))


@pytest.mark.parametrize("k", [40, 3000])
def test_nonfinite_rows_and_columns(gb, k):
    # k = 3000: the column maxima of B run over 16 K ranges; the non-finite values
    # of B sit in the first and the last range, and a column's largest magnitude
    # in a middle one
    import torch
    A, B, _ = inputs("uniform", 70, 50, k, 33, with_c=False)
    A[4, 7] = np.inf
    B[9, 13] = np.nan
    if k > 40:
        B[k - 3, 40] = -np.inf
        B[k // 2, 20] = 1.0e6
    q = gb.Queue(gb.Device(0), torch.cuda.current_stream())
    dA, dB = to_dev(A), to_dev(B)
    dC = torch.zeros((70, 50), dtype=torch.float64, device="cuda")
    gb.dgemm(dA, dB, dC, 1.0, 0.0, precision="emulated", slices=8, queue=q)
    with pytest.raises(gb.GbError, match="GB_ERR_NONFINITE"):
        q.wait()
    q.wait()  # the status was cleared by the first wait
    got = dC.cpu().numpy()
    want = ozaki.emulated_gemm(1.0, A, B, s=8)
    assert np.all(np.isnan(got[4, :])) and np.all(np.isnan(got[:, 13]))
    if k > 40:
        assert np.all(np.isnan(got[:, 40])) and not np.any(np.isnan(got[:3, 20]))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert np.array_equal(got[fin], want[fin])


def test_workspace_errors(gb):
    import torch
    A, B, C0 = inputs("uniform", 16, 16, 16, 34)
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
    with pytest.raises(gb.GbError, match="GB_ERR_WORKSPACE"):
        gb.dgemm(dA, dB, dC, precision="emulated", slices=8,
                 workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.dgemm(dA, dB, dC, precision="emulated", slices=17)


@pytest.mark.parametrize("n,s,kind", [(4096, 10, "uniform"), (8192, 10, "uniform"),
                                      (8192, 11, "uniform"), (8192, 11, "hard")])
def test_full_size_sampled_rows(gb, n, s, kind):
    # square sizes of the emulated workload (uniform, and the 16-decade hard set
    # at the slice count it needs): 8 sampled rows against the model (bit-exact)
    # and against the double-double reference (FP64 bound)
    A, B, _ = inputs(kind, n, n, n, g.BASE_SEED + (2 if kind == "uniform" else 3), with_c=False)
    got = emulate(gb, A, B, None, 1.0, 0.0, s)
    rows = np.random.default_rng(n + s).choice(n, 8, replace=False)
    want = ozaki.emulated_gemm(1.0, A, B, s=s, rows=rows)
    assert np.array_equal(got[rows], want)
    assert within_bound(got[rows], 1.0, A, B, 0.0, None, rows=rows) <= 1.0


@pytest.mark.parametrize("s", [10, 12])
def test_emulated_writes_only_c(gb, s):
    """C as a window of a larger canary-filled buffer (ldc > n, rows above and
    below): the emulated path writes exactly the m x n window."""
    import torch
    m, n, k = 200, 97, 150
    A, B, C0 = inputs("uniform", m, n, k, 35)
    canary = -12345.678
    big = np.full((m + 3, n + 7), canary)
    big[1:1 + m, 2:2 + n] = C0
    dbig = to_dev(big)
    dC = dbig[1:1 + m, 2:2 + n]
    gb.dgemm(to_dev(A), to_dev(B), dC, 1.5, 0.5, precision="emulated", slices=s)
    torch.cuda.synchronize()
    out = dbig.cpu().numpy()
    mask = np.ones_like(out, dtype=bool)
    mask[1:1 + m, 2:2 + n] = False
    assert np.all(out[mask] == canary)
    assert np.array_equal(out[1:1 + m, 2:2 + n], ozaki.emulated_gemm(1.5, A, B, 0.5, C0, s=s))
