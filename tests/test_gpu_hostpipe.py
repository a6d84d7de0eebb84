"""GPU parity of the host-buffer GEMM (gb_dgemm_host): operands and result in
pinned host memory, copied in bands and overlapped with the computation.

Each result equals, bit for bit, the same GEMM on device copies through gb_dgemm
(the same kernels on the same data; the band split of the emulated path only
changes which launch computes an output), for 1, 2, 3 and 4 row bands (the first
one in up to four column blocks of B, the last in one or two launches), leading
dimensions wider than the rows, beta = 0 and beta != 0, two calls in a row on
one workspace, and the native precision.
"""
import numpy as np
import pytest

from synth import generators as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def pinned(a, pad=0):
    """A pinned host tensor holding `a`, with `pad` extra columns (wider ld)."""
    import torch
    rows, cols = a.shape
    t = torch.empty((rows, cols + pad), dtype=torch.float64, pin_memory=True)
    t[:, :cols] = torch.from_numpy(a)
    if pad:
        t[:, cols:] = float("nan")  # never read
    return t[:, :cols]


def device_reference(gb, A, B, C0, alpha, beta, precision, s):
    import torch
    dC = torch.from_numpy(C0.copy()).cuda()
    gb.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC, alpha, beta,
             precision=precision, slices=s)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("m,n,k,s,beta,pad", [(900, 130, 70, 10, 0.0, 0),     # one band
                                              (2100, 300, 257, 10, 0.5, 3),
                                              (4500, 97, 129, 12, -1.0, 1),
                                              (8192, 2048, 32, 10, 0.5, 1),   # 2 bands, split
                                              (8100, 4090, 24, 11, 0.0, 0),   # 4 bands, 3 blocks
                                              (6144, 4096, 96, 10, 0.0, 2),   # 4 blocks of B
                                              (4096, 4096, 4096, 10, 0.5, 0)])  # last band split
def test_emulated_host_buffers_match_device_gemm(gb, m, n, k, s, beta, pad):
    import torch
    seed = 8100 + m
    A = g.matrix("uniform", m, k, seed, 0)
    B = g.matrix("uniform", k, n, seed, 1)
    C0 = g.matrix("uniform", m, n, seed, 2)
    want = device_reference(gb, A, B, C0, 1.5, beta, "emulated", s)
    hA, hB, hC = pinned(A, pad), pinned(B, pad), pinned(C0, pad)
    gb.dgemm_host(hA, hB, hC, 1.5, beta, precision="emulated", slices=s)
    torch.cuda.synchronize()
    assert np.array_equal(hC.numpy(), want)


def test_two_calls_in_a_row_share_the_workspace(gb):
    import torch
    m, n, k, s = 2304, 200, 96, 11
    ws = gb.alloc_workspace(gb.host_workspace_size("emulated", s, m, n, k))
    outs, wants = [], []
    for seed in (8301, 8302):
        A = g.matrix("uniform", m, k, seed, 0)
        B = g.matrix("hard", k, n, seed, 1)
        wants.append(device_reference(gb, A, B, np.zeros((m, n)), 1.0, 0.0, "emulated", s))
        hC = pinned(np.zeros((m, n)))
        gb.dgemm_host(pinned(A), pinned(B), hC, precision="emulated", slices=s, workspace=ws)
        outs.append(hC)
    torch.cuda.synchronize()
    for got, want in zip(outs, wants):
        assert np.array_equal(got.numpy(), want)


def test_native_host_buffers_match_device_gemm(gb):
    import torch
    m, n, k = 300, 200, 100
    A = g.matrix("uniform", m, k, 8401, 0)
    B = g.matrix("uniform", k, n, 8401, 1)
    C0 = g.matrix("uniform", m, n, 8401, 2)
    want = device_reference(gb, A, B, C0, -0.5, 2.0, "native", 0)
    hC = pinned(C0, 2)
    gb.dgemm_host(pinned(A, 1), pinned(B), hC, -0.5, 2.0, precision="native")
    torch.cuda.synchronize()
    assert np.array_equal(hC.numpy(), want)


def test_small_workspace_rejected(gb):
    m, n, k = 64, 64, 64
    need = gb.host_workspace_size("emulated", 10, m, n, k)
    ws = gb.alloc_workspace(need - 256)
    z = np.zeros((m, m))
    with pytest.raises(gb.GbError, match="WORKSPACE"):
        gb.dgemm_host(pinned(z), pinned(z), pinned(z), precision="emulated", slices=10,
                      workspace=ws)


@pytest.mark.parametrize("precision", ["native", "emulated"])
def test_degenerate_host_buffer_gemms(gb, precision):
    """alpha = 0 and k = 0 give beta C without reading A or B (the copies of A and
    B are skipped too); m = 0 is a no-op."""
    import torch
    m, n = 70, 90
    C0 = g.matrix("uniform", m, n, 8501, 2)
    A = g.matrix("uniform", m, 33, 8501, 0)
    B = g.matrix("uniform", 33, n, 8501, 1)
    hC = pinned(C0)
    gb.dgemm_host(pinned(A), pinned(B), hC, 0.0, 0.25, precision=precision, slices=10)
    torch.cuda.synchronize()
    assert np.array_equal(hC.numpy(), 0.25 * C0)
    hC = pinned(C0)
    gb.dgemm_host(pinned(np.zeros((m, 0))), pinned(np.zeros((0, n))), hC, 1.0, -2.0,
                  precision=precision, slices=10)
    torch.cuda.synchronize()
    assert np.array_equal(hC.numpy(), -2.0 * C0)
    empty = pinned(np.zeros((0, n)))
    gb.dgemm_host(pinned(np.zeros((0, 33))), pinned(B), empty, precision=precision, slices=10)
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", range(12))
def test_random_host_buffer_gemms(gb, case):
    # seeded random shapes across the band / column-block schedule (m up to 8192
    # rows, n up to 3000 columns), slice counts, alpha, beta and padded host rows:
    # every result equals the device GEMM bit for bit
    import torch
    rng = np.random.default_rng(8300 + case)
    m = int(rng.integers(1, 8193))
    n = int(rng.integers(1, 3001))
    k = int(rng.integers(1, 301))
    s = int(rng.integers(1, 17))
    alpha = float(rng.choice([1.0, -0.75, 2.0, 0.5]))
    beta = float(rng.choice([0.0, 0.5, -1.0]))
    pad = int(rng.integers(0, 4))
    seed = 8400 + case
    A = g.matrix("uniform", m, k, seed, 0)
    B = g.matrix("uniform", k, n, seed, 1)
    C0 = g.matrix("uniform", m, n, seed, 2)
    want = device_reference(gb, A, B, C0, alpha, beta, "emulated", s)
    hA, hB, hC = pinned(A, pad), pinned(B, pad), pinned(C0, pad)
    gb.dgemm_host(hA, hB, hC, alpha, beta, precision="emulated", slices=s)
    torch.cuda.synchronize()
    assert np.array_equal(hC.numpy().view(np.int64), want.view(np.int64)), (m, n, k, s)
