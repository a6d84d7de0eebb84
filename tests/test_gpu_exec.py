"""GPU parity of DAXPY (Section 4.1) against the CPU oracle, bit for bit (one
fused multiply-add per element on both sides), over default and explicit work
divisions, unaligned vectors and edge cases; and of the generic executor
enqueueing the same kernel with an explicit work division."""
import ctypes

import numpy as np
import pytest

from oracle import cgemm
from synth import generators as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def vecs(n, seed):
    return (g.uniform_pm1(g.raw_stream(seed, 0, n)), g.uniform_pm1(g.raw_stream(seed, 1, n)))


@pytest.mark.parametrize("n", [1, 7, 1000, (1 << 20) + 3])
def test_daxpy_bit_exact(gb, n):
    import torch
    x, y = vecs(n, 70 + n % 13)
    alpha = 1.0 / 3.0
    want = cgemm.daxpy(alpha, x, y)
    dy = torch.from_numpy(y).cuda()
    gb.daxpy(alpha, torch.from_numpy(x).cuda(), dy)
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy(), want)


@pytest.mark.parametrize("B,V", [(32, 1), (128, 2), (256, 8), (1024, 4)])
def test_daxpy_explicit_workdivs_and_unaligned(gb, B, V):
    import torch
    n = 100003
    x, y = vecs(n + 1, 80)
    want = cgemm.daxpy(-2.5, x[1:], y[1:])
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    wd = gb.Workdiv.make([-(-n // (B * V))], [B], [V])
    gb.daxpy(-2.5, dx[1:], dy[1:], workdiv=wd)   # 8-byte but not 16-byte aligned
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy()[1:], want)
    assert dy.cpu().numpy()[0] == y[0]


def test_daxpy_edge_cases_and_rejections(gb):
    import torch
    x, y = vecs(64, 81)
    dy = torch.from_numpy(y).cuda()
    gb.daxpy(0.0, torch.full((64,), float("nan"), dtype=torch.float64, device="cuda"), dy)
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy(), y)          # alpha = 0: y untouched
    for grid, block, elems in [([1], [256], [4]),       # does not cover 64 x 4? covers 1024: ok
                               ([1], [100], [1]),       # not a multiple of 32
                               ([1], [256], [3])]:      # no such V
        wd = gb.Workdiv.make(grid, block, elems)
        if block == [256] and elems == [4]:
            gb.daxpy(1.0, torch.from_numpy(x).cuda(), dy, workdiv=wd)
            continue
        with pytest.raises(gb.GbError, match="INVALID_WORKDIV"):
            gb.daxpy(1.0, torch.from_numpy(x).cuda(), dy, workdiv=wd)
    with pytest.raises(gb.GbError, match="INVALID_WORKDIV"):
        gb.daxpy(1.0, torch.from_numpy(x).cuda(), dy, workdiv=gb.Workdiv.make([1], [32], [1]))


def test_generic_executor_runs_a_kernel_with_a_workdiv(gb):
    import torch
    n = 5000
    x, y = vecs(n, 82)
    want = cgemm.daxpy(0.75, x, y)
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    k = gb.kernel_handle("daxpy_v2")
    wd = gb.Workdiv.make([-(-n // (64 * 2))], [64], [2])
    gb.enqueue(k, wd, [ctypes.c_int64(n), ctypes.c_double(0.75),
                       ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dy.data_ptr())])
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy(), want)
    # a two-dimensional division runs too (rows on y, columns on x): 5 x 1000
    dy2 = torch.from_numpy(y).cuda()
    wd2 = gb.Workdiv.make([1, 5], [1, 512], [1, 2])
    gb.enqueue(k, wd2, [ctypes.c_int64(n), ctypes.c_double(0.75),
                        ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dy2.data_ptr())])
    torch.cuda.synchronize()
    assert np.array_equal(dy2.cpu().numpy(), want)
    with pytest.raises(gb.GbError, match="INVALID_WORKDIV"):
        gb.enqueue(k, gb.Workdiv.make([1, 1], [64, 64], [1, 1]), [ctypes.c_int64(0)] * 4)
    with pytest.raises(KeyError):
        gb.kernel_handle("nope")


def test_executor_launch_of_a_dgemm_kernel_equals_gb_dgemm(gb):
    # the paper's zero-overhead comparison: the same tiled kernel through the
    # DGEMM entry point and raw through the executor gives the same bits
    import torch
    m, n, k = 100, 70, 90
    A = torch.from_numpy(g.matrix("uniform", m, k, 83, 0)).cuda()
    B = torch.from_numpy(g.matrix("uniform", k, n, 83, 1)).cuda()
    C0 = torch.from_numpy(g.matrix("uniform", m, n, 83, 2)).cuda()
    want = C0.clone()
    gb.dgemm(A, B, want, 1.5, 0.5, kernel="tiled")
    got = C0.clone()
    P = ctypes.c_void_p
    gb.enqueue(gb.kernel_handle("dgemm_tiled16"),
               gb.Workdiv.make([-(-m // 16), -(-n // 16)], [16, 16], [1, 1]),
               [ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(k), ctypes.c_double(1.5),
                P(A.data_ptr()), ctypes.c_int64(k), P(B.data_ptr()), ctypes.c_int64(n),
                ctypes.c_double(0.5), P(got.data_ptr()), ctypes.c_int64(n)])
    torch.cuda.synchronize()
    assert torch.equal(got, want)
