"""The launch schedule of the host-buffer GEMM (gb_dgemm_host, emulated), host side
only: the launches tile C exactly once on whole output tiles, the first band
walks the column blocks of B in order, the first block is small and the blocks
fill whole waves of the SMs, and the last band ends on a small block."""
import ctypes

import pytest

from paper_1602_08477_gb300 import _lib, build


@pytest.fixture(scope="module")
def gb():
    build()
    import paper_1602_08477_gb300 as gb
    return gb


def bn_of(s):
    return 48 if s <= 10 else 32


SHAPES = [(10, 8192, 8192, 8192, 0.0), (10, 4096, 4096, 4096, 0.5), (11, 8100, 4090, 24, 0.0),
          (10, 8192, 2048, 32, 0.5), (12, 4500, 97, 129, -1.0), (16, 8192, 8192, 8192, 0.0),
          (1, 8192, 8192, 8192, 0.0), (10, 16384, 16384, 16384, 0.0), (9, 1000, 7000, 300, 0.0),
          (11, 129, 33, 1, 1.0)]


@pytest.mark.parametrize("s,m,n,k,beta", SHAPES)
@pytest.mark.parametrize("sms", [152, 148, 7])
def test_launches_tile_c_once_on_tile_edges(gb, s, m, n, k, beta, sms):
    pieces = gb.host_schedule(s, m, n, k, beta, sm_count=sms)
    assert 1 <= len(pieces) <= 10
    bn = bn_of(s)
    area = 0
    for r0, r1, c0, c1 in pieces:
        assert 0 <= r0 < r1 <= m and 0 <= c0 < c1 <= n
        assert r0 % 128 == 0 and (r1 % 128 == 0 or r1 == m)
        assert c0 % bn == 0 and (c1 % bn == 0 or c1 == n)
        area += (r1 - r0) * (c1 - c0)
    assert area == m * n
    for i, a in enumerate(pieces):  # pairwise disjoint
        for b in pieces[i + 1:]:
            assert a[1] <= b[0] or b[1] <= a[0] or a[3] <= b[2] or b[3] <= a[2]
    # the first band's launches walk the column blocks of B from left to right,
    # and come before every other band's
    band0 = [p for p in pieces if p[0] == 0]
    assert pieces[:len(band0)] == band0
    assert band0[0][2] == 0 and band0[-1][3] == n
    for a, b in zip(band0, band0[1:]):
        assert a[3] == b[2]
    # later bands in row order
    rows = [p[0] for p in pieces]
    assert rows == sorted(rows)


def test_square_8192_starts_on_a_small_block_and_fills_whole_waves(gb):
    # 2048-row bands (16 tile rows) x 171 tile columns: 19 tile columns are the
    # smallest block of whole waves (16 x 19 = 2 x 152 tiles)
    pieces = gb.host_schedule(10, 8192, 8192, 8192, 0.0, sm_count=152)
    first = pieces[0]
    assert first == (0, 2048, 0, 19 * 48)
    band0 = [p for p in pieces if p[0] == 0]
    assert len(band0) >= 3
    for r0, r1, c0, c1 in band0[:-1]:
        tiles = (r1 - r0) // 128 * ((c1 - c0) // 48)
        assert tiles % 152 == 0
    # blocks never shrink (the link stays ahead of the products)
    widths = [c1 - c0 for _, _, c0, c1 in band0[:-1]]
    assert widths == sorted(widths)
    # the last band in two launches, the second the smaller
    last = [p for p in pieces if p[0] == 6144]
    assert len(last) == 2 and last[1][3] - last[1][2] < last[0][3] - last[0][2]


def test_small_problem_is_one_launch(gb):
    assert gb.host_schedule(10, 900, 130, 70, 0.0, sm_count=152) == [(0, 900, 0, 130)]


def test_empty_and_bad_arguments(gb):
    lib = _lib.load()
    count = ctypes.c_int(-1)
    buf = (ctypes.c_int64 * 40)()
    assert lib.gb_dgemm_host_schedule(10, 0, 100, 100, 0.0, 152, buf, 10, ctypes.byref(count)) == 0
    assert count.value == 0
    assert lib.gb_dgemm_host_schedule(10, 100, 100, 0, 0.0, 152, buf, 10, ctypes.byref(count)) == 0
    assert count.value == 0
    # too small an output array: the count is still reported
    assert lib.gb_dgemm_host_schedule(10, 8192, 8192, 8192, 0.0, 152, buf, 2,
                                      ctypes.byref(count)) == 1
    assert count.value == 10
    assert lib.gb_dgemm_host_schedule(17, 8, 8, 8, 0.0, 152, buf, 10, ctypes.byref(count)) == 1
    assert lib.gb_dgemm_host_schedule(10, -1, 8, 8, 0.0, 152, buf, 10, ctypes.byref(count)) == 1
    assert lib.gb_dgemm_host_schedule(10, 8, 8, 8, 0.0, 0, buf, 10, ctypes.byref(count)) == 1
    assert lib.gb_dgemm_host_schedule(10, 8, 8, 8, 0.0, 152, None, 10, ctypes.byref(count)) == 1
