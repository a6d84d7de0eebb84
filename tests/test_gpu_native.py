"""GPU parity of the native FP64 kernels (naive, tiled, dfma, dmma) against the CPU
oracle: bit-exact on integer inputs and closed forms, within the FP64 bound on
floating-point inputs, with ragged shapes, padded leading dimensions, canaries
around C, BLAS edge cases and work-division validation."""
import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

from gpu_util import inputs, to_dev, within_bound

pytestmark = pytest.mark.gpu

KERNELS = ["naive", "tiled", "dfma", "dmma"]


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def run(gb, kernel, A, B, C0, alpha, beta, **kw):
    dA, dB = to_dev(A), to_dev(B)
    dC = to_dev(C0) if C0 is not None else None
    out = gb.dgemm(dA, dB, dC, alpha, beta, kernel=kernel, **kw)
    import torch
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kernel", KERNELS)
def test_config0_integer_variant_bit_exact(gb, kernel):
    # C = 1.5 A B + 0.5 C, n = 256, integers in [-8, 8]: unique exact result
    A, B, C0 = inputs("int8", 256, 256, 256, g.BASE_SEED + 100)
    want = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    got = run(gb, kernel, A, B, C0, 1.5, 0.5)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kernel", KERNELS)
def test_config0_uniform_within_bound(gb, kernel):
    A, B, C0 = inputs("uniform", 256, 256, 256, g.BASE_SEED + 0)
    got = run(gb, kernel, A, B, C0, 1.5, 0.5)
    assert within_bound(got, 1.5, A, B, 0.5, C0) <= 1.0


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 17, 5), (65, 63, 129), (255, 257, 33),
                                   (130, 1, 300), (1, 200, 77)])
def test_ragged_shapes_with_padding_and_canaries(gb, kernel, m, n, k):
    import torch
    A = g.matrix("uniform", m, k, 77, 0, ld=k + 3)        # NaN-poisoned padding
    B = g.matrix("uniform", k, n, 77, 1, ld=n + 5)
    C0 = g.matrix("uniform", m, n, 77, 2)
    canary = -12345.678
    Cbig = np.full((m + 2, n + 6), canary)
    Cbig[1:m + 1, 2:n + 2] = C0
    dA, dB, dCbig = to_dev(A), to_dev(B), to_dev(Cbig)
    gb.dgemm(dA[:, :k], dB[:, :n], dCbig[1:m + 1, 2:n + 2], 1.5, 0.5, kernel=kernel)
    torch.cuda.synchronize()
    out = dCbig.cpu().numpy()
    inner = out[1:m + 1, 2:n + 2]
    mask = np.ones_like(out, dtype=bool)
    mask[1:m + 1, 2:n + 2] = False
    assert np.all(out[mask] == canary)
    Ac, Bc = np.ascontiguousarray(A[:, :k]), np.ascontiguousarray(B[:, :n])
    assert np.isfinite(inner).all()
    assert within_bound(inner, 1.5, Ac, Bc, 0.5, C0) <= 1.0


@pytest.mark.parametrize("kernel", KERNELS)
def test_closed_forms_bit_exact(gb, kernel):
    n = 97
    rng = np.random.default_rng(5)
    B = g.matrix("uniform", n, 45, 8, 1)
    assert np.array_equal(run(gb, kernel, np.eye(n), B, None, 1.0, 0.0), B)
    perm = rng.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    assert np.array_equal(run(gb, kernel, P, B, None, 1.0, 0.0), B[perm])
    k = 1000
    assert np.all(run(gb, kernel, np.ones((33, k)), np.ones((k, 40)), None, 1.0, 0.0) == k)
    u, v = rng.integers(-9, 10, 50).astype(float), rng.integers(-9, 10, 60).astype(float)
    x, y = rng.integers(-9, 10, 70).astype(float), rng.integers(-9, 10, 70).astype(float)
    got = run(gb, kernel, np.outer(u, x), np.outer(y, v), None, 1.0, 0.0)
    assert np.array_equal(got, np.outer(u, v) * float(int(x.astype(int) @ y.astype(int))))


@pytest.mark.parametrize("kernel", KERNELS)
def test_blas_edge_cases(gb, kernel):
    import torch
    A, B, C0 = inputs("uniform", 40, 30, 20, 9)
    # beta = 0 does not read C (NaN there must not propagate)
    got = run(gb, kernel, A, B, np.full((40, 30), np.nan), 2.0, 0.0)
    assert np.isfinite(got).all()
    # alpha = 0: C <- beta C, A and B not read (NaN operands)
    got = run(gb, kernel, np.full_like(A, np.nan), np.full_like(B, np.nan), C0, 0.0, 0.25)
    assert np.array_equal(got, 0.25 * C0)
    # k = 0
    dC = to_dev(C0)
    gb.dgemm(torch.empty((40, 0), dtype=torch.float64, device="cuda"),
             torch.empty((0, 30), dtype=torch.float64, device="cuda"), dC, 1.0, 0.5,
             kernel=kernel)
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), 0.5 * C0)
    # m = 0 is a no-op
    gb.dgemm(torch.empty((0, 20), dtype=torch.float64, device="cuda"), to_dev(B),
             torch.empty((0, 30), dtype=torch.float64, device="cuda"), 1.0, 0.0, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_nonfinite_propagates_in_place(gb, kernel):
    A, B, _ = inputs("uniform", 20, 24, 16, 10, with_c=False)
    A[3, 5] = np.inf
    B[7, 11] = np.nan
    want = cgemm.dgemm(1.0, A, B)
    got = run(gb, kernel, A, B, None, 1.0, 0.0)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isinf(got), np.isinf(want))


@pytest.mark.parametrize("grid_block_elem,kernel", [
    (((4, 10), (32, 8), (1, 1)), "naive"),
    (((13, 3), (8, 32), (1, 1)), "naive"),
    (((13, 10), (8, 8), (1, 1)), "tiled"),
    (((4, 3), (32, 32), (1, 1)), "tiled"),
    (((4, 3), (16, 16), (2, 2)), "dfma"),
    (((1, 1), (16, 16), (8, 8)), "dfma"),
    (((7, 5), (2, 2), (16, 16)), "dmma"),
    (((1, 2), (4, 2), (32, 32)), "dmma"),
])
def test_explicit_workdivs_same_result(gb, grid_block_elem, kernel):
    A, B, C0 = inputs("uniform", 100, 70, 90, 11)
    wd = gb.Workdiv.make(*grid_block_elem)
    got = run(gb, kernel, A, B, C0, 1.0, 1.0, workdiv=wd)
    assert within_bound(got, 1.0, A, B, 1.0, C0) <= 1.0


def test_bad_workdivs_rejected_on_host(gb):
    A, B, C0 = inputs("uniform", 100, 70, 90, 11)
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
    for gbe, kernel in [(((3, 2), (32, 8), (1, 1)), "naive"),      # does not cover n
                        (((13, 10), (8, 16), (1, 1)), "tiled"),    # not square
                        (((4, 3), (16, 16), (3, 3)), "dfma"),      # no such variant
                        (((7, 5), (2, 2), (8, 8)), "dmma")]:
        with pytest.raises(gb.GbError, match="GB_ERR_INVALID_WORKDIV"):
            gb.dgemm(dA, dB, dC, 1.0, 0.0, kernel=kernel, workdiv=gb.Workdiv.make(*gbe))
    assert np.array_equal(dC.cpu().numpy(), C0)  # nothing was enqueued


def test_bad_arguments_rejected_on_host(gb):
    import torch
    A, B, C0 = inputs("uniform", 16, 16, 16, 12)
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C0)
    with pytest.raises(gb.GbError, match="GB_ERR_INVALID_ARG"):
        gb.dgemm(dA, dB, dC, float("nan"), 0.0)
    q = gb.default_queue()
    lib = gb.load()
    import ctypes
    # lda < k
    st = lib.gb_dgemm(q.handle, None, 0, 0, 0, 16, 16, 16, 1.0, ctypes.c_void_p(dA.data_ptr()), 8,
                      ctypes.c_void_p(dB.data_ptr()), 16, 0.0, ctypes.c_void_p(dC.data_ptr()), 16,
                      None, 0)
    assert st == 1
    # misaligned C
    st = lib.gb_dgemm(q.handle, None, 0, 0, 0, 4, 4, 4, 1.0, ctypes.c_void_p(dA.data_ptr()), 16,
                      ctypes.c_void_p(dB.data_ptr()), 16, 0.0,
                      ctypes.c_void_p(dC.data_ptr() + 4), 16, None, 0)
    assert st == 1
    torch.cuda.synchronize()


def test_blocking_queue_returns_after_work(gb):
    import torch
    dev = gb.Device(0)
    s = torch.cuda.Stream()
    q = gb.Queue(dev, s, blocking=True)
    A, B, C0 = inputs("int8", 64, 64, 64, 13)
    dA, dB = to_dev(A), to_dev(B)
    dC = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    gb.dgemm(dA, dB, dC, 1.0, 0.0, queue=q)
    assert s.query()  # blocking queue: the stream is idle on return
    assert np.array_equal(dC.cpu().numpy(), cgemm.dgemm(1.0, A, B))
    q.wait()
    q.close()


@pytest.mark.parametrize("n", [1024, 4096, 8192, 10240])
def test_sweep_sizes_sampled_rows(gb, n):
    # full-size sweep points of the square DGEMM (alpha = 1, beta = 0): the
    # outputs of 12 sampled rows of every kernel the sweep reports (naive, tiled,
    # DFMA, DMMA, and the AUTO choice) against the double-double reference and
    # the oracle computed row by row
    A, B, _ = inputs("uniform", n, n, n, g.BASE_SEED + 1, with_c=False)
    rows = np.random.default_rng(n).choice(n, 12, replace=False)
    ref = cgemm.dgemm_rows(rows, 1.0, A, B)
    hi, lo = cgemm.dgemm_dd_rows(A, B, rows)
    bound = exact.error_bound(n, 1.0, cgemm.dgemm_rows(rows, 1.0, np.abs(A), np.abs(B)))
    kernels = ["auto"] if n in (1024, 8192) else ["auto", "naive", "tiled", "dfma", "dmma"]
    for kernel in kernels:
        got = run(gb, kernel, A, B, None, 1.0, 0.0)
        assert np.all(np.abs(exact.residual(got[rows], 1.0, hi, lo)) <= bound), kernel
        # and the oracle itself on those rows is within the same bound
        assert np.all(np.abs(got[rows] - ref) <= 2 * bound), kernel
