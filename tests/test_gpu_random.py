"""Seeded random-shape parity of both paths against the CPU oracle.

Each case draws m, n, k (1 .. 300, 1 .. 300, 1 .. 700), a slice count 1 .. 16,
alpha and beta (including 0, negative and power-of-two values), padded leading
dimensions (operands are views into wider buffers whose padding is NaN, so a
kernel that reads it is caught) and an input kind (uniform, the 16-decade hard
set, integers).  The emulated result must equal the step model bit for bit; every
native kernel must stay within the FP64 bound of the double-double reference, and
equal it exactly on integer inputs.
"""
import numpy as np
import pytest

from oracle import cgemm, exact, ozaki
from synth import generators as g

pytestmark = pytest.mark.gpu

ALPHAS = [1.0, -1.5, 0.5, 2.0 ** -3, 0.0, 3.25]
BETAS = [0.0, 0.5, -2.0, 1.0]
KINDS = ["uniform", "hard", "int8"]


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def draw(case):
    rng = np.random.default_rng(16020 + case)
    m, n = (int(x) for x in rng.integers(1, 301, 2))
    k = int(rng.integers(1, 701))
    s = int(rng.integers(1, 17))
    alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
    beta = BETAS[int(rng.integers(len(BETAS)))]
    kind = KINDS[int(rng.integers(len(KINDS)))]
    pads = [int(x) for x in rng.integers(0, 9, 3)]
    return m, n, k, s, alpha, beta, kind, pads


def padded(torch, X, pad):
    """X as a view into a NaN-padded buffer with leading dimension cols + pad."""
    rows, cols = X.shape
    buf = torch.full((rows, cols + pad), float("nan"), dtype=torch.float64, device="cuda")
    v = buf[:, :cols]
    v.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return buf, v


@pytest.mark.parametrize("case", range(48))
def test_random_shapes_both_paths(gb, case):
    import torch
    m, n, k, s, alpha, beta, kind, pads = draw(case)
    seed = 7700 + case
    A = g.matrix(kind, m, k, seed, g.STREAM_A)
    B = g.matrix(kind, k, n, seed, g.STREAM_B)
    C0 = g.matrix(kind, m, n, seed, g.STREAM_C)
    _, dA = padded(torch, A, pads[0])
    _, dB = padded(torch, B, pads[1])
    # emulated: bit-exact against the step model
    cbuf, dC = padded(torch, C0, pads[2])
    gb.dgemm(dA, dB, dC, alpha, beta, precision="emulated", slices=s)
    torch.cuda.synchronize()
    want = ozaki.emulated_gemm(alpha, A, B, beta, C0, s=s)
    got = dC.cpu().numpy()
    assert np.array_equal(got.view(np.int64), np.ascontiguousarray(want).view(np.int64)), \
        (m, n, k, s, alpha, beta, kind)
    assert bool(torch.isnan(cbuf[:, n:]).all())        # padding of C untouched
    # native kernels: within the FP64 bound of the double-double reference
    hi, lo = cgemm.dgemm_dd_rows(A, B)
    bound = exact.error_bound(k, alpha, cgemm.dgemm(1.0, np.abs(A), np.abs(B)), beta, C0)
    for kernel in ("auto", "naive", "tiled", "dfma", "dmma"):
        cbuf, dC = padded(torch, C0, pads[2])
        gb.dgemm(dA, dB, dC, alpha, beta, kernel=kernel)
        torch.cuda.synchronize()
        got = dC.cpu().numpy()
        res = exact.residual(got, alpha, hi, lo, beta, C0)
        assert np.all(np.abs(res) <= bound), (kernel, m, n, k, alpha, beta, kind)
        if kind == "int8":
            # integers with exact partial sums: every kernel gives the exact result
            assert np.array_equal(got, cgemm.dgemm(alpha, A, B, beta, C0.copy())), kernel
        assert bool(torch.isnan(cbuf[:, n:]).all())


@pytest.mark.parametrize("group", range(3))
def test_random_groups(gb, group):
    # 40 problems of random shapes, precisions, slice counts, alpha / beta and
    # padded leading dimensions in one graph-captured plan: each result equals the
    # same GEMM as a single launch (native: the DFMA kernel the grouped tiles
    # accumulate like; emulated: bit for bit, and the step model)
    import torch
    rng = np.random.default_rng(99100 + group)
    probs, host, bufs = [], [], []
    for i in range(40):
        m, n = (int(x) for x in rng.integers(1, 260, 2))
        k = int(rng.integers(1, 600))
        emulated = bool(rng.random() < 0.5)
        s = int(rng.integers(1, 17))
        alpha = ALPHAS[int(rng.integers(len(ALPHAS)))]
        beta = BETAS[int(rng.integers(len(BETAS)))]
        kind = KINDS[int(rng.integers(len(KINDS)))]
        pads = [int(x) for x in rng.integers(0, 6, 3)]
        seed = 8800 + 100 * group + i
        A = g.matrix(kind, m, k, seed, g.STREAM_A)
        B = g.matrix(kind, k, n, seed, g.STREAM_B)
        C0 = g.matrix(kind, m, n, seed, g.STREAM_C)
        ba, dA = padded(torch, A, pads[0])
        bb, dB = padded(torch, B, pads[1])
        bc, dC = padded(torch, C0, pads[2])
        bufs += [ba, bb, bc]
        probs.append(dict(A=dA, B=dB, C=dC, alpha=alpha, beta=beta,
                          precision="emulated" if emulated else "native", slices=s))
        host.append((A, B, C0, pads))
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    for p, (A, B, C0, pads) in zip(probs, host):
        _, dA = padded(torch, A, pads[0])
        _, dB = padded(torch, B, pads[1])
        _, single = padded(torch, C0, pads[2])
        if p["precision"] == "emulated":
            gb.dgemm(dA, dB, single, p["alpha"], p["beta"], precision="emulated",
                     slices=p["slices"])
        else:
            gb.dgemm(dA, dB, single, p["alpha"], p["beta"], kernel="dfma")
        torch.cuda.synchronize()
        got = p["C"].cpu().numpy()
        assert np.array_equal(got.view(np.int64), single.cpu().numpy().view(np.int64))
        if p["precision"] == "emulated":
            want = ozaki.emulated_gemm(p["alpha"], A, B, p["beta"], C0, s=p["slices"])
            assert np.array_equal(got.view(np.int64), np.ascontiguousarray(want).view(np.int64))
    plan.close()
