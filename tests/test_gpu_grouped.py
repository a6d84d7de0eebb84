"""GPU parity of the grouped (persistent, graph-captured) GEMMs.

The grouped result of each problem equals the single-launch result bit for bit
(every native tile variant accumulates fma(A[i,l], B[l,j], acc) in l order like the
single DFMA kernel; same digits and products in the emulated path), and each is within the FP64 bound of the
oracle.  Problem sizes follow the grouped workload's recipe (m, n, k
log-uniform in [16, 512]) at a reduced count, plus edge cases.
"""
import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def make_group(count, seed, precision="native", tile="auto", emulated_every=0):
    ms, ns, ks = g.grouped_problems(seed, count)
    probs, host = [], []
    for i, (m, n, k) in enumerate(zip(ms, ns, ks)):
        A = g.matrix("uniform", int(m), int(k), seed + i, 0)
        B = g.matrix("uniform", int(k), int(n), seed + i, 1)
        C0 = g.matrix("uniform", int(m), int(n), seed + i, 2)
        prec = precision
        if emulated_every and i % emulated_every == 0:
            prec = "emulated"
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=1.0, beta=0.5,
                          precision=prec, slices=12, tile=tile))
        host.append((A, B, C0))
    return probs, host


def check_bound(probs, host):
    worst = 0.0
    for p, (A, B, C0) in zip(probs, host):
        got = p["C"].cpu().numpy()
        k = A.shape[1]
        ref = cgemm.dgemm(p["alpha"], A, B, p["beta"], C0.copy())
        bound = exact.error_bound(k, p["alpha"], cgemm.dgemm(1.0, np.abs(A), np.abs(B)),
                                  p["beta"], C0)
        # the oracle is itself within the bound of C*, so |got - ref| <= 2 bound
        diff = np.abs(got - ref)
        assert np.all(diff[bound == 0] == 0)
        ratio = diff[bound > 0] / bound[bound > 0]
        worst = max(worst, float(np.max(ratio)) if ratio.size else 0.0)
    return worst


@pytest.mark.parametrize("tile", ["auto", "64x64", "32x32", "64x32", "32x64"])
def test_native_group_matches_single_launches_bit_exact(gb, tile):
    import torch
    probs, host = make_group(96, 4401, tile=tile)
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["launches"] == 1 and info["emulated_tiles"] == 0
    for p, (A, B, C0) in zip(probs, host):
        single = to_dev(C0)
        gb.dgemm(to_dev(A), to_dev(B), single, p["alpha"], p["beta"], kernel="dfma")
        torch.cuda.synchronize()
        assert torch.equal(p["C"], single)
    assert check_bound(probs, host) <= 2.0
    plan.close()


def test_graph_replay_recomputes(gb):
    import torch
    probs, host = make_group(64, 4402)
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    first = [p["C"].clone() for p in probs]
    for p, (_, _, C0) in zip(probs, host):
        p["C"].copy_(to_dev(C0))
    plan.run()
    plan.run()  # beta = 0.5: the second replay updates C again
    torch.cuda.synchronize()
    for p, f, (A, B, C0) in zip(probs, first, host):
        again = f.clone()
        gb.dgemm(to_dev(A), to_dev(B), again, p["alpha"], p["beta"], kernel="dfma")
        torch.cuda.synchronize()
        assert torch.equal(p["C"], again)
    plan.close()


def test_emulated_and_mixed_group(gb):
    import torch
    probs, host = make_group(60, 4403, emulated_every=3)
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["emulated_tiles"] > 0 and info["native_tiles"] > 0 and info["launches"] == 4
    for p, (A, B, C0) in zip(probs, host):
        single = to_dev(C0)
        if p["precision"] == "emulated":
            gb.dgemm(to_dev(A), to_dev(B), single, p["alpha"], p["beta"], precision="emulated",
                     slices=p["slices"])
        else:
            gb.dgemm(to_dev(A), to_dev(B), single, p["alpha"], p["beta"], kernel="dfma")
        torch.cuda.synchronize()
        assert torch.equal(p["C"], single)
    assert check_bound(probs, host) <= 2.0
    plan.close()


def test_emulated_group_with_several_slice_counts(gb):
    """Problems of different s run in one launch set per slice count (split rows,
    column strips, products); each equals its single launch."""
    import torch
    ms, ns, ks = g.grouped_problems(5519, 24)
    slices = [3, 16, 8, 12]
    probs, host = [], []
    for i, (m, n, k) in enumerate(zip(ms, ns, ks)):
        A = g.matrix("hard", int(m), int(k), 5519 + i, 0)
        B = g.matrix("hard", int(k), int(n), 5519 + i, 1)
        C0 = g.matrix("uniform", int(m), int(n), 5519 + i, 2)
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=-0.75, beta=0.5,
                          precision="emulated", slices=slices[i % 4]))
        host.append((A, B, C0))
    plan = gb.GroupedPlan(probs, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["native_tiles"] == 0 and info["launches"] == 3 * len(set(slices))
    for p, (A, B, C0) in zip(probs, host):
        single = to_dev(C0)
        gb.dgemm(to_dev(A), to_dev(B), single, p["alpha"], p["beta"], precision="emulated",
                 slices=p["slices"])
        torch.cuda.synchronize()
        assert torch.equal(p["C"], single)
    plan.close()


def test_emulated_group_at_the_tuned_slice_count_meets_the_fp64_bound(gb):
    """The grouped workload's recipe (m, n, k log-uniform in [16, 512], uniform
    [-1, 1]) at s = 11, the slice count its benchmark uses: every problem within
    the FP64 bound against the double-double reference.  (At s = 10 the CPU model
    of the split-precision steps already exceeds the bound on a k = 19 problem of
    this set: the bound falls faster with k than the digit-truncation error.)"""
    import torch
    from gpu_util import within_bound
    ms, ns, ks = g.grouped_problems(g.BASE_SEED + 3, 40)
    probs, host = [], []
    for i, (m, n, k) in enumerate(zip(ms, ns, ks)):
        A = g.matrix("uniform", int(m), int(k), 7100 + i, 0)
        B = g.matrix("uniform", int(k), int(n), 7100 + i, 1)
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=torch.zeros((int(m), int(n)),
                     dtype=torch.float64, device="cuda"), precision="emulated", slices=11))
        host.append((A, B))
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    for p, (A, B) in zip(probs, host):
        assert within_bound(p["C"].cpu().numpy(), 1.0, A, B, 0.0, np.zeros_like(p["C"].cpu().numpy())) <= 1.0


def test_slices_zero_takes_the_tables_count(gb):
    """A problem submitted with slices = 0 runs at the slice count of the tuning
    table's entry for its K (else 11): bit-identical to the same group with the
    counts given explicitly, and within the FP64 bound against the oracle."""
    import torch
    big = (1 << 31) - 1
    ms, ns, ks = g.grouped_problems(8821, 30)
    table = [(big, big, 64, "emu_s12"), (big, big, 256, "emu_s10")]
    want = [12 if k <= 64 else 10 if k <= 256 else 11 for k in ks]
    probs, explicit, host = [], [], []
    for i, (m, n, k) in enumerate(zip(ms, ns, ks)):
        A = g.matrix("uniform", int(m), int(k), 8821 + i, 0)
        B = g.matrix("uniform", int(k), int(n), 8821 + i, 1)
        C0 = g.matrix("uniform", int(m), int(n), 8821 + i, 2)
        base = dict(A=to_dev(A), B=to_dev(B), alpha=1.5, beta=0.5, precision="emulated")
        probs.append(dict(base, C=to_dev(C0), slices=0))
        explicit.append(dict(base, C=to_dev(C0), slices=want[i]))
        host.append((A, B, C0))
    saved = gb.tune_get()
    gb.tune_set(table)
    try:
        assert [gb.tune_lookup_slices(int(m), int(n), int(k)) for m, n, k in zip(ms, ns, ks)] == want
        plan = gb.GroupedPlan(probs, use_graph=True)
        plan.run()
        torch.cuda.synchronize()
        assert plan.info()["launches"] == 3 * len(set(want))
        plan.close()
    finally:
        gb.tune_set(saved)
    gb.dgemm_grouped(explicit)
    torch.cuda.synchronize()
    for p, q in zip(probs, explicit):
        assert torch.equal(p["C"], q["C"])
    assert check_bound(probs, host) <= 2.0


def test_edge_problems_in_a_group(gb):
    import torch
    A, B, C0 = (g.matrix("uniform", 40, 30, 9, 0), g.matrix("uniform", 30, 20, 9, 1),
                g.matrix("uniform", 40, 20, 9, 2))
    e = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    probs = [
        dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=0.0, beta=0.25),           # beta C
        dict(A=to_dev(A), B=to_dev(B), C=torch.full((40, 20), float("nan"), dtype=torch.float64,
                                                      device="cuda"), alpha=1.0, beta=0.0),
        dict(A=e, B=torch.empty((5, 7), dtype=torch.float64, device="cuda"),
             C=torch.empty((0, 7), dtype=torch.float64, device="cuda")),               # m = 0
        dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=1.0, beta=1.0,
             precision="emulated", slices=0),
    ]
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    assert np.array_equal(probs[0]["C"].cpu().numpy(), 0.25 * C0)
    assert np.isfinite(probs[1]["C"].cpu().numpy()).all()
    bound = exact.error_bound(30, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)), 1.0, C0)
    ref = cgemm.dgemm(1.0, A, B, 1.0, C0.copy())
    assert np.all(np.abs(probs[3]["C"].cpu().numpy() - ref) <= 2 * bound)


def test_invalid_descriptor_rejected(gb):
    A = to_dev(g.matrix("uniform", 8, 8, 1, 0))
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.dgemm_grouped([dict(A=A, B=A, C=A.clone(), precision="emulated", slices=40)])


@pytest.mark.parametrize("tile", ["64x64", "32x32", "64x32", "32x64"])
def test_native_group_ragged_edges(gb, tile):
    """Warps skip the FMAs of padding rows, columns and K indices: problems whose
    m, n, k end inside a warp's 4 x 8 block, inside a 16-wide K stage, or below
    one block (m, n, k = 1) still give the single-launch bits and stay within the
    FP64 bound of the oracle (integer-valued inputs: exact)."""
    import torch
    sizes = [(1, 1, 1), (3, 5, 7), (4, 8, 16), (5, 9, 17), (33, 31, 15), (65, 63, 1),
             (63, 65, 33), (31, 1, 40), (1, 70, 3), (97, 17, 47), (64, 64, 16), (2, 130, 9)]
    probs, host = [], []
    for i, (m, n, k) in enumerate(sizes):
        kind = "int8" if i % 2 else "uniform"
        A = g.matrix(kind, m, k, 6100 + i, 0)
        B = g.matrix(kind, k, n, 6100 + i, 1)
        C0 = g.matrix(kind, m, n, 6100 + i, 2)
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=to_dev(C0), alpha=1.5, beta=0.5,
                          tile=tile))
        host.append((A, B, C0))
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    for i, (p, (A, B, C0)) in enumerate(zip(probs, host)):
        single = to_dev(C0)
        gb.dgemm(to_dev(A), to_dev(B), single, 1.5, 0.5, kernel="dfma")
        torch.cuda.synchronize()
        assert torch.equal(p["C"], single)
        if i % 2:
            star = np.array([[float(v) for v in row]
                             for row in exact.fraction_gemm(1.5, A, B, 0.5, C0)])
            assert np.array_equal(p["C"].cpu().numpy(), star)
    assert check_bound(probs, host) <= 2.0


def test_emulated_group_wide_problems_run_transposed(gb):
    """Problems with n well above m run as C^T = B^T A^T (B's columns on the
    128-row side of the tiles): each still equals the single launch bit for bit,
    with beta != 0, leading dimensions wider than the rows, and NaN / Inf lines
    (their rows of C, or columns, are NaN)."""
    import torch
    sizes = [(16, 500, 40, 10), (20, 300, 129, 11), (33, 2000, 64, 12), (130, 140, 70, 10),
             (40, 97, 33, 9), (500, 16, 40, 10)]
    probs, host = [], []
    for i, (m, n, k, s) in enumerate(sizes):
        A = g.matrix("uniform", m, k, 9200 + i, 0)
        B = g.matrix("hard" if i % 2 else "uniform", k, n, 9200 + i, 1)
        C0 = g.matrix("uniform", m, n, 9200 + i, 2)
        if i == 0:
            A[3, 7] = np.nan
            B[5, 411] = np.inf
        Aw = np.full((m, k + 3), np.nan)
        Aw[:, :k] = A
        dA = to_dev(Aw)[:, :k]
        probs.append(dict(A=dA, B=to_dev(B), C=to_dev(C0), alpha=1.25, beta=-0.5,
                          precision="emulated", slices=s))
        host.append((A, B, C0))
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    for i, (p, (A, B, C0)) in enumerate(zip(probs, host)):
        single = to_dev(C0)
        gb.dgemm(to_dev(A), to_dev(B), single, 1.25, -0.5, precision="emulated",
                 slices=p["slices"])
        torch.cuda.synchronize()
        got = p["C"].cpu().numpy()
        assert np.array_equal(got, single.cpu().numpy(), equal_nan=True)
        if i == 0:
            assert np.isnan(got[3]).all() and np.isnan(got[:, 411]).all()
            mask = np.ones_like(got, dtype=bool)
            mask[3] = False
            mask[:, 411] = False
            assert np.isfinite(got[mask]).all()
    # the NaN / Inf input left its status on the queue: reported once, then cleared
    q = gb.default_queue()
    with pytest.raises(gb.GbError, match="GB_ERR_NONFINITE"):
        q.wait()
    q.wait()


def test_emulated_group_writes_only_c(gb):
    """Every C of a group (wide problems run transposed, tall ones not) is a window
    of a larger canary-filled buffer: only the m x n windows change."""
    import torch
    canary = -777.25
    sizes = [(16, 500, 40), (300, 20, 64), (50, 51, 33)]
    probs, bigs, wins = [], [], []
    for i, (m, n, k) in enumerate(sizes):
        A = g.matrix("uniform", m, k, 9300 + i, 0)
        B = g.matrix("uniform", k, n, 9300 + i, 1)
        big = to_dev(np.full((m + 2, n + 5), canary))
        C = big[1:1 + m, 3:3 + n]
        C.zero_()
        probs.append(dict(A=to_dev(A), B=to_dev(B), C=C, precision="emulated", slices=11))
        bigs.append(big)
        wins.append((m, n))
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    for big, (m, n) in zip(bigs, wins):
        out = big.cpu().numpy()
        mask = np.ones_like(out, dtype=bool)
        mask[1:1 + m, 3:3 + n] = False
        assert np.all(out[mask] == canary)
        assert np.isfinite(out[1:1 + m, 3:3 + n]).all()


def test_emulated_orientations_give_the_same_bits(gb):
    # the two orientations of the emulated product tiles (A's rows or B's columns
    # on the 128-line side, as the tuning table may choose per size cell) compute
    # the same exact level sums and round them once: bit-identical results, equal
    # to single launches, and different tile counts
    import torch
    results, tiles = {}, {}
    for orient in ("emu_rows", "emu_cols", "auto"):
        probs, host = make_group(40, 4409)
        for p in probs:
            p["precision"] = "emulated"
            p["slices"] = 11
            p["tile"] = orient
        plan = gb.GroupedPlan(probs, use_graph=True)
        plan.run()
        torch.cuda.synchronize()
        tiles[orient] = plan.info()["emulated_tiles"]
        results[orient] = [p["C"].clone() for p in probs]
        plan.close()
    for a, b, c in zip(results["emu_rows"], results["emu_cols"], results["auto"]):
        assert torch.equal(a, b) and torch.equal(a, c)
    assert tiles["emu_rows"] != tiles["emu_cols"]
    for (A, B, C0), got in zip(host, results["auto"]):
        single = to_dev(C0)
        gb.dgemm(to_dev(A), to_dev(B), single, 1.0, 0.5, precision="emulated", slices=11)
        torch.cuda.synchronize()
        assert torch.equal(got, single)


def test_unknown_orientations_rejected(gb):
    probs, _ = make_group(2, 4410)
    probs[0]["tile"] = "emu_rows"          # native problem with an emulated orientation
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.GroupedPlan(probs, use_graph=False)
    probs[0]["tile"] = "64x64"
    probs[1].update(precision="emulated", tile="32x32")   # emulated problem, native tile
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.GroupedPlan(probs, use_graph=False)


def test_trivial_problems_write_beta_c_bit_exactly(gb):
    # alpha == 0 or k == 0 in a group: C <- beta C with the bits of a single
    # launch (and of the oracle): a zero of C times a negative beta stays -0.0,
    # and beta == 0 writes +0.0 whatever alpha is
    import torch
    C0 = np.zeros((9, 7))
    C0[::2] = g.matrix("int8", 5, 7, 4420, 2)
    A = g.matrix("uniform", 9, 6, 4420, 0)
    B = g.matrix("uniform", 6, 7, 4420, 1)
    cases = [(0.0, -2.0, 6), (1.5, -2.0, 0), (-1.5, 0.0, 0), (0.0, 0.0, 6), (2.0, 0.5, 0)]
    probs = []
    for alpha, beta, k in cases:
        Ak = np.ascontiguousarray(A[:, :max(k, 1)])
        Bk = np.ascontiguousarray(B[:max(k, 1)])
        dA = to_dev(Ak)[:, :k] if k else torch.empty((9, 0), dtype=torch.float64, device="cuda")
        dB = to_dev(Bk)[:k] if k else torch.empty((0, 7), dtype=torch.float64, device="cuda")
        probs.append(dict(A=dA, B=dB, C=to_dev(C0), alpha=alpha, beta=beta))
    gb.dgemm_grouped(probs)
    torch.cuda.synchronize()
    for p, (alpha, beta, k) in zip(probs, cases):
        want = cgemm.dgemm(alpha, np.zeros((9, 1)), np.zeros((1, 7)), beta, C0.copy(), k=0)
        got = p["C"].cpu().numpy()
        assert np.array_equal(got.view(np.int64), want.view(np.int64)), (alpha, beta, k)
        single = to_dev(C0)
        gb.dgemm(p["A"], p["B"], single, alpha, beta)
        torch.cuda.synchronize()
        assert torch.equal(single.view(torch.int64), p["C"].view(torch.int64)), (alpha, beta, k)
