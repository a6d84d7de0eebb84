"""GPU tests of the request server: each result is the same alone and in the mix
(bit for bit), budget admission, the device operand generator, host-side
rejection of a request that can never fit."""
import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    assert torch.cuda.is_available()
    return gb


def test_device_generator_matches_host_generator(gb):
    import torch
    t = torch.empty((37, 53), dtype=torch.float64, device="cuda")
    gb.fill_uniform(t, 1234, 1)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), g.matrix("uniform", 37, 53, 1234, 1))


def _requests(count, seed):
    sizes = g.log_uniform_ints(seed, 30, count, 16, 700)
    prec = (g.raw_stream(seed, 31, count) % np.uint64(5)) == 0  # ~20% emulated
    reqs = []
    for i in range(count):
        n = int(sizes[i])
        m = max(1, n // 2 + i % 7)
        k = max(1, n - i % 5)
        A = g.matrix("uniform", m, k, seed + i, 0)
        B = g.matrix("uniform", k, n, seed + i, 1)
        C0 = g.matrix("uniform", m, n, seed + i, 2)
        reqs.append(dict(m=m, n=n, k=k, A=A, B=B, C=C0, alpha=1.0, beta=0.5,
                         precision="emulated" if prec[i] else "native", slices=12))
    return reqs


def test_results_alone_equal_results_in_the_mix(gb):
    # 200 requests: the serving spot-check count, each compared alone, in the mix
    # and against the oracle
    reqs = _requests(200, 5500)
    # in the mix: all submitted at once to a server with small batches and a
    # budget that forces admission waits
    mix = gb.Server(hbm_budget_bytes=64 << 20, n_streams=3, max_batch=8)
    outs, ids = [], []
    for r in reqs:
        out = np.empty((r["m"], r["n"]))
        outs.append(out)
        ids.append(mix.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"],
                              r["slices"], A=r["A"], B=r["B"], C=r["C"], out=out))
    mix.drain(600)
    st = mix.stats()
    assert st["completed"] == len(reqs) and st["peak_bytes"] <= 64 << 20
    assert st["batches"] > 1
    for rid in ids:
        done, status, lat = mix.poll(rid)
        assert done and status == 0 and lat >= 0
    mix.close()
    # alone: one request per server
    for r, out in zip(reqs, outs):
        solo = gb.Server(hbm_budget_bytes=64 << 20, n_streams=1, max_batch=1)
        alone = np.empty((r["m"], r["n"]))
        solo.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"], r["slices"],
                    A=r["A"], B=r["B"], C=r["C"], out=alone)
        solo.drain(600)
        solo.close()
        assert np.array_equal(alone, out)
        # and within the FP64 bound of the oracle
        ref, _ = cgemm.dgemm_omp(r["alpha"], r["A"], r["B"], r["beta"], r["C"].copy())
        absab, _ = cgemm.dgemm_omp(1.0, np.abs(r["A"]), np.abs(r["B"]))
        bound = exact.error_bound(r["k"], r["alpha"], absab, r["beta"], r["C"])
        assert np.all(np.abs(out - ref) <= 2 * bound)


def test_lanes_run_large_requests_alone(gb):
    # native requests of >= 2^31 flops take the large lane (one plain GEMM launch
    # each); the rest are batched.  Each result equals the same request served
    # alone (single-stream server, same policy) and meets the FP64 bound; the FIFO
    # policy serves the same requests through grouped launches only.
    reqs = _requests(24, 7100)
    for i, (m, n, k) in enumerate([(1100, 1100, 1100), (700, 1500, 2100), (2050, 1030, 1040)]):
        seed = 7200 + i
        reqs.insert(5 * i + 2, dict(m=m, n=n, k=k, A=g.matrix("uniform", m, k, seed, 0),
                                    B=g.matrix("uniform", k, n, seed, 1),
                                    C=g.matrix("uniform", m, n, seed, 2), alpha=-0.75, beta=0.5,
                                    precision="native", slices=0))
    large = sum(1 for r in reqs if r["precision"] == "native"
                and 2.0 * r["m"] * r["n"] * r["k"] >= 2.0 ** 31)
    assert large == 3
    results = {}
    for policy, streams in (("lanes", 4), ("fifo", 2)):
        srv = gb.Server(hbm_budget_bytes=256 << 20, n_streams=streams, max_batch=16,
                        policy=policy)
        outs = []
        for r in reqs:
            out = np.empty((r["m"], r["n"]))
            outs.append(out)
            srv.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"],
                       r["slices"], A=r["A"], B=r["B"], C=r["C"], out=out)
        srv.drain(600)
        st = srv.stats()
        srv.close()
        assert st["completed"] == len(reqs)
        assert st["large_launches"] == (large if policy == "lanes" else 0)
        results[policy] = outs
    for i, r in enumerate(reqs):
        solo = gb.Server(hbm_budget_bytes=256 << 20, n_streams=1, max_batch=16)
        alone = np.empty((r["m"], r["n"]))
        solo.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"], r["slices"],
                    A=r["A"], B=r["B"], C=r["C"], out=alone)
        solo.drain(600)
        solo.close()
        assert np.array_equal(alone, results["lanes"][i])
        ref, _ = cgemm.dgemm_omp(r["alpha"], r["A"], r["B"], r["beta"], r["C"].copy())
        absab, _ = cgemm.dgemm_omp(1.0, np.abs(r["A"]), np.abs(r["B"]))
        bound = exact.error_bound(r["k"], r["alpha"], absab, r["beta"], r["C"])
        for policy in ("lanes", "fifo"):
            assert np.all(np.abs(results[policy][i] - ref) <= 2 * bound)


def test_server_rejects_an_unknown_policy(gb):
    with pytest.raises(ValueError):
        gb.Server(hbm_budget_bytes=8 << 20, policy="lifo")


def test_device_generated_operands(gb):
    import torch
    srv = gb.Server(hbm_budget_bytes=256 << 20, n_streams=2, max_batch=16)
    m, n, k = 300, 200, 150
    out = np.empty((m, n))
    rid = srv.submit(m, n, k, 1.5, 0.5, "native", 0, out=out, seed=777)
    srv.drain(120)
    assert srv.poll(rid)[0]
    A = g.matrix("uniform", m, k, 777, 0)
    B = g.matrix("uniform", k, n, 777, 1)
    C0 = g.matrix("uniform", m, n, 777, 2)
    ref = cgemm.dgemm(1.5, A, B, 0.5, C0.copy())
    bound = exact.error_bound(k, 1.5, cgemm.dgemm(1.0, np.abs(A), np.abs(B)), 0.5, C0)
    assert np.all(np.abs(out - ref) <= 2 * bound)
    srv.close()
    torch.cuda.synchronize()


def test_request_that_never_fits_is_rejected_on_the_host(gb):
    srv = gb.Server(hbm_budget_bytes=8 << 20, n_streams=1, max_batch=4)
    with pytest.raises(gb.GbError, match="OUT_OF_BUDGET"):
        srv.submit(1024, 1024, 1024)   # 24 MiB of operands > 8 MiB
    ok = srv.submit(64, 64, 64)
    srv.drain(60)
    assert srv.poll(ok)[0]
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_requests_admitted_while_a_large_gemm_runs(gb):
    # continuous batching: a large native GEMM (n = 6144, ~0.37 s on the FP64
    # pipe) is on the device when 24 small requests arrive; they are admitted,
    # batched and finished while it still runs, and every result (the large one
    # too) equals the same request served alone, bit for bit
    import time
    import torch
    big = 6144
    reqs = _requests(24, 9200)  # host operands made first: generating them takes ~1 s
    srv = gb.Server(hbm_budget_bytes=2 << 30, n_streams=4, max_batch=8)
    big_out = np.empty((big, big))
    big_id = srv.submit(big, big, big, 1.0, 0.0, "native", 0, out=big_out, seed=9100)
    t0 = time.perf_counter()
    while srv.stats()["in_flight"] == 0 and time.perf_counter() - t0 < 10:
        time.sleep(0.001)
    assert srv.stats()["in_flight"] >= 1
    outs, ids = [], []
    for r in reqs:
        out = np.empty((r["m"], r["n"]))
        outs.append(out)
        ids.append(srv.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"],
                              r["slices"], A=r["A"], B=r["B"], C=r["C"], out=out))
    while not all(srv.poll(i)[0] for i in ids) and time.perf_counter() - t0 < 60:
        time.sleep(0.001)
    assert all(srv.poll(i)[0] for i in ids)
    # the small requests finished while the large GEMM was still on the device
    assert not srv.poll(big_id)[0]
    srv.drain(120)
    assert srv.poll(big_id)[0] and srv.poll(big_id)[1] == 0
    srv.close()
    for r, out in zip(reqs, outs):
        solo = gb.Server(hbm_budget_bytes=64 << 20, n_streams=1, max_batch=1)
        alone = np.empty((r["m"], r["n"]))
        solo.submit(r["m"], r["n"], r["k"], r["alpha"], r["beta"], r["precision"], r["slices"],
                    A=r["A"], B=r["B"], C=r["C"], out=alone)
        solo.drain(600)
        solo.close()
        assert np.array_equal(alone, out)
    solo = gb.Server(hbm_budget_bytes=2 << 30, n_streams=1, max_batch=1)
    alone = np.empty((big, big))
    solo.submit(big, big, big, 1.0, 0.0, "native", 0, out=alone, seed=9100)
    solo.drain(120)
    solo.close()
    assert np.array_equal(alone, big_out)
    # and the large result against the oracle on sampled rows
    rows = np.array([0, 1777, big - 1])
    A = g.matrix("uniform", big, big, 9100, 0, row_indices=rows)
    B = g.matrix("uniform", big, big, 9100, 1)
    ref = cgemm.dgemm(1.0, A, B)
    bound = exact.error_bound(big, 1.0, cgemm.dgemm(1.0, np.abs(A), np.abs(B)))
    assert np.all(np.abs(big_out[rows] - ref) <= 2 * bound)
    torch.cuda.synchronize()
