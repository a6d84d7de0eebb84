"""Benchmark of the FP64 GEMM C = A B (square, uniform[-1, 1], alpha = 1, beta = 0).

One step = one FP64-accurate GEMM at the configured n through the emulated path
(--path crt, the default: residues of A and of B, the residue products as BF16
GEMMs on the tensor cores, Chinese-remainder reconstruction and one FP64
rounding; --path e4m3: split of A, split of B, tensor-core slice products + FP64
recombination), the path whose result is checked against the FP64 error bound;
the native FP64 path
(the library's default kernel at that size) is timed beside it on the same
inputs.  Inputs (8 n^2 bytes each) are larger than the 129 MB L2 at the default
n, so no flush is needed.  At one GPU the same JSON line also carries, as
sub-records: the accuracy of both paths against a double-double reference on
sampled rows (`parity`), the same inputs through the emulated path the line does
not time (`other_path`: E4M3 digit slices beside the default residues) and the
BF16 digit format (`bf16_digits`), the 16-decade hard set at its slice count (`hard`),
the 2048-problem grouped workload against one launch per GEMM (`grouped`) and
two short serving runs, at the specified and at a sustainable arrival rate
(`serve`).  Other workloads print their own line (--workload).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 8192] [--slices 10]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU: independent replicas (no collective on the data path); value is the
sum over ranks of the work done divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
SMS = 152
SM_MAX_MHZ = 2070.0
# FP64 pipe of the GB300 SM: 2 FP64 FMA / clock / SM (4 flop), derived from the
# chip's unit counts and clocks; the DFMA kernels reach 99% of it.
FP64_FLOP_PER_CLK_SM = 4.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of the kernel as it is now:
# (kernel, n, slices) -> bytes.  Reported only for that exact workload.
MEASURED_TRAFFIC = {("emu_products_kernel", 8192, 10): int(9.80e9 + 559.31e6),
                    ("crt_products_kernel", 8192, 13): int(13.08e9 + 2.05e9)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--path", default="crt", choices=["crt", "e4m3"],
                   help="emulated path of the main line: residues modulo --moduli primes, or "
                        "--slices E4M3 digit slices (the other one is a sub-record)")
    p.add_argument("--moduli", type=int, default=13)
    p.add_argument("--slices", type=int, default=10)
    p.add_argument("--group-slices", type=int, default=11)
    p.add_argument("--native-steps", type=int, default=2)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--workload", default="dgemm",
                   choices=["dgemm", "grouped", "serve", "serve-sweep", "sweep", "d0", "daxpy"])
    p.add_argument("--rates", default="50,75,100,125,150,200",
                   help="arrival rates (requests/s) of --workload serve-sweep")
    p.add_argument("--sizes", default="1024,2048,4096,8192,10240")
    p.add_argument("--problems", type=int, default=2048)
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-rate", type=float, default=2000.0)
    p.add_argument("--serve-budget-gb", type=float, default=40.0)
    p.add_argument("--serve-streams", type=int, default=4)
    p.add_argument("--serve-batch", type=int, default=64)
    p.add_argument("--no-serve-baseline", action="store_true",
                   help="skip the one-GEMM-per-launch run of the same serving trace")
    p.add_argument("--hard-slices", type=int, default=11)
    p.add_argument("--hard-moduli", type=int, default=14)
    p.add_argument("--bf16-slices", type=int, default=7)
    p.add_argument("--sub-serve-seconds", type=float, default=10.0)
    p.add_argument("--no-sub-records", action="store_true",
                   help="default workload only: skip the hard, grouped and serving sub-records")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over all ranks (the slowest replica's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Whole-job throughput of independent replicas (weak scaling): the units all
    ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / (slowest_ms * 1e-3)


def cpu_baseline(n, seed, seconds, A=None, B=None):
    """The CPU oracle (plain C, OpenMP over rows) on a bounded sample of rows of
    the same GEMM; returns the baseline record and the computed rows."""
    import numpy as np
    from oracle import cgemm
    from synth import generators as g
    if A is None:
        A = g.matrix("uniform", n, n, seed, g.STREAM_A)
        B = g.matrix("uniform", n, n, seed, g.STREAM_B)
    threads = os.cpu_count() or 1
    rows = 4
    while True:
        sel = np.arange(rows, dtype=np.int64) * (n // rows)
        t0 = time.perf_counter()
        C, used = cgemm.dgemm_omp(1.0, np.ascontiguousarray(A[sel]), B, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.3 or rows >= n:
            break
        rows = min(n, max(rows * 2, int(rows * seconds * 0.4 / max(dt, 1e-3))))
    flops = 2.0 * rows * n * n
    rec = {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": used, "kind": "oracle",
           "sample": f"{rows} of {n} rows of C = A B (n = {n}), plain C oracle, "
                     f"{used} OpenMP threads, {dt:.2f} s"}
    return rec, sel, C


def dgemm_metric_config(n, world):
    """Metric name and config of the square-DGEMM workload, shared by both arms."""
    metric = "FP64-accurate GEMM TFLOP/s (emulated path; native FP64 beside it)"
    config = {"workload": f"square DGEMM C = A B, m = n = k = {n}, uniform[-1,1], "
                          f"alpha = 1, beta = 0 (sweep point n = {n})",
              "flush": "inputs larger than L2 (no flush needed)",
              "parallelism": f"replicas x{world}"}
    return metric, config


def gpu_path(kind, count):
    if kind == "crt":
        return (f"GPU: emulated FP64 by residues, b-bit integers modulo {count} primes as BF16 "
                "GEMMs on tcgen05 (FP32 sums of 256 K, exact), Chinese-remainder "
                "reconstruction, one FP64 rounding")
    return (f"GPU: emulated FP64, {count} E4M3 slices, tcgen05 FP32 accumulation, exact "
            "integer recombination, one FP64 rounding")


CPU_PATH = ("CPU oracle: plain C definition loops (-O2, no FMA contraction), OpenMP over "
            "rows, on a sample of rows of C")


def matrix_threads(kind, rows, cols, seed, sid, workers=None):
    """synth.generators.matrix built from row blocks on several threads (the
    values are a pure function of the element index, so blocks are independent)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from synth import generators as g
    workers = workers or min(16, os.cpu_count() or 1)
    out = np.empty((rows, cols), dtype=np.float64)
    step = -(-rows // (4 * workers))

    def block(r0):
        r1 = min(rows, r0 + step)
        out[r0:r1] = g.matrix(kind, rows, cols, seed, sid, row_indices=np.arange(r0, r1))
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(block, range(0, rows, step)))
    return out


def rho_rows(got_rows, A, B, rows, hilo=None):
    """max |C - C*| / bound over the given rows, C* the double-double value of A B
    (alpha = 1, beta = 0)."""
    import numpy as np
    from oracle import cgemm, exact
    hi, lo = hilo if hilo is not None else cgemm.dgemm_dd_rows(A, B, rows)
    bound = exact.error_bound(A.shape[1], 1.0, cgemm.dgemm_rows(rows, 1.0, np.abs(A), np.abs(B)))
    res = exact.residual(got_rows, 1.0, hi, lo)
    return float(np.max(np.abs(res) / bound))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synth import generators as g
    import numpy as np
    seed = g.BASE_SEED + 1
    n = args.n
    A = g.matrix("uniform", n, n, seed, g.STREAM_A)
    B = g.matrix("uniform", n, n, seed, g.STREAM_B)
    # size one step to ~a few seconds of oracle work
    rec, sel, _ = cpu_baseline(n, seed, 3.0, A, B)
    rows = len(sel)
    from oracle import cgemm
    for _ in range(args.warmup):
        cgemm.dgemm_omp(1.0, np.ascontiguousarray(A[sel]), B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cgemm.dgemm_omp(1.0, np.ascontiguousarray(A[sel]), B)
    dt = time.perf_counter() - t0
    value = 2.0 * rows * n * n * args.steps / dt / 1e12
    rec = dict(rec, value=value, sample=f"{rows} of {n} rows of C = A B per step "
                                         f"(n = {n}), plain C oracle")
    metric, config = dgemm_metric_config(n, args.gpus)
    out = {"impl": "reference", "path": CPU_PATH, "metric": metric, "value": value,
           "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded splitmix64, uniform[-1,1])",
           "config": config,
           "cpu_baseline": rec,
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _grouped_inputs(gb, torch, count, seed, precision, slices):
    """The group's operands: every A, every B and every C packed one after another
    (16-byte aligned) in three device arenas, so a caller can move all of them
    with one copy per arena."""
    from synth import generators as g
    ms, ns, ks = g.grouped_problems(seed, count)

    def offsets(sizes):
        offs, o = [], 0
        for z in sizes:
            offs.append(o)
            o += (int(z) + 1) // 2 * 2
        return offs, o
    offA, totA = offsets(ms * ks)
    offB, totB = offsets(ks * ns)
    offC, totC = offsets(ms * ns)
    arenas = {"A": torch.empty(totA, dtype=torch.float64, device="cuda"),
              "B": torch.empty(totB, dtype=torch.float64, device="cuda"),
              "C": torch.zeros(totC, dtype=torch.float64, device="cuda")}
    probs = []
    for i, (m, n, k) in enumerate(zip(ms, ns, ks)):
        m, n, k = int(m), int(n), int(k)
        A = arenas["A"][offA[i]:offA[i] + m * k].view(m, k)
        B = arenas["B"][offB[i]:offB[i] + k * n].view(k, n)
        C = arenas["C"][offC[i]:offC[i] + m * n].view(m, n)
        gb.fill_uniform(A, seed + i, 0)
        gb.fill_uniform(B, seed + i, 1)
        probs.append(dict(A=A, B=B, C=C, alpha=1.0, beta=0.0, precision=precision,
                          slices=slices))
    torch.cuda.synchronize()
    return probs, ms, ns, ks, arenas


def _time_stream(torch, fn, steps, warmup):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def grouped_measure(args, steps, warmup, baselines=True, e2e=True):
    """2048 independent GEMMs, m, n, k log-uniform in [16, 512]: one persistent
    launch in a CUDA graph, native and emulated, against one launch per GEMM.
    Returns the record (without printing)."""
    import numpy as np
    import torch

    import paper_1602_08477_gb300 as gb
    from paper_1602_08477_gb300 import autotune
    from synth import generators as g
    try:
        autotune.load()
        tuned = "shipped tuning table"
    except Exception:
        tuned = "size rule (no tuning table)"
    seed = g.BASE_SEED + 3
    # the smallest slice count at which every problem of this recipe meets the FP64
    # bound: the bound falls faster with k than the digit-truncation error, and at
    # s = 10 some problems with k < 32 exceed it
    s = args.group_slices
    probs, ms, ns, ks, arenas = _grouped_inputs(gb, torch, args.problems, seed, "native", s)
    flops = float(np.sum(2.0 * ms * ns * ks))
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    plan = gb.GroupedPlan(probs, use_graph=True)
    native_ms = _time_stream(torch, plan.run, steps, warmup)
    info = plan.info()
    per_ms = per_graph_ms = None
    if baselines:
        # one launch per GEMM, same kernels' default variants, uncaptured
        q = gb.default_queue()

        def per_gemm():
            for p in probs:
                gb.dgemm(p["A"], p["B"], p["C"], 1.0, 0.0, kernel="auto", queue=q)
        per_ms = _time_stream(torch, per_gemm, max(1, steps // 2), 1)
        # one launch per GEMM, captured in a CUDA graph
        cap_stream = torch.cuda.Stream()
        cap_q = gb.Queue(gb.Device(0), cap_stream)
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap_stream):
            for p in probs:
                gb.dgemm(p["A"], p["B"], p["C"], 1.0, 0.0, kernel="auto", queue=cap_q)
        per_graph_ms = _time_stream(torch, graph.replay, steps, 1)
    # emulated group (same problems)
    eprobs = [dict(p, precision="emulated", C=torch.zeros_like(p["C"])) for p in probs]
    eplan = gb.GroupedPlan(eprobs, use_graph=True)
    emu_ms = _time_stream(torch, eplan.run, steps, warmup)
    einfo = eplan.info()
    # the same emulated group with each problem's slice count left to the tuning
    # table (slices = 0), and its error against the group at 16 slices relative to
    # the FP64 bound 2 (k + 2) u (|A||B|), |A||B| from the library's native GEMMs
    tprobs = [dict(p, slices=0, C=torch.zeros_like(p["C"])) for p in eprobs]
    tplan = gb.GroupedPlan(tprobs, use_graph=True)
    tuned_ms = _time_stream(torch, tplan.run, steps, warmup)
    tinfo = tplan.info()
    tplan.close()
    rprobs = [dict(p, slices=16, C=torch.zeros_like(p["C"])) for p in eprobs]
    gb.dgemm_grouped(rprobs)
    torch.cuda.synchronize()
    u = 2.0 ** -53
    rho_t = rho_f = 0.0
    for p, fp, r, k in zip(tprobs, eprobs, rprobs, ks):
        bound = 2.0 * (int(k) + 2) * u * gb.dgemm(p["A"].abs(), p["B"].abs())
        rho_t = max(rho_t, float(((p["C"] - r["C"]).abs() / bound).max()))
        rho_f = max(rho_f, float(((fp["C"] - r["C"]).abs() / bound).max()))
    del rprobs
    counts = {}
    for m, n, k in zip(ms, ns, ks):
        c = gb.tune_lookup_slices(int(m), int(n), int(k))
        counts[c] = counts.get(c, 0) + 1
    rules = None
    if baselines and tuned == "shipped tuning table":
        # the same groups with the tuning table emptied: the native size rule and
        # the emulated padding rule choose every tile
        gb.tune_set([])
        try:
            rplan = gb.GroupedPlan(probs, use_graph=True)
            rn_ms = _time_stream(torch, rplan.run, steps, warmup)
            rplan.close()
            reprobs = [dict(p, C=torch.zeros_like(p["C"])) for p in eprobs]
            replan = gb.GroupedPlan(reprobs, use_graph=True)
            re_ms = _time_stream(torch, replan.run, steps, warmup)
            re_tiles = replan.info()["emulated_tiles"]
            replan.close()
        finally:
            autotune.load()
        rules = {"native_ms": round(rn_ms, 3), "native_tflops": round(flops / rn_ms / 1e9, 4),
                 "emulated_ms": round(re_ms, 3),
                 "emulated_tflops_fp64_equiv": round(flops / re_ms / 1e9, 3),
                 "emulated_tiles": re_tiles,
                 "note": "tuning table emptied: native size rule, emulated padding rule"}
    clk = clocks.stop()
    pk, pk_kind = peaks()
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    value = flops / (native_ms * 1e-3) / 1e12
    emu_tf = flops / (emu_ms * 1e-3) / 1e12
    pair_flops = s * (s + 1) / 2 * flops
    out = {
        "metric": "grouped FP64 GEMM TFLOP/s (one persistent launch in a CUDA graph)",
        "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": round(native_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (device splitmix64, uniform[-1,1])",
        "config": {"workload": f"{args.problems} independent GEMMs, m, n, k log-uniform in "
                               "[16, 512], alpha = 1, beta = 0", "tiles": tuned,
                   "flush": "none: operands (~1 GB) larger than L2"},
        "gpu_launches": info["launches"] * steps,
        "roofline": {"bound": "alu", "kernel": "grouped_native_kernel",
                     "achieved": round(value, 4), "peak": round(fp64_peak, 4),
                     "unit": "TFLOP/s", "frac": round(value / fp64_peak, 4),
                     "peak_kind": "derived: 152 SM x 4 flop/clk x 2070 MHz",
                     "algorithmic": f"sum 2mnk = {flops:.4g} flop per launch"},
        "emulated": {"slices": s, "ms": round(emu_ms, 3), "tflops_fp64_equiv": round(emu_tf, 3),
                     "tensor_frac": round(pair_flops / (emu_ms * 1e-3) / 1e12 /
                                          (2.0 * pk["bf16_tflops"]), 4),
                     "launches": einfo["launches"], "rho_max_vs_s16": rho_f},
        "emulated_tuned_slices": {
            "slices": "per problem from the tuning table (slices = 0)",
            "problems_per_slice_count": {str(c): v for c, v in sorted(counts.items())},
            "ms": round(tuned_ms, 3), "tflops_fp64_equiv": round(flops / tuned_ms / 1e9, 3),
            "launches": tinfo["launches"], "tiles": tinfo["emulated_tiles"],
            "rho_max_vs_s16": rho_t,
            "note": "rho = max |C - C_16| / (2 (k+2) u |A||B|) over all outputs, C_16 the "
                    "same group at 16 slices"},
        "tiles": {"native": info["native_tiles"], "emulated": einfo["emulated_tiles"]},
        "e2e": None, "clocks": clk,
    }
    if rules is not None:
        out["untuned_rules"] = rules
    if baselines:
        out["one_launch_per_gemm"] = {
            "ms": round(per_ms, 3), "tflops": round(flops / per_ms / 1e9, 4),
            "graph_ms": round(per_graph_ms, 3),
            "graph_tflops": round(flops / per_graph_ms / 1e9, 4), "launches": args.problems}
    if e2e:
        # end to end: the packed operands from pinned host memory (one copy per
        # arena), the graph-captured group, the packed results back
        hostA = arenas["A"].cpu().pin_memory()
        hostB = arenas["B"].cpu().pin_memory()
        hostC = torch.empty(arenas["C"].shape, dtype=torch.float64).pin_memory()
        h2d = (hostA.numel() + hostB.numel()) * 8
        d2h = hostC.numel() * 8

        def e2e_step():
            arenas["A"].copy_(hostA, non_blocking=True)
            arenas["B"].copy_(hostB, non_blocking=True)
            plan.run()
            hostC.copy_(arenas["C"], non_blocking=True)
        e2e_ms = _time_stream(torch, e2e_step, max(1, steps // 2), 1)
        out["e2e"] = {"value": round(flops / e2e_ms / 1e9, 4), "unit": "TFLOP/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    plan.close()
    eplan.close()
    del probs, eprobs, arenas
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def run_grouped(args):
    """The grouped workload alone (its own JSON line)."""
    import torch

    import paper_1602_08477_gb300 as gb
    torch.cuda.set_device(0)
    gb.build()
    print(json.dumps(grouped_measure(args, args.steps, args.warmup)), flush=True)
    return 0


def _serve_trace(args, gb, g, np, max_batch, policy="lanes"):
    """One run of the arrival trace through a server with batches of at most
    `max_batch` requests under `policy` ("fifo" with max_batch = 1: every GEMM
    its own launch, in arrival order).  Returns the stats."""
    seed = g.BASE_SEED + 4
    count = int(args.serve_rate * args.serve_seconds * 1.2) + 16
    gaps = g.poisson_gaps_ms(seed, count, args.serve_rate) * 1e-3
    arrivals = np.cumsum(gaps)
    sizes = g.log_uniform_ints(seed, 21, count, 64, 4096)
    emulated = (g.raw_stream(seed, 22, count) % np.uint64(5)) == 0
    s = SERVE_SLICES
    srv = gb.Server(int(args.serve_budget_gb * 2 ** 30), n_streams=args.serve_streams,
                    max_batch=max_batch, policy=policy)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    submitted, offered = 0, 0.0
    ids = []
    queue_trace = []  # (seconds, queued, on the device) every half second
    next_sample = 0.0
    for i in range(count):
        t = arrivals[i]
        if t > args.serve_seconds:
            break
        now = time.perf_counter() - t0
        if now >= next_sample:
            q = srv.stats()
            queue_trace.append((round(now, 2), int(q["pending"]), int(q["in_flight"])))
            next_sample += 0.5
        if t > now:
            time.sleep(t - now)
        n = int(sizes[i])
        prec = "emulated" if emulated[i] else "native"
        ids.append((srv.submit(n, n, n, 1.0, 0.0, prec, s, seed=seed * 1000003 + i), n, prec))
        submitted += 1
        offered += 2.0 * n ** 3
    wall = time.perf_counter() - t0
    st = srv.stats()
    clk = clocks.stop()
    done_native = done_emu = 0.0
    lane_lat = {"small": [], "large": []}
    lane_count = {"small": 0, "large": 0}
    arrival_lat = []  # (arrival second, latency ms or None when not completed)
    for idx, (rid, n, prec) in enumerate(ids):
        done, status, lat = srv.poll(rid)
        arrival_lat.append((float(arrivals[idx]), lat if done and status == 0 else None))
        lane = "large" if prec == "native" and 2.0 * n ** 3 >= 2.0 ** 31 else "small"
        lane_count[lane] += 1
        if done and status == 0:
            lane_lat[lane].append(lat)
            if prec == "native":
                done_native += 2.0 * n ** 3
            else:
                done_emu += 2.0 * n ** 3
    srv.close()
    pk, _ = peaks()
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6
    fp8_peak = 2.0 * pk["bf16_tflops"] * 1e12
    # roofline time of the work completed: native flops on the FP64 pipe, emulated
    # pair products on the FP8 tensor pipe
    bound_s = done_native / fp64_peak + done_emu * s * (s + 1) / 2 / fp8_peak
    st["roofline_frac"] = bound_s / max(st["busy_s"], 1e-9)
    st["offered_tflops"] = offered / max(wall, 1e-9) / 1e12
    st["submit_wall_s"] = wall
    st["clocks"] = clk
    st["submitted_here"] = submitted
    st["queue_trace"] = queue_trace
    st["arrival_lat"] = arrival_lat
    # latency per class of request (the lanes' rule: native and 2 n^3 >= 2^31 is
    # large), completed requests only, with how many of the class were submitted
    st["by_class"] = {
        c: {"submitted": lane_count[c], "completed": len(v),
            "p50_ms": round(float(np.percentile(v, 50)), 3) if v else None,
            "p99_ms": round(float(np.percentile(v, 99)), 3) if v else None}
        for c, v in lane_lat.items()}
    return st


def _serve_summary(st):
    return {"p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
            "max_ms": round(st["max_ms"], 3), "tflops": round(st["tflops"], 4),
            "submitted": st["submitted"], "completed": st["completed"],
            "pending_at_end": st["pending"], "in_flight_at_end": st["in_flight"],
            "max_queue": st["max_queue"], "batches": st["batches"],
            "mean_batch": round(st["mean_batch"], 2), "large_launches": st["large_launches"],
            "peak_arena_gb": round(st["peak_bytes"] / 2 ** 30, 3),
            "roofline_frac": round(st["roofline_frac"], 4), "by_class": st["by_class"]}


SERVE_SLICES = 12


def serve_warm(args, gb, s):
    """Warm the serving kernels on a few small requests (not counted)."""
    srv = gb.Server(int(args.serve_budget_gb * 2 ** 30), n_streams=args.serve_streams,
                    max_batch=args.serve_batch)
    for i in range(4):
        srv.submit(64, 64, 64, precision="emulated" if i % 2 else "native", slices=s, seed=i)
    srv.drain(60)
    srv.close()


def serve_record(args, gb, g, np, rate, seconds):
    """A short run of the serving trace at `rate` requests/s: the summary."""
    a = argparse.Namespace(**vars(args))
    a.serve_rate, a.serve_seconds = rate, seconds
    st = _serve_trace(a, gb, g, np, args.serve_batch)
    out = _serve_summary(st)
    out["rate_per_s"] = rate
    out["seconds"] = seconds
    out["offered_tflops"] = round(st["offered_tflops"], 3)
    out["clocks"] = st["clocks"]
    out.update(stability(st, seconds))
    return out


def run_serve(args):
    """Poisson arrivals of square GEMMs, n log-uniform in [64, 4096], 20% emulated,
    HBM-budget admission, continuous batching; p50/p99 latency and TFLOP/s, beside
    the same trace served one GEMM per launch."""
    import numpy as np
    import torch

    import paper_1602_08477_gb300 as gb
    from paper_1602_08477_gb300 import autotune
    from synth import generators as g
    torch.cuda.set_device(0)
    gb.build()
    try:
        autotune.load()
    except Exception:
        pass
    s = SERVE_SLICES
    serve_warm(args, gb, s)
    st = _serve_trace(args, gb, g, np, args.serve_batch)
    single = None if args.no_serve_baseline else _serve_trace(args, gb, g, np, 1, "fifo")
    serve = _serve_summary(st)
    serve["offered_tflops"] = round(st["offered_tflops"], 3)
    serve["submit_wall_s"] = round(st["submit_wall_s"], 2)
    # queue length over time: [seconds, queued, on the device] at up to 21 points
    tr = st["queue_trace"]
    pick = sorted(set(np.linspace(0, len(tr) - 1, min(21, len(tr))).astype(int).tolist())) if tr else []
    serve["queue_over_time"] = [list(tr[i]) for i in pick]
    out = {
        "metric": "serving FP64 GEMM p50/p99 latency (ms) and TFLOP/s",
        "value": round(st["tflops"], 4), "unit": "TFLOP/s", "n_gpus": 1,
        "steps": int(st["submitted_here"]), "warmup": 4, "ms_per_step": round(st["mean_ms"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (device splitmix64 per request seed, uniform[-1,1])",
        "config": {"workload": f"Poisson arrivals {args.serve_rate:g}/s for "
                               f"{args.serve_seconds:g} s, square n log-uniform in [64, 4096], "
                               f"20% emulated (s = {s}), {args.serve_budget_gb:g} GB budget",
                   "streams": args.serve_streams, "max_batch": args.serve_batch,
                   "policy": "lanes: native >= 2^31 flops alone on low-priority streams, "
                             "the rest batched on high-priority streams"},
        "serve": serve,
        "roofline": {"bound": "mixed", "frac": round(st["roofline_frac"], 4),
                     "note": "roofline time of the completed work (native on the FP64 pipe, "
                             "emulated pair products on the FP8 tensor pipe) / busy time"},
        "gpu_launches": int(st["batches"]) * 5,
        "e2e": {"value": round(st["tflops"], 4), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0, "note": "operands generated on the device per request"},
        "clocks": st["clocks"],
    }
    if single is not None:
        out["one_launch_per_gemm"] = dict(_serve_summary(single),
                                          note="same arrival trace, one queue in arrival "
                                               "order, every GEMM its own grouped launch")
    print(json.dumps(out), flush=True)
    return 0


def stability(st, seconds):
    """p99 latency of the requests that arrived in the first and in the second
    half of the run (a request still unfinished at the end counts as waiting
    until the end), and whether the run was sustainable: every request finished
    and p99 did not grow from the first half to the second by more than half."""
    import numpy as np
    halves = ([], [])
    unfinished = 0
    for t, lat in st["arrival_lat"]:
        if lat is None:
            unfinished += 1
            lat = (seconds - t) * 1e3
        halves[0 if t < seconds / 2 else 1].append(lat)
    p99 = [float(np.percentile(h, 99)) if h else None for h in halves]
    ok = unfinished == 0 and p99[0] is not None and p99[1] is not None and p99[1] <= 1.5 * p99[0]
    return {"p99_first_half_ms": round(p99[0], 2) if p99[0] is not None else None,
            "p99_second_half_ms": round(p99[1], 2) if p99[1] is not None else None,
            "unfinished": unfinished, "sustainable": bool(ok)}


def run_serve_sweep(args):
    """Serving at increasing Poisson arrival rates (--rates, --serve-seconds each,
    the specified size and precision mix): p50/p99, TFLOP/s and whether p99 stays
    flat over the run; the highest rate that does is the sustainable rate."""
    import numpy as np
    import torch

    import paper_1602_08477_gb300 as gb
    from paper_1602_08477_gb300 import autotune
    from synth import generators as g
    torch.cuda.set_device(0)
    gb.build()
    try:
        autotune.load()
    except Exception:
        pass
    serve_warm(args, gb, SERVE_SLICES)
    res = []
    for rate in (float(x) for x in args.rates.split(",")):
        a = argparse.Namespace(**vars(args))
        a.serve_rate = rate
        st = _serve_trace(a, gb, g, np, args.serve_batch)
        rec = dict(_serve_summary(st), rate_per_s=rate, offered_tflops=round(st["offered_tflops"], 3),
                   clocks=st["clocks"])
        rec.update(stability(st, args.serve_seconds))
        res.append(rec)
    ok = [r["rate_per_s"] for r in res if r["sustainable"]]
    print(json.dumps({"metric": "serving p50/p99 latency (ms) and TFLOP/s per arrival rate",
                      "unit": "ms", "seconds_per_rate": args.serve_seconds,
                      "config": {"workload": "Poisson arrivals, square n log-uniform in [64, 4096], "
                                             f"20% emulated (s = {SERVE_SLICES}), "
                                             f"{args.serve_budget_gb:g} GB budget",
                                 "streams": args.serve_streams, "max_batch": args.serve_batch},
                      "highest_sustainable_rate_per_s": max(ok) if ok else None,
                      "rates": res}), flush=True)
    return 0


def run_sweep(args):
    """Native square DGEMM sweep n in {1024, ..., 10240}: naive vs tiled vs DFMA vs
    DMMA kernels, TFLOP/s and fraction of the FP64 peak; the vendor library's FP64
    GEMM (cuBLAS via torch.matmul) beside them as context, and the two emulated
    paths (FP64-accurate: --slices E4M3 digit slices, --moduli residues) at the same
    sizes."""
    import torch

    import paper_1602_08477_gb300 as gb
    torch.cuda.set_device(0)
    gb.build()
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    res = []
    for n in (int(x) for x in args.sizes.split(",")):
        A = torch.empty((n, n), dtype=torch.float64, device="cuda")
        B = torch.empty((n, n), dtype=torch.float64, device="cuda")
        C = torch.empty((n, n), dtype=torch.float64, device="cuda")
        gb.fill_uniform(A, 1602084771, 0)
        gb.fill_uniform(B, 1602084771, 1)
        ws = gb.alloc_workspace(gb.workspace_size("emulated", args.slices, n, n, n))
        ws_crt = gb.alloc_workspace(gb.workspace_size("emulated_crt", args.moduli, n, n, n))
        for kernel in ("naive", "tiled", "dfma", "dmma", "cublas", "emulated", "emulated_crt"):
            if kernel == "cublas":
                # context only: the vendor library's FP64 GEMM through torch.matmul
                f = lambda: torch.matmul(A, B, out=C)
            elif kernel == "emulated":
                # the FP64-accurate split-precision path at the bench's slice count
                f = lambda: gb.dgemm(A, B, C, precision="emulated", slices=args.slices,
                                     workspace=ws)
            elif kernel == "emulated_crt":
                # the FP64-accurate residue path at the bench's number of moduli
                f = lambda: gb.dgemm(A, B, C, precision="emulated_crt", slices=args.moduli,
                                     workspace=ws_crt)
            else:
                f = lambda: gb.dgemm(A, B, C, kernel=kernel)
            steps = 10 if kernel.startswith("emulated") else (1 if n >= 4096 else 3)
            ms = _time_stream(torch, f, steps, 1)
            tf = 2.0 * n ** 3 / ms / 1e9
            res.append(dict(n=n, kernel=kernel, ms=round(ms, 3), tflops=round(tf, 4),
                            frac_fp64_peak=round(tf / fp64_peak, 4)))
        del A, B, C, ws, ws_crt
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "native FP64 DGEMM TFLOP/s per kernel", "unit": "TFLOP/s",
                      "peak": round(fp64_peak, 4), "sweep": res}), flush=True)
    return 0


def run_d0(args):
    """C = 1.5 A B + 0.5 C at n = 256 (uniform[-1, 1]): device microseconds and
    TFLOP/s per call for each kernel, and the host cost of one C-ABI call
    (validation + launch, through the Python binding) next to the host cost of
    one minimal torch kernel launch, the zero-overhead comparison of the paper
    transposed to this library."""
    import numpy as np
    import torch

    import paper_1602_08477_gb300 as gb
    from synth import generators as g
    torch.cuda.set_device(0)
    gb.build()
    n = 256
    seed = g.BASE_SEED
    A = torch.from_numpy(g.matrix("uniform", n, n, seed, g.STREAM_A)).cuda()
    B = torch.from_numpy(g.matrix("uniform", n, n, seed, g.STREAM_B)).cuda()
    C0 = torch.from_numpy(g.matrix("uniform", n, n, seed, g.STREAM_C)).cuda()
    C = C0.clone()
    q = gb.default_queue()
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    flops = 2.0 * n ** 3
    calls = 200
    res = {}
    for kernel in ("auto", "naive", "tiled", "dfma", "dmma", "emulated"):
        if kernel == "emulated":
            ws = gb.alloc_workspace(gb.workspace_size("emulated", 11, n, n, n))
            f = lambda: gb.dgemm(A, B, C, 1.5, 0.5, precision="emulated", slices=11, queue=q,
                                 workspace=ws)
        else:
            f = (lambda kk: (lambda: gb.dgemm(A, B, C, 1.5, 0.5, kernel=kk, queue=q)))(kernel)
        ms = _time_stream(torch, f, calls, 10)
        res[kernel] = {"us_per_call": round(ms * 1e3, 2),
                       "tflops": round(flops / ms / 1e9, 4),
                       "frac_fp64_peak": round(flops / ms / 1e9 / fp64_peak, 4)}
    # host cost per call through the C ABI (ctypes, prebuilt arguments): gb_dgemm
    # (validation, variant resolution, launch) against a raw launch of the same
    # tiled kernel by the generic executor; few enough calls that the launch
    # queue never fills, so the host is never throttled by the GPU
    import ctypes
    lib = gb.load()
    P = ctypes.c_void_p
    dargs = (q.handle, None, 2, 0, 0, n, n, n, 1.5, P(A.data_ptr()), n, P(B.data_ptr()), n, 0.5,
             P(C.data_ptr()), n, None, 0)
    kt = gb.kernel_handle("dgemm_tiled16")
    vals = [ctypes.c_int64(n), ctypes.c_int64(n), ctypes.c_int64(n), ctypes.c_double(1.5),
            P(A.data_ptr()), ctypes.c_int64(n), P(B.data_ptr()), ctypes.c_int64(n),
            ctypes.c_double(0.5), P(C.data_ptr()), ctypes.c_int64(n)]
    argv = (P * len(vals))(*[ctypes.cast(ctypes.pointer(v), P) for v in vals])
    wd = gb.Workdiv.make([n // 16, n // 16], [16, 16], [1, 1])

    def host_us(fn, reps=150):
        best = 1e9
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            t1 = time.perf_counter()
            torch.cuda.synchronize()
            best = min(best, (t1 - t0) / reps * 1e6)
        return best

    api_us = host_us(lambda: lib.gb_dgemm(*dargs))
    raw_us = host_us(lambda: lib.gb_enqueue(q.handle, ctypes.byref(wd), P(kt), argv, 0))
    dev_raw = _time_stream(torch, lambda: lib.gb_enqueue(q.handle, ctypes.byref(wd), P(kt), argv, 0),
                           calls, 10)
    out = {
        "metric": "DGEMM C = 1.5 A B + 0.5 C at n = 256: device us per call, TFLOP/s",
        "unit": "us", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
        "data": "synthetic (seeded splitmix64, uniform[-1,1])",
        "config": {"workload": "square DGEMM n = 256, alpha = 1.5, beta = 0.5"},
        "kernels": res,
        "api_vs_raw_launch": {
            "host_us_gb_dgemm": round(api_us, 3), "host_us_raw_launch": round(raw_us, 3),
            "host_overhead_us": round(api_us - raw_us, 3),
            "device_us_gb_dgemm_tiled": res["tiled"]["us_per_call"],
            "device_us_raw_launch_tiled": round(dev_raw * 1e3, 2),
            "note": "same tiled kernel; raw = gb_enqueue with a prebuilt work division"},
    }
    print(json.dumps(out), flush=True)
    return 0


def run_daxpy(args):
    """DAXPY y <- alpha x + y (Section 4.1) over 2^28 doubles per vector (2 GiB,
    far larger than L2): HBM GB/s against the measured copy bandwidth, for the
    library's work division and explicit ones."""
    import torch

    import paper_1602_08477_gb300 as gb
    torch.cuda.set_device(0)
    gb.build()
    n = 1 << 28
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    gb.fill_uniform(x.view(1 << 14, 1 << 14), 1602084777, 0)
    gb.fill_uniform(y.view(1 << 14, 1 << 14), 1602084777, 1)
    pk, pk_kind = peaks()
    res = {}
    for name, (B, V) in {"default": (256, 4), "B128_V8": (128, 8), "B512_V2": (512, 2),
                         "B1024_V1": (1024, 1)}.items():
        wd = gb.Workdiv.make([-(-n // (B * V))], [B], [V])
        ms = _time_stream(torch, lambda: gb.daxpy(1.0000001, x, y, workdiv=wd), args.steps,
                          args.warmup)
        gbs = 24.0 * n / (ms * 1e-3) / 1e9
        res[name] = {"ms": round(ms, 4), "GBps": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}
    best = max(res.values(), key=lambda r: r["GBps"])
    out = {"metric": "DAXPY HBM bandwidth", "value": best["GBps"], "unit": "GB/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"],
           "higher_is_better": True, "dtype": "f64", "data": "synthetic (device splitmix64)",
           "config": {"workload": "DAXPY n = 2^28, 24 bytes per element (read x, y; write y)",
                      "flush": "vectors larger than L2"},
           "roofline": {"bound": "hbm", "achieved": best["GBps"], "peak": pk["hbm_gbs"],
                        "unit": "GB/s", "frac": best["frac"], "peak_kind": f"{pk_kind} copy"},
           "workdivs": res}
    print(json.dumps(out), flush=True)
    return 0


def hard_record(args, gb, g, np, torch, A, B, C, q):
    """The 16-decade hard set at n through the main line's emulated path with the
    count it needs there (--hard-moduli residues, or --hard-slices E4M3 slices), the
    whole path per step; rho of both paths against the double-double reference on
    sampled rows."""
    n, s = args.n, args.hard_slices
    prec = "emulated_crt" if args.path == "crt" else "emulated"
    if args.path == "crt":
        s = args.hard_moduli
    seed = g.BASE_SEED + 3
    A_h = matrix_threads("hard", n, n, seed, g.STREAM_A)
    B_h = matrix_threads("hard", n, n, seed, g.STREAM_B)
    A.copy_(torch.from_numpy(A_h))
    B.copy_(torch.from_numpy(B_h))
    ws = gb.alloc_workspace(gb.workspace_size(prec, s, n, n, n))
    clocks = ClockSampler(0)
    clocks.start()
    step = lambda: gb.dgemm(A, B, C, precision=prec, slices=s, queue=q, workspace=ws)
    ms = _time_stream(torch, step, 5, 2)
    clk = clocks.stop()
    q.wait()
    rows = np.random.default_rng(n + s).choice(n, 4, replace=False)
    got_e = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    Cn = torch.zeros_like(C)
    gb.dgemm(A, B, Cn, 1.0, 0.0, kernel="auto", queue=q)
    got_n = Cn[torch.from_numpy(rows).cuda()].cpu().numpy()
    from oracle import cgemm
    hilo = cgemm.dgemm_dd_rows(A_h, B_h, rows)
    del ws, Cn
    torch.cuda.empty_cache()
    return {"workload": f"square DGEMM C = A B, n = {n}, entries +-(1+f) 2^E with E uniform in "
                        "[-27, 26] (16 decades), random signs",
            "path": prec, "slices" if prec == "emulated" else "moduli": s,
            "ms_per_step": round(ms, 3),
            "tflops": round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 3),
            "rho_emulated": rho_rows(got_e, A_h, B_h, rows, hilo),
            "rho_native": rho_rows(got_n, A_h, B_h, rows, hilo),
            "rows_checked": len(rows), "steps": 5, "warmup": 2, "clocks": clk}


def other_path_record(args, gb, np, torch, A, B, C, q, A_h, B_h):
    """The main line's inputs through the emulated path it does not time: the E4M3
    digit slices beside residues, or the other way round; whole path per step,
    its dominant kernel's time and rho against the double-double reference."""
    n = args.n
    crt = args.path != "crt"  # the other path
    N, s = args.moduli, args.slices
    ws = gb.alloc_workspace(gb.workspace_size("emulated_crt", N, n, n, n) if crt
                            else gb.workspace_size("emulated", s, n, n, n))
    stream = torch.cuda.current_stream()

    def run(ev=None):
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("split_a", "split_b"))
        else:
            gb.emulated_steps(A, B, C, 1.0, 0.0, s, ws, queue=q, steps=("split_a", "split_b"))
        if ev is not None:
            ev[0].record(stream)
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("products",))
        else:
            gb.emulated_steps(A, B, C, 1.0, 0.0, s, ws, queue=q, steps=("products",))
        if ev is not None:
            ev[1].record(stream)
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("combine",))

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(5)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for e in evs:
        run(e)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / 5
    prod_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    q.wait()
    rows = np.random.default_rng(n + 7).choice(n, 4, replace=False)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    from oracle import cgemm
    hilo = cgemm.dgemm_dd_rows(A_h, B_h, rows)
    del ws
    torch.cuda.empty_cache()
    pk, pk_kind = peaks()
    flops = 2.0 * n ** 3
    if crt:
        work, peak, kernel = N * flops, pk["bf16_tflops"], "crt_products_kernel"
        desc = f"{N} moduli (residues, BF16 GEMMs)"
    else:
        work, peak, kernel = s * (s + 1) / 2 * flops, 2.0 * pk["bf16_tflops"], "emu_products_kernel"
        desc = f"{s} E4M3 digit slices"
    achieved = work / (prod_ms * 1e-3) / 1e12
    return {"path": desc, "ms_per_step": round(ms, 3),
            "tflops": round(flops / (ms * 1e-3) / 1e12, 3),
            "products": {"kernel": kernel, "launch_ms": round(prod_ms, 3),
                         "achieved": round(achieved, 1), "peak": round(peak, 1),
                         "frac": round(achieved / peak, 4)},
            "rho_emulated": rho_rows(got, A_h, B_h, rows, hilo), "rows_checked": len(rows),
            "steps": 5, "warmup": 2}


def bf16_record(args, gb, np, torch, A, B, C, q, A_h, B_h):
    """The same uniform GEMM through the second digit format (8-bit digits in
    BF16, kind::f16 MMAs) at the slice count that meets the FP64 bound there
    (--bf16-slices), the whole path per step; rho against the double-double
    reference on sampled rows."""
    n, s = args.n, args.bf16_slices
    ws = gb.alloc_workspace(gb.workspace_size("emulated_bf16", s, n, n, n))
    clocks = ClockSampler(0)
    clocks.start()
    step = lambda: gb.dgemm(A, B, C, precision="emulated_bf16", slices=s, queue=q, workspace=ws)
    ms = _time_stream(torch, step, 5, 2)
    clk = clocks.stop()
    q.wait()
    rows = np.random.default_rng(n + 100 * s).choice(n, 4, replace=False)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    from oracle import cgemm
    hilo = cgemm.dgemm_dd_rows(A_h, B_h, rows)
    del ws
    torch.cuda.empty_cache()
    pairs = s * (s + 1) / 2 * 2.0 * n ** 3
    return {"workload": f"square DGEMM C = A B, n = {n}, uniform[-1,1] (the main line's inputs)",
            "digits": "8-bit signed digits in BF16, kind::f16 MMAs, FP32 level sums read out "
                      "every 1024 / s K indices",
            "slices": s, "ms_per_step": round(ms, 3),
            "tflops": round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 3),
            "bf16_pair_tflops_whole_path": round(pairs / (ms * 1e-3) / 1e12, 1),
            "rho_emulated": rho_rows(got, A_h, B_h, rows, hilo),
            "rows_checked": len(rows), "steps": 5, "warmup": 2, "clocks": clk}


def grouped_sub_record(args):
    """The grouped workload, summarised for the default line."""
    r = grouped_measure(args, 5, 2, baselines=True, e2e=False)
    return {"workload": r["config"]["workload"], "tiles": r["config"]["tiles"],
            "native_tflops": r["value"], "native_ms": r["ms_per_step"],
            "native_frac_fp64_peak": r["roofline"]["frac"],
            "emulated": r["emulated"], "emulated_tuned_slices": r["emulated_tuned_slices"],
            "one_launch_per_gemm": r["one_launch_per_gemm"],
            "untuned_rules": r.get("untuned_rules"),
            "launches_per_step": r["gpu_launches"] // 5, "clocks": r["clocks"]}


SUSTAINABLE_RATE = 100.0


def serve_sub_record(args, gb, g, np):
    """Two short serving runs: the specified 2000 requests/s (overloaded: large
    native requests queue without bound) and a rate the GPU sustains."""
    serve_warm(args, gb, SERVE_SLICES)
    out = {"workload": "Poisson arrivals, square n log-uniform in [64, 4096], 20% emulated "
                       f"(s = {SERVE_SLICES}), {args.serve_budget_gb:g} GB budget, "
                       f"{args.serve_streams} streams, batches of <= {args.serve_batch}"}
    out["specified_rate"] = serve_record(args, gb, g, np, args.serve_rate, args.sub_serve_seconds)
    out["sustainable_rate"] = serve_record(args, gb, g, np, SUSTAINABLE_RATE,
                                           args.sub_serve_seconds)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "grouped":
        return run_grouped(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "serve-sweep":
        return run_serve_sweep(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "d0":
        return run_d0(args)
    if args.workload == "daxpy":
        return run_daxpy(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1602_08477_gb300 as gb
    from synth import generators as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    gb.build()
    dev = gb.Device(local)
    stream = torch.cuda.current_stream()
    q = gb.Queue(dev, stream)

    def barrier():
        if world > 1:
            dist.barrier()

    def slowest(x):
        return max_over_ranks(x, world)

    n, s = args.n, args.slices
    N = args.moduli
    crt = args.path == "crt"
    seed = g.BASE_SEED + 1
    A_h = matrix_threads("uniform", n, n, seed, g.STREAM_A)
    B_h = matrix_threads("uniform", n, n, seed, g.STREAM_B)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    ws = gb.alloc_workspace(gb.workspace_size("emulated_crt", N, n, n, n) if crt
                            else gb.workspace_size("emulated", s, n, n, n))
    flops = 2.0 * n * n * n
    # the dominant kernel's algorithmic work per launch: the residue products (N BF16
    # GEMMs of the whole K) or the slice-pair products (s (s+1) / 2 FP8 GEMMs)
    pair_flops = N * flops if crt else s * (s + 1) / 2 * flops

    def step(ev=None):
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("split_a", "split_b"))
        else:
            gb.emulated_steps(A, B, C, 1.0, 0.0, s, ws, queue=q, steps=("split_a", "split_b"))
        if ev is not None:
            ev[0].record(stream)
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("products",))
        else:
            gb.emulated_steps(A, B, C, 1.0, 0.0, s, ws, queue=q, steps=("products",))
        if ev is not None:
            ev[1].record(stream)
        if crt:
            gb.emulated_crt_steps(A, B, C, 1.0, 0.0, N, ws, queue=q, steps=("combine",))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    q.wait()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = slowest(t0.elapsed_time(t1))
    prod_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    q.wait()
    emu_C = C.clone()
    del ws
    torch.cuda.empty_cache()

    # native FP64 leg on the same inputs (the library's default kernel at this size)
    Cn = torch.zeros_like(C)
    gb.dgemm(A, B, Cn, 1.0, 0.0, kernel="auto", queue=q)
    torch.cuda.synchronize()
    n0 = torch.cuda.Event(enable_timing=True)
    n1 = torch.cuda.Event(enable_timing=True)
    n0.record(stream)
    for _ in range(args.native_steps):
        gb.dgemm(A, B, Cn, 1.0, 0.0, kernel="auto", queue=q)
    n1.record(stream)
    torch.cuda.synchronize()
    native_ms = slowest(n0.elapsed_time(n1)) / args.native_steps
    clk = clocks.stop()

    # end to end through the public API with pinned host buffers: gb_dgemm_host
    # copies A and B in (A in row bands, B in column blocks), computes each piece as
    # its operands arrive and copies each piece of C back while the next ones compute
    A_p = torch.from_numpy(A_h).pin_memory()
    B_p = torch.from_numpy(B_h).pin_memory()
    C_p = torch.empty((n, n), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps)
    e2e_prec, e2e_count = ("emulated_crt", N) if crt else ("emulated", s)
    hws = gb.alloc_workspace(gb.host_workspace_size(e2e_prec, e2e_count, n, n, n))

    def e2e_step():
        gb.dgemm_host(A_p, B_p, C_p, 1.0, 0.0, precision=e2e_prec, slices=e2e_count, queue=q,
                      workspace=hws)

    # the host link's rate just before and just after the timed steps (one plain
    # pinned -> device copy of A each): the end-to-end figure moves with it, and
    # the link is shared with the other GPUs of the machine
    link_dst = torch.empty((n, n), dtype=torch.float64, device="cuda")

    def link_gbs():
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        link_dst.copy_(A_p, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        return round(8 * n * n / l0.elapsed_time(l1) / 1e6, 1)

    e2e_step()
    torch.cuda.synchronize()
    link_before = link_gbs()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps - 1)]
    e0.record(stream)
    for i in range(e2e_steps):
        e2e_step()
        if i + 1 < e2e_steps:
            marks[i].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = slowest(e0.elapsed_time(e1)) / e2e_steps
    bounds = [e0] + marks + [e1]
    e2e_each = sorted(bounds[i].elapsed_time(bounds[i + 1]) for i in range(e2e_steps))
    q.wait()
    link_after = link_gbs()
    del link_dst

    ms_step = ms_total / args.steps
    value = replica_value(flops, world, ms_step) / 1e12
    pk, pk_kind = peaks()
    fp8_peak = 2.0 * pk["bf16_tflops"]
    achieved = pair_flops / (prod_ms * 1e-3) / 1e12
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    native_tflops = flops / (native_ms * 1e-3) / 1e12
    if crt:
        roof = {"bound": "tensor", "kernel": "crt_products_kernel",
                "achieved": round(achieved, 1), "peak": round(pk["bf16_tflops"], 1),
                "unit": "TFLOP/s", "frac": round(achieved / pk["bf16_tflops"], 4),
                "peak_kind": f"{pk_kind} bf16 burst",
                "traffic": MEASURED_TRAFFIC.get(("crt_products_kernel", n, N)),
                "launch_ms": round(prod_ms, 4),
                "algorithmic": f"N * 2 n^3 = {pair_flops:.4g} BF16 flop per launch "
                               f"(N = {N} moduli)"}
    else:
        roof = {"bound": "tensor", "kernel": "emu_products_kernel",
                "achieved": round(achieved, 1), "peak": round(fp8_peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / fp8_peak, 4),
                "peak_kind": f"{pk_kind} bf16 burst x 2 (FP8 nominal ratio)",
                "traffic": MEASURED_TRAFFIC.get(("emu_products_kernel", n, s)),
                "launch_ms": round(prod_ms, 4),
                "algorithmic": f"s(s+1)/2 * 2 n^3 = {pair_flops:.4g} FP8 flop per launch"}

    metric, config = dgemm_metric_config(n, world)
    out = {
        "path": gpu_path("crt", N) if crt else gpu_path("e4m3", s),
        "metric": metric,
        "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded splitmix64, uniform[-1,1])",
        "config": config,
        "gpu_launches": (5 if crt else 4) * args.steps,
        "roofline": roof,
        "native": {"kernel": "dfma" if n > 2048 else "tiled", "value": round(native_tflops, 4),
                   "unit": "TFLOP/s",
                   "ms_per_call": round(native_ms, 2),
                   "roofline": {"bound": "alu", "achieved": round(native_tflops, 4),
                                "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                                "frac": round(native_tflops / fp64_peak, 4),
                                "peak_kind": "derived: 152 SM x 4 flop/clk x 2070 MHz"}},
        "e2e": {"value": round(replica_value(flops, world, e2e_ms) / 1e12, 3), "unit": "TFLOP/s",
                "h2d_bytes_per_step": 2 * 8 * n * n, "d2h_bytes_per_step": 8 * n * n,
                "ms_per_step": round(e2e_ms, 4),
                "step_ms_min_median_max": [round(e2e_each[0], 3),
                                           round(e2e_each[len(e2e_each) // 2], 3),
                                           round(e2e_each[-1], 3)],
                "link_h2d_gbs_before_after": [link_before, link_after]},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rec, sel, Crows = cpu_baseline(n, seed, args.cpu_seconds, A_h, B_h)
        out["cpu_baseline"] = rec
        pick = np.linspace(0, len(sel) - 1, min(16, len(sel))).astype(np.int64)
        sel, Crows = sel[pick], Crows[pick]
        from oracle import cgemm, exact
        absab = cgemm.dgemm_rows(sel, 1.0, np.abs(A_h), np.abs(B_h))
        bound = exact.error_bound(n, 1.0, absab)
        got_e = emu_C[torch.from_numpy(sel).cuda()].cpu().numpy()
        got_n = Cn[torch.from_numpy(sel).cuda()].cpu().numpy()
        hilo = cgemm.dgemm_dd_rows(A_h, B_h, sel)
        out["parity"] = {
            "rows_checked": int(len(sel)),
            "rho_emulated": rho_rows(got_e, A_h, B_h, sel, hilo),
            "rho_native": rho_rows(got_n, A_h, B_h, sel, hilo),
            "emulated_vs_oracle_over_bound": float(np.max(np.abs(got_e - Crows) / bound)),
            "native_vs_oracle_over_bound": float(np.max(np.abs(got_n - Crows) / bound)),
            "note": "rho = max |C - C*| / (2 (k+2) u |A||B|), C* the double-double value of A B "
                    "on the sampled rows; the *_vs_oracle figures compare with the FP64 oracle's "
                    "own rows, which carry their own rounding error"}
    if rank == 0 and world == 1 and not args.no_sub_records:
        del A_p, B_p, C_p, hws
        torch.cuda.empty_cache()
        out["other_path"] = other_path_record(args, gb, np, torch, A, B, C, q, A_h, B_h)
        out["bf16_digits"] = bf16_record(args, gb, np, torch, A, B, C, q, A_h, B_h)
        out["hard"] = hard_record(args, gb, g, np, torch, A, B, C, q)
        out["grouped"] = grouped_sub_record(args)
        out["serve"] = serve_sub_record(args, gb, g, np)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
