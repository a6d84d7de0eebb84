"""Autotuner of the grouped kernels per problem-size cell.

The problem space (m, n, k) is cut into cells by the thresholds THRESHOLDS
(a cell is (m_max, n_max, k_max), the smallest thresholds >= the sizes).  For
every cell the tuner builds a batch of problems of that cell's sizes, runs the
grouped plan once per candidate with that candidate forced (CUDA-event timing,
median of several graph replays) and keeps the fastest:

  * native problems: the DFMA tile variant (64x64, 32x32, 64x32, 32x64);
  * emulated problems: the orientation of the 128 x bn product tiles (A's rows
    or B's columns on the 128-line side), which sets the padding, the tile count
    and whether the epilogue's stores to C are coalesced;
  * the slice count of emulated problems submitted with slices = 0, per K cell
    (kind "slices"): the fastest of SLICE_CANDIDATES whose result stays within
    RHO_TARGET of the FP64 error bound 2 (k + 2) u (|A||B|)_ij on every problem
    of the cell's batch (m and n log-uniform over [16, 512], uniform[-1, 1]
    entries).  The error is taken against the same group at REF_SLICES slices,
    whose own error is far below the bound, and |A||B| comes from the library's
    native kernels.  The bound grows like k^2 and the truncation error of the
    digits like sqrt(k), so short dot products need more digits.

The result is one first-match table (cells in lexicographic order, so the first
entry of a problem's kind that it matches is its own cell), saved as JSON and
loaded into the library with gb_tune_set.

    python -m paper_1602_08477_gb300.autotune [--out tune_table.json] [--kinds native,emulated,slices]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

THRESHOLDS = (32, 64, 128, 256, 512)
CANDIDATES = ("64x64", "32x32", "64x32", "32x64")
EMU_CANDIDATES = ("emu_rows", "emu_cols")
EMU_SLICES = 11
SLICE_CANDIDATES = (9, 10, 11, 12)
REF_SLICES = 16
RHO_TARGET = 0.25
# a slice count other than EMU_SLICES must beat it by this fraction of its time in
# the cell: a group whose problems use two counts runs two launch sets (split
# rows, column strips, products) one after the other, and their tails cost more
# than a gain of a percent or two in one cell
MIN_GAIN = 0.03
ANY = (1 << 31) - 1  # m_max / n_max of the slice-count entries: every size
DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.json")


def cell_of(x: int) -> int:
    for t in THRESHOLDS:
        if x <= t:
            return t
    return 1 << 30


def _cell_sizes(cell_max: int) -> tuple[int, int]:
    lo = 1
    for t in THRESHOLDS:
        if t == cell_max:
            break
        lo = t + 1
    return lo, cell_max


def time_variant(problems, tile: str, reps: int = 5) -> float:
    """Median ms of one grouped run with every problem forced to `tile`."""
    import torch

    from .grouped import GroupedPlan
    for p in problems:
        p["tile"] = tile
    plan = GroupedPlan(problems, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    times = []
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    plan.close()
    return statistics.median(times)


def tune(batch: int = 96, seed: int = 20240, reps: int = 5, log=print, kind: str = "native"):
    """Measure every cell for problems of `kind` ("native" or "emulated");
    returns the entry list [(m_max, n_max, k_max, tile)] and a report."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed + (0 if kind == "native" else 1))
    cands = CANDIDATES if kind == "native" else EMU_CANDIDATES
    entries, report = [], []
    for mm in THRESHOLDS:
        for nn in THRESHOLDS:
            for kk in THRESHOLDS:
                probs = []
                for _ in range(batch):
                    m = int(rng.integers(*_cell_sizes(mm), endpoint=True))
                    n = int(rng.integers(*_cell_sizes(nn), endpoint=True))
                    k = int(rng.integers(*_cell_sizes(kk), endpoint=True))
                    A = torch.rand((m, k), dtype=torch.float64, device="cuda")
                    B = torch.rand((k, n), dtype=torch.float64, device="cuda")
                    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
                    p = dict(A=A, B=B, C=C, alpha=1.0, beta=0.0)
                    if kind == "emulated":
                        p.update(precision="emulated", slices=EMU_SLICES)
                    probs.append(p)
                ms = {t: time_variant(probs, t, reps) for t in cands}
                best = min(ms, key=ms.get)
                entries.append((mm, nn, kk, best))
                report.append(dict(kind=kind, cell=[mm, nn, kk], ms=ms, best=best))
                log(f"{kind} cell m<={mm} n<={nn} k<={kk}: " +
                    " ".join(f"{t}={v:.3f}ms" for t, v in ms.items()) + f" -> {best}")
    return entries, report


def _time_group(problems, reps: int = 5) -> float:
    """Median ms of one graph replay of the group."""
    import torch

    from .grouped import GroupedPlan
    plan = GroupedPlan(problems, use_graph=True)
    plan.run()
    torch.cuda.synchronize()
    times = []
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    plan.close()
    return statistics.median(times)


def group_rho(problems, ref, bounds) -> float:
    """Largest |C - C_ref| / bound over the outputs of a group (after a run)."""
    worst = 0.0
    for p, r, b in zip(problems, ref, bounds):
        worst = max(worst, float(((p["C"] - r).abs() / b).max()))
    return worst


def choose_slices(ms) -> int:
    """The cell's slice count from the times {s: ms} of the counts that met the
    accuracy target: the fastest, unless EMU_SLICES met it and the fastest is
    not MIN_GAIN faster; REF_SLICES when none met it."""
    if not ms:
        return REF_SLICES
    best = min(ms, key=ms.get)
    if EMU_SLICES in ms and ms[best] > (1.0 - MIN_GAIN) * ms[EMU_SLICES]:
        return EMU_SLICES
    return best


def tune_slices(batch: int = 96, seed: int = 20240, reps: int = 5, log=print):
    """Per K cell: the fastest slice count that keeps every problem of the cell's
    batch within RHO_TARGET of the FP64 bound; entries [(ANY, ANY, k_max,
    "emu_s<s>")] and a report."""
    import math

    import numpy as np
    import torch

    from .gemm import dgemm
    from .grouped import GroupedPlan
    rng = np.random.default_rng(seed + 2)
    u = 2.0 ** -53
    entries, report = [], []
    for kk in THRESHOLDS:
        lo, hi = _cell_sizes(kk)
        lo = max(lo, 16)
        probs, bounds = [], []
        for _ in range(batch):
            m, n = (int(round(math.exp(rng.uniform(math.log(16), math.log(512)))))
                    for _ in range(2))
            k = int(rng.integers(lo, hi, endpoint=True))
            A = torch.rand((m, k), dtype=torch.float64, device="cuda") * 2 - 1
            B = torch.rand((k, n), dtype=torch.float64, device="cuda") * 2 - 1
            C = torch.zeros((m, n), dtype=torch.float64, device="cuda")
            probs.append(dict(A=A, B=B, C=C, alpha=1.0, beta=0.0, precision="emulated"))
            bounds.append(2.0 * (k + 2) * u * dgemm(A.abs(), B.abs()))
        ref_probs = [dict(p, slices=REF_SLICES) for p in probs]
        plan = GroupedPlan(ref_probs, use_graph=False)
        plan.run()
        torch.cuda.synchronize()
        plan.close()
        ref = [p["C"].clone() for p in probs]
        rho, ms = {}, {}
        for s in SLICE_CANDIDATES:
            cand = [dict(p, slices=s) for p in probs]
            plan = GroupedPlan(cand, use_graph=False)
            plan.run()
            torch.cuda.synchronize()
            plan.close()
            rho[s] = group_rho(cand, ref, bounds)
            if rho[s] <= RHO_TARGET:
                ms[s] = _time_group(cand, reps)
        best = choose_slices(ms)
        entries.append((ANY, ANY, kk, f"emu_s{best}"))
        report.append(dict(kind="slices", cell=[ANY, ANY, kk], rho=rho, ms=ms, best=best))
        log(f"slices cell k<={kk}: " + " ".join(
            f"s={s}: rho {rho[s]:.3g}" + (f" {ms[s]:.3f}ms" if s in ms else " (over)")
            for s in SLICE_CANDIDATES) + f" -> {best}")
    return entries, report


def save(entries, path: str = DEFAULT_TABLE, report=None, meta=None):
    with open(path, "w") as f:
        json.dump({"thresholds": list(THRESHOLDS), "entries": [list(e) for e in entries],
                   "meta": meta or {}, "report": report or []}, f, indent=1)


def table_path(path: str | None = None) -> str:
    """The table to read: `path`, else $GB_TUNE_TABLE, else the shipped table."""
    return path or os.environ.get("GB_TUNE_TABLE") or DEFAULT_TABLE


def load(path: str | None = None, apply: bool = True):
    """Read a table (see table_path) and (by default) install it in the library."""
    with open(table_path(path)) as f:
        d = json.load(f)
    entries = [tuple(e) for e in d["entries"]]
    if apply:
        from .grouped import tune_set
        tune_set(entries)
    return entries


def kind_of(tile) -> str:
    """Kind of a table entry's tile: "native", "emulated" (orientation) or "slices"."""
    from .grouped import TILES, TUNE_SLICES
    t = TILES[tile] if isinstance(tile, str) else tile
    if t in (TILES["emu_rows"], TILES["emu_cols"]):
        return "emulated"
    if TUNE_SLICES < t <= TUNE_SLICES + 16:
        return "slices"
    return "native"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--batch", type=int, default=96)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--kinds", default="native,emulated,slices",
                    help="problem kinds to tune; the other kind's entries are kept from "
                         "the current table")
    a = ap.parse_args()
    import torch

    from .compile_lib import build
    build()
    kinds = [k for k in a.kinds.split(",") if k]
    try:
        with open(table_path()) as f:
            old = json.load(f)
    except Exception:
        old = {"entries": [], "report": [], "meta": {}}
    entries = [tuple(e) for e in old["entries"] if kind_of(e[3]) not in kinds]
    report = [r for r in old.get("report", []) if r.get("kind", "native") not in kinds]
    for kind in kinds:
        if kind == "slices":
            e, r = tune_slices(batch=a.batch, reps=a.reps)
        else:
            e, r = tune(batch=a.batch, reps=a.reps, kind=kind)
        entries += e
        report += r
    meta = dict(old.get("meta", {}))
    meta.update({"device": torch.cuda.get_device_name(0), "batch": a.batch, "reps": a.reps,
                 "emulated_slices": EMU_SLICES, "slice_rho_target": RHO_TARGET,
                 "slice_reference": REF_SLICES, "slice_min_gain": MIN_GAIN})
    save(entries, a.out, report, meta=meta)
    print(f"wrote {a.out} ({len(entries)} entries)")


if __name__ == "__main__":
    main()
