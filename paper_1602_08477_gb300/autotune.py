"""Autotuner of the grouped kernels per problem-size cell.

The problem space (m, n, k) is cut into cells by the thresholds THRESHOLDS
(a cell is (m_max, n_max, k_max), the smallest thresholds >= the sizes).  For
every cell the tuner builds a batch of problems of that cell's sizes, runs the
grouped plan once per candidate with that candidate forced (CUDA-event timing,
median of several graph replays) and keeps the fastest:

  * native problems: the DFMA tile variant (64x64, 32x32, 64x32, 32x64);
  * emulated problems: the orientation of the 128 x bn product tiles (A's rows
    or B's columns on the 128-line side), which sets the padding, the tile count
    and whether the epilogue's stores to C are coalesced.

The result is one first-match table (cells in lexicographic order, so the first
entry of a problem's kind that it matches is its own cell), saved as JSON and
loaded into the library with gb_tune_set.

    python -m paper_1602_08477_gb300.autotune [--out tune_table.json] [--kinds native,emulated]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--batch", type=int, default=96)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--kinds", default="native,emulated",
                    help="problem kinds to tune; the other kind's entries are kept from "
                         "the current table")
    a = ap.parse_args()
    import torch

    from .compile_lib import build
    from .grouped import TILES
    build()
    kinds = [k for k in a.kinds.split(",") if k]
    try:
        with open(table_path()) as f:
            old = json.load(f)
    except Exception:
        old = {"entries": [], "report": [], "meta": {}}
    emu_ids = (TILES["emu_rows"], TILES["emu_cols"])

    def kind_of(tile):
        return "emulated" if (TILES[tile] if isinstance(tile, str) else tile) in emu_ids \
            else "native"
    entries = [tuple(e) for e in old["entries"] if kind_of(e[3]) not in kinds]
    report = [r for r in old.get("report", []) if r.get("kind", "native") not in kinds]
    for kind in kinds:
        e, r = tune(batch=a.batch, reps=a.reps, kind=kind)
        entries += e
        report += r
    meta = dict(old.get("meta", {}))
    meta.update({"device": torch.cuda.get_device_name(0), "batch": a.batch, "reps": a.reps,
                 "emulated_slices": EMU_SLICES})
    save(entries, a.out, report, meta=meta)
    print(f"wrote {a.out} ({len(entries)} entries)")


if __name__ == "__main__":
    main()
