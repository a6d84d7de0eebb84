"""Binding of include/gb_grouped.h: many GEMMs in one persistent launch.

Marshalling only: descriptors are filled from torch tensors and handed to the
library, which builds its tables in a torch-allocated workspace.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import check, precision_code

TUNE_SLICES = 100  # GB_TUNE_SLICES: a table entry of tile TUNE_SLICES + s gives slice count s
TILES = {"auto": 0, "64x64": 1, "32x32": 2, "64x32": 3, "32x64": 4,
         "emu_rows": 5, "emu_cols": 6}
TILES.update({f"emu_s{s}": TUNE_SLICES + s for s in range(1, 17)})
TILE_NAMES = {v: k for k, v in TILES.items()}


class GemmDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("tile", ctypes.c_int32)]


_i64, _int, _vp, _sz, _st = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
_lib.extra_signatures({
    "gb_grouped_workspace_size": (_st, [ctypes.POINTER(GemmDesc), _i64, ctypes.POINTER(_sz)]),
    "gb_grouped_plan_create": (_st, [_vp, ctypes.POINTER(GemmDesc), _i64, _vp, _sz, _int,
                                     ctypes.POINTER(_vp)]),
    "gb_grouped_plan_run": (_st, [_vp]),
    "gb_grouped_plan_info": (_st, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                   ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double)]),
    "gb_grouped_plan_destroy": (_st, [_vp]),
    "gb_dgemm_grouped": (_st, [_vp, ctypes.POINTER(GemmDesc), _i64, _vp, _sz]),
    "gb_tune_set": (_st, [ctypes.POINTER(TuneEntry), _i64]),
    "gb_tune_get": (_st, [ctypes.POINTER(TuneEntry), _i64, ctypes.POINTER(_i64)]),
    "gb_tune_lookup": (_st, [_i64, _i64, _i64, ctypes.POINTER(ctypes.c_int32)]),
    "gb_tune_lookup_emulated": (_st, [_int, _i64, _i64, _i64, ctypes.POINTER(ctypes.c_int32)]),
    "gb_tune_lookup_slices": (_st, [_i64, _i64, _i64, ctypes.POINTER(ctypes.c_int32)]),
})


def _ld(t, cols):
    return max(t.stride(0) if t.shape[0] > 1 else cols, cols, 1)


def make_descs(problems):
    """problems: iterable of dicts with A, B, C (float64 CUDA tensors) and
    optional alpha, beta, precision ("native"/"emulated"), slices, tile."""
    problems = list(problems)
    arr = (GemmDesc * max(1, len(problems)))()
    for i, p in enumerate(problems):
        A, B, C = p["A"], p["B"], p["C"]
        m, k = A.shape
        n = B.shape[1]
        d = arr[i]
        d.m, d.n, d.k = m, n, k
        d.alpha = p.get("alpha", 1.0)
        d.beta = p.get("beta", 0.0)
        d.A, d.lda = A.data_ptr(), _ld(A, k)
        d.B, d.ldb = B.data_ptr(), _ld(B, n)
        d.C, d.ldc = C.data_ptr(), _ld(C, n)
        d.precision = precision_code(p.get("precision", "native"))
        d.slices = p.get("slices", 0)
        d.tile = TILES[p.get("tile", "auto")] if isinstance(p.get("tile", "auto"), str) else p["tile"]
        d.reserved = 0
    return arr, len(problems)


def workspace_size(descs, count) -> int:
    out = ctypes.c_size_t()
    check(_lib.load().gb_grouped_workspace_size(descs, count, ctypes.byref(out)),
          "gb_grouped_workspace_size")
    return out.value


class GroupedPlan:
    """A group of GEMMs captured (optionally) in a CUDA graph; run() replays it."""

    def __init__(self, problems, queue=None, use_graph: bool = True, device=None):
        import torch
        from .gemm import default_queue
        self.problems = list(problems)
        self.descs, self.count = make_descs(self.problems)
        self.queue = queue or default_queue()
        nbytes = workspace_size(self.descs, self.count)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")
        h = ctypes.c_void_p()
        check(_lib.load().gb_grouped_plan_create(self.queue.handle, self.descs, self.count,
                                                 ctypes.c_void_p(self.workspace.data_ptr()),
                                                 self.workspace.numel(), int(use_graph),
                                                 ctypes.byref(h)), "gb_grouped_plan_create")
        self.handle = h

    def run(self):
        check(_lib.load().gb_grouped_plan_run(self.handle), "gb_grouped_plan_run")

    def info(self):
        nt, et, la, fl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_double()
        check(_lib.load().gb_grouped_plan_info(self.handle, ctypes.byref(nt), ctypes.byref(et),
                                               ctypes.byref(la), ctypes.byref(fl)),
              "gb_grouped_plan_info")
        return {"native_tiles": nt.value, "emulated_tiles": et.value, "launches": la.value,
                "flops": fl.value}

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().gb_grouped_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgemm_grouped(problems, queue=None):
    """Run a group once (no graph)."""
    import torch
    from .gemm import default_queue
    descs, count = make_descs(problems)
    q = queue or default_queue()
    nbytes = workspace_size(descs, count)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
    check(_lib.load().gb_dgemm_grouped(q.handle, descs, count, ctypes.c_void_p(ws.data_ptr()),
                                       ws.numel()), "gb_dgemm_grouped")
    return ws


def tune_set(entries):
    """entries: list of (m_max, n_max, k_max, tile name or id)."""
    arr = (TuneEntry * max(1, len(entries)))()
    for i, (mm, nn, kk, t) in enumerate(entries):
        arr[i].m_max, arr[i].n_max, arr[i].k_max = mm, nn, kk
        arr[i].tile = TILES[t] if isinstance(t, str) else t
    check(_lib.load().gb_tune_set(arr, len(entries)), "gb_tune_set")


def tune_get():
    n = ctypes.c_int64()
    check(_lib.load().gb_tune_get(None, 0, ctypes.byref(n)), "gb_tune_get")
    arr = (TuneEntry * max(1, n.value))()
    check(_lib.load().gb_tune_get(arr, n.value, ctypes.byref(n)), "gb_tune_get")
    return [(e.m_max, e.n_max, e.k_max, TILE_NAMES[e.tile]) for e in arr[:n.value]]


def tune_lookup(m, n, k) -> str:
    """Tile of a native problem of this shape under the installed table."""
    t = ctypes.c_int32()
    check(_lib.load().gb_tune_lookup(m, n, k, ctypes.byref(t)), "gb_tune_lookup")
    return TILE_NAMES[t.value]


def tune_lookup_slices(m, n, k) -> int:
    """Slice count of an emulated problem of this shape given slices = 0."""
    t = ctypes.c_int32()
    check(_lib.load().gb_tune_lookup_slices(m, n, k, ctypes.byref(t)), "gb_tune_lookup_slices")
    return t.value


def tune_lookup_emulated(m, n, k, slices=11) -> str:
    """Orientation ("emu_rows" or "emu_cols") of an emulated problem of this shape."""
    t = ctypes.c_int32()
    check(_lib.load().gb_tune_lookup_emulated(slices, m, n, k, ctypes.byref(t)),
          "gb_tune_lookup_emulated")
    return TILE_NAMES[t.value]
