"""Binding of include/gb_serve.h: the GEMM request server (marshalling only)."""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import check, precision_code


class Request(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("precision", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("A_host", ctypes.c_void_p), ("B_host", ctypes.c_void_p),
                ("C_host", ctypes.c_void_p), ("C_out", ctypes.c_void_p),
                ("seed", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("tflops", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("max_queue", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mean_batch", ctypes.c_double),
                ("peak_bytes", ctypes.c_size_t), ("large_launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_i64, _int, _vp, _sz, _st = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
_lib.extra_signatures({
    "gb_server_create": (_st, [_vp, _sz, _int, _int, ctypes.POINTER(_vp)]),
    "gb_server_create_ex": (_st, [_vp, _sz, _int, _int, _int, ctypes.POINTER(_vp)]),
    "gb_server_submit": (_st, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "gb_server_poll": (_st, [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(_int),
                             ctypes.POINTER(ctypes.c_double)]),
    "gb_server_drain": (_st, [_vp, ctypes.c_double]),
    "gb_server_stats_get": (_st, [_vp, ctypes.POINTER(ServerStats)]),
    "gb_server_destroy": (_st, [_vp]),
    "gb_fill_uniform": (_st, [_vp, _vp, _i64, _i64, _i64, ctypes.c_uint64, ctypes.c_int32]),
})


def _ptr(a):
    if a is None:
        return None
    return ctypes.c_void_p(a.ctypes.data) if hasattr(a, "ctypes") else ctypes.c_void_p(a.data_ptr())


class Server:
    """Requests in, results out; budget-admitted and batched on the device."""

    POLICIES = {"lanes": 0, "fifo": 1}

    def __init__(self, hbm_budget_bytes: int, n_streams: int = 4, max_batch: int = 64,
                 device=None, policy: str = "lanes"):
        """policy "lanes": large native requests alone on low-priority streams,
        small ones batched on high-priority streams; "fifo": one queue, every
        batch a grouped launch (max_batch = 1: one launch per GEMM)."""
        from .gemm import Device
        if policy not in self.POLICIES:
            raise ValueError(f"policy must be one of {sorted(self.POLICIES)}")
        self.device = device or Device(0)
        h = ctypes.c_void_p()
        check(_lib.load().gb_server_create_ex(self.device.handle, hbm_budget_bytes, n_streams,
                                              max_batch, self.POLICIES[policy],
                                              ctypes.byref(h)), "gb_server_create_ex")
        self.handle = h
        self._keep = {}

    def submit(self, m, n, k, alpha=1.0, beta=0.0, precision="native", slices=0, A=None, B=None,
               C=None, out=None, seed=0):
        """A, B, C, out: C-contiguous float64 host arrays (numpy) or None (device-
        generated operands from `seed`).  Returns the request id."""
        r = Request(m, n, k, alpha, beta, precision_code(precision), slices,
                    _ptr(A), _ptr(B), _ptr(C), _ptr(out), seed)
        rid = ctypes.c_uint64()
        check(_lib.load().gb_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)),
              "gb_server_submit")
        if A is not None or out is not None:
            self._keep[rid.value] = (A, B, C, out)  # host buffers live until done
        return rid.value

    def poll(self, rid):
        done, st, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(_lib.load().gb_server_poll(self.handle, rid, ctypes.byref(done), ctypes.byref(st),
                                         ctypes.byref(lat)), "gb_server_poll")
        return bool(done.value), st.value, lat.value

    def drain(self, timeout_s=600.0):
        check(_lib.load().gb_server_drain(self.handle, timeout_s), "gb_server_drain")

    def stats(self):
        s = ServerStats()
        check(_lib.load().gb_server_stats_get(self.handle, ctypes.byref(s)), "gb_server_stats_get")
        return s.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().gb_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fill_uniform(t, seed: int, stream_id: int):
    """Fill a float64 CUDA matrix with the request generator's values."""
    import torch
    rows, cols = t.shape
    s = torch.cuda.current_stream().cuda_stream
    check(_lib.load().gb_fill_uniform(ctypes.c_void_p(s), ctypes.c_void_p(t.data_ptr()), rows,
                                      cols, max(t.stride(0), cols, 1), seed, stream_id),
          "gb_fill_uniform")
    return t
