"""Binding of include/gb_mem.h: pitched host and device buffers, explicit
copies, queues with their own stream, and DGEMM over buffers.

With these the library runs without PyTorch: allocate, copy and compute
through the C ABI only.  Marshalling only; no arithmetic here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import KERNELS, check, precision_code


class GbBuf(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("device", ctypes.c_int32), ("dim", ctypes.c_uint32),
                ("extent", ctypes.c_uint64 * 3), ("elem_bytes", ctypes.c_uint64),
                ("pitch_bytes", ctypes.c_uint64)]


_st, _vp = ctypes.c_int, ctypes.c_void_p
_lib.extra_signatures({
    "gb_buf_alloc": (_st, [_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
                           ctypes.POINTER(GbBuf)]),
    "gb_buf_free": (_st, [ctypes.POINTER(GbBuf)]),
    "gb_buf_ld": (_st, [ctypes.POINTER(GbBuf), ctypes.POINTER(ctypes.c_int64)]),
    "gb_buf_copy": (_st, [_vp, ctypes.POINTER(GbBuf), ctypes.POINTER(GbBuf),
                          ctypes.POINTER(ctypes.c_uint64)]),
    "gb_queue_create_owned": (_st, [_vp, ctypes.c_int, ctypes.POINTER(_vp)]),
})


def _u64s(vals):
    return (ctypes.c_uint64 * 3)(*(list(vals) + [1] * (3 - len(vals))))


class Buffer:
    """A pitched buffer of float64 (or another element size) on a device or in
    page-locked host memory (``device=None``)."""

    def __init__(self, shape, device=None, dtype=np.float64):
        self.dtype = np.dtype(dtype)
        self.shape = tuple(int(x) for x in shape)
        self.raw = GbBuf()
        check(_lib.load().gb_buf_alloc(device.handle if device is not None else None,
                                       len(self.shape), _u64s(self.shape), self.dtype.itemsize,
                                       ctypes.byref(self.raw)), "gb_buf_alloc")
        self.device = device

    @property
    def ld(self) -> int:
        out = ctypes.c_int64()
        check(_lib.load().gb_buf_ld(ctypes.byref(self.raw), ctypes.byref(out)), "gb_buf_ld")
        return out.value

    @property
    def pitch_bytes(self) -> int:
        return self.raw.pitch_bytes

    @property
    def ptr(self) -> int:
        return self.raw.ptr or 0

    def numpy(self) -> np.ndarray:
        """A strided view of a host buffer's memory (no copy)."""
        if self.raw.device >= 0:
            raise ValueError("numpy() views host buffers only; copy a device buffer first")
        rows = int(np.prod(self.shape[:-1])) if len(self.shape) > 1 else 1
        if not self.raw.ptr or rows == 0 or self.shape[-1] == 0:
            return np.zeros(self.shape, dtype=self.dtype)
        nbytes = self.raw.pitch_bytes * rows
        flat = (ctypes.c_ubyte * nbytes).from_address(self.raw.ptr)
        # row stride = pitch; plane stride = pitch * rows per plane; element stride
        strides = [self.dtype.itemsize]
        acc = self.raw.pitch_bytes
        for d in range(len(self.shape) - 2, -1, -1):
            strides.insert(0, acc)
            acc *= self.shape[d]
        return np.ndarray(self.shape, self.dtype, flat, 0, tuple(strides))

    def free(self):
        if self.raw.ptr:
            check(_lib.load().gb_buf_free(ctypes.byref(self.raw)), "gb_buf_free")

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def copy(queue, dst: Buffer, src: Buffer, extents=None):
    """Enqueue the copy of the leading ``extents`` block of src into dst."""
    ext = _u64s(extents) if extents is not None else None
    check(_lib.load().gb_buf_copy(queue.handle, ctypes.byref(dst.raw), ctypes.byref(src.raw), ext),
          "gb_buf_copy")


class OwnedQueue:
    """A queue with a CUDA stream of its own (no PyTorch involved)."""

    def __init__(self, device, blocking: bool = False):
        h = ctypes.c_void_p()
        check(_lib.load().gb_queue_create_owned(device.handle, int(blocking), ctypes.byref(h)),
              "gb_queue_create_owned")
        self.device = device
        self.handle = h
        self.blocking = blocking

    def wait(self):
        check(_lib.load().gb_queue_wait(self.handle), "gb_queue_wait")

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().gb_queue_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgemm_buffers(queue, A: Buffer, B: Buffer, C: Buffer, alpha: float = 1.0, beta: float = 0.0,
                  *, kernel: str = "auto", precision: str = "native", slices: int = 0,
                  workspace: Buffer | None = None):
    """C <- alpha A B + beta C over 2-D float64 device buffers (leading
    dimensions from their pitches).  Emulated precision takes a device
    workspace buffer of at least gemm.workspace_size bytes (1-D, uint8)."""
    (m, k), (k2, n) = A.shape, B.shape
    if k2 != k or C.shape != (m, n):
        raise ValueError(f"shapes {A.shape} x {B.shape} -> {C.shape} do not match")
    prec = precision_code(precision)
    ws = ctypes.c_void_p(workspace.ptr) if workspace is not None else None
    wbytes = workspace.shape[0] * workspace.dtype.itemsize if workspace is not None else 0
    check(_lib.load().gb_dgemm(queue.handle, None, KERNELS[kernel], prec, slices, m, n, k, alpha,
                               ctypes.c_void_p(A.ptr), max(A.ld, 1), ctypes.c_void_p(B.ptr),
                               max(B.ld, 1), beta, ctypes.c_void_p(C.ptr), max(C.ld, 1), ws,
                               wbytes), "gb_dgemm")
