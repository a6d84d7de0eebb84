"""Python binding of the C ABI over PyTorch tensors (device memory and streams).

Thin marshalling layer: it takes torch float64 CUDA tensors, passes their
pointers, leading dimensions and torch's CUDA stream to the C library, and
raises GbError on a non-OK status.  Every step of the GEMM runs in the
library's CUDA kernels; there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (GB_PREC_NATIVE, KERNELS, EmulatedLayout, Workdiv, check,
                   precision_code)


class Device:
    """A CUDA device handle (explicit: nothing becomes implicitly current)."""

    def __init__(self, index: int = 0):
        lib = _lib.load()
        h = ctypes.c_void_p()
        check(lib.gb_device_get(index, ctypes.byref(h)), "gb_device_get")
        self.index = index
        self.handle = h
        sm, ma, mi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib.gb_device_info(h, ctypes.byref(sm), ctypes.byref(ma), ctypes.byref(mi)),
              "gb_device_info")
        self.sm_count, self.cc = sm.value, (ma.value, mi.value)

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.gb_device_release(self.handle)
            self.handle = None


class Queue:
    """In-order work queue wrapping a CUDA stream (torch's current stream by default)."""

    def __init__(self, device: Device, stream=None, blocking: bool = False):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device.index)
        self.device = device
        self.stream = stream
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        check(_lib.load().gb_queue_create(device.handle, ctypes.c_void_p(raw), int(blocking),
                                          ctypes.byref(h)), "gb_queue_create")
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


_devices: dict = {}
_queues: dict = {}


def default_queue(device_index: int | None = None) -> Queue:
    """A non-blocking queue on torch's current stream of the device."""
    import torch
    idx = torch.cuda.current_device() if device_index is None else device_index
    stream = torch.cuda.current_stream(idx)
    key = (idx, stream.cuda_stream)
    q = _queues.get(key)
    if q is None:
        dev = _devices.get(idx)
        if dev is None:
            dev = _devices[idx] = Device(idx)
        q = _queues[key] = Queue(dev, stream)
    return q


def workdiv_suggest(kernel: str, m: int, n: int, k: int, device: Device | None = None):
    wd = Workdiv()
    chosen = ctypes.c_int()
    check(_lib.load().gb_workdiv_suggest(device.handle if device else None, KERNELS[kernel], m, n,
                                         k, ctypes.byref(wd), ctypes.byref(chosen)),
          "gb_workdiv_suggest")
    return wd, chosen.value


def workspace_size(precision: str, slices: int, m: int, n: int, k: int) -> int:
    out = ctypes.c_size_t()
    prec = precision_code(precision)
    check(_lib.load().gb_dgemm_workspace_size(prec, slices, m, n, k, ctypes.byref(out)),
          "gb_dgemm_workspace_size")
    return out.value


def emulated_layout(slices: int, m: int, n: int, k: int) -> EmulatedLayout:
    lay = EmulatedLayout()
    check(_lib.load().gb_emulated_layout_get(slices, m, n, k, ctypes.byref(lay)),
          "gb_emulated_layout_get")
    return lay


def _matrix_args(t, name):
    import torch
    if t is None:
        return None, 1
    if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D float64 CUDA tensor")
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    ld = t.stride(0) if t.shape[0] > 1 else max(1, t.shape[1])
    return ctypes.c_void_p(t.data_ptr()), ld


def alloc_workspace(nbytes: int, device=None):
    import torch
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device or "cuda")


def dgemm(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, *, kernel: str = "auto",
          precision: str = "native", slices: int = 0, workdiv: Workdiv | None = None,
          queue: Queue | None = None, workspace=None):
    """C <- alpha * A @ B + beta * C on the GPU; returns C.

    A (m x k), B (k x n), C (m x n) are float64 CUDA tensors, row-major, any
    leading dimension (a column slice of a wider tensor is fine).  C is created
    (zeros) when None.  precision: "native", "emulated" (E4M3 digits) or
    "emulated_bf16" (BF16 digits) or "emulated_crt" (residues modulo `slices`
    primes, 0 = 13); kernel: "auto", "naive", "tiled", "dfma",
    "dmma"; slices: emulated digit slices (0 = the precision's default).
    """
    import torch
    m, k = A.shape
    k2, n = B.shape
    if k2 != k:
        raise ValueError(f"inner dimensions differ: {A.shape} x {B.shape}")
    if C is None:
        C = torch.zeros((m, n), dtype=torch.float64, device=A.device)
        beta = 0.0
    if tuple(C.shape) != (m, n):
        raise ValueError(f"C has shape {tuple(C.shape)}, expected {(m, n)}")
    q = queue or default_queue(A.device.index)
    pa, lda = _matrix_args(A, "A")
    pb, ldb = _matrix_args(B, "B")
    pc, ldc = _matrix_args(C, "C")
    lda, ldb, ldc = max(lda, k, 1), max(ldb, n, 1), max(ldc, n, 1)
    prec = precision_code(precision)
    ws_ptr, ws_bytes = None, 0
    if prec != GB_PREC_NATIVE:
        need = workspace_size(precision, slices, m, n, k)
        if workspace is None:
            workspace = alloc_workspace(need, A.device)
        ws_ptr, ws_bytes = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    wd = ctypes.byref(workdiv) if workdiv is not None else None
    check(_lib.load().gb_dgemm(q.handle, wd, KERNELS[kernel], prec, slices, m, n, k, alpha,
                               pa, lda, pb, ldb, beta, pc, ldc, ws_ptr, ws_bytes), "gb_dgemm")
    return C


def host_workspace_size(precision: str, slices: int, m: int, n: int, k: int) -> int:
    """Device workspace bytes of dgemm_host for these sizes."""
    out = ctypes.c_size_t()
    prec = precision_code(precision)
    check(_lib.load().gb_dgemm_host_workspace_size(prec, slices, m, n, k, ctypes.byref(out)),
          "gb_dgemm_host_workspace_size")
    return out.value


def host_schedule(slices: int, m: int, n: int, k: int, beta: float = 0.0, *,
                  sm_count: int) -> list:
    """The products launches of dgemm_host (emulated) on a device with `sm_count`
    SMs, in enqueue order: a list of (row0, row1, col0, col1) blocks of C."""
    buf = (ctypes.c_int64 * 40)()
    count = ctypes.c_int()
    check(_lib.load().gb_dgemm_host_schedule(slices, m, n, k, beta, sm_count, buf, 10,
                                             ctypes.byref(count)), "gb_dgemm_host_schedule")
    return [tuple(buf[4 * p:4 * p + 4]) for p in range(count.value)]


def _host_matrix_args(t, name):
    import torch
    if t.dtype != torch.float64 or t.is_cuda or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D float64 host (CPU) tensor")
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    ld = t.stride(0) if t.shape[0] > 1 else max(1, t.shape[1])
    return ctypes.c_void_p(t.data_ptr()), ld


def dgemm_host(A, B, C, alpha: float = 1.0, beta: float = 0.0, *, precision: str = "native",
               slices: int = 0, queue: Queue | None = None, workspace=None):
    """C <- alpha * A @ B + beta * C with A, B, C float64 tensors in host memory
    (pinned for overlapped copies); the library copies them in, computes and
    copies C back, overlapped on the queue (gb_dgemm_host).  The result is in C
    once the queue has passed the call (torch.cuda.synchronize or queue.wait)."""
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError(f"shapes differ: {tuple(A.shape)} x {tuple(B.shape)} -> {tuple(C.shape)}")
    q = queue or default_queue()
    pa, lda = _host_matrix_args(A, "A")
    pb, ldb = _host_matrix_args(B, "B")
    pc, ldc = _host_matrix_args(C, "C")
    lda, ldb, ldc = max(lda, k, 1), max(ldb, n, 1), max(ldc, n, 1)
    prec = precision_code(precision)
    need = host_workspace_size(precision, slices, m, n, k)
    if workspace is None:
        workspace = alloc_workspace(need)
    check(_lib.load().gb_dgemm_host(q.handle, prec, slices, m, n, k, alpha, pa, lda, pb, ldb,
                                    beta, pc, ldc, ctypes.c_void_p(workspace.data_ptr()),
                                    workspace.numel() * workspace.element_size()),
          "gb_dgemm_host")
    return C


def emulated_steps(A, B, C, alpha, beta, slices, workspace, queue: Queue | None = None,
                   steps=("split_a", "split_b", "products")):
    """Run the emulated path's steps one by one (e1+e2 for A, for B, e3+e4)."""
    m, k = A.shape
    n = B.shape[1]
    q = queue or default_queue(A.device.index)
    lib = _lib.load()
    ws, wsb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel()
    if "split_a" in steps:
        pa, lda = _matrix_args(A, "A")
        check(lib.gb_emulated_split_a(q.handle, slices, m, n, k, pa, max(lda, k, 1), ws, wsb),
              "gb_emulated_split_a")
    if "split_b" in steps:
        pb, ldb = _matrix_args(B, "B")
        check(lib.gb_emulated_split_b(q.handle, slices, m, n, k, pb, max(ldb, n, 1), ws, wsb),
              "gb_emulated_split_b")
    if "products" in steps:
        pc, ldc = _matrix_args(C, "C")
        check(lib.gb_emulated_products(q.handle, slices, m, n, k, alpha, beta, pc,
                                       max(ldc, n, 1), ws, wsb), "gb_emulated_products")
    return C


CRT_STEPS = ("split_a", "split_b", "products", "combine")


def emulated_crt_steps(A, B, C, alpha, beta, moduli, workspace, queue: Queue | None = None,
                       steps=CRT_STEPS):
    """Run the residue precision's steps one by one (gb_emulated_crt_step): the
    residues of A's rows, of B's columns, the residue products, the
    reconstruction into C."""
    m, k = A.shape
    n = B.shape[1]
    q = queue or default_queue(A.device.index)
    lib = _lib.load()
    ws, wsb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel()
    pa, lda = _matrix_args(A, "A")
    pb, ldb = _matrix_args(B, "B")
    pc, ldc = _matrix_args(C, "C")
    for st in steps:
        check(lib.gb_emulated_crt_step(q.handle, CRT_STEPS.index(st), moduli, m, n, k, alpha,
                                       pa, max(lda, k, 1), pb, max(ldb, n, 1), beta, pc,
                                       max(ldc, n, 1), ws, wsb), "gb_emulated_crt_step")
    return C
