"""Binding of include/gb_exec.h: the generic work-division executor and DAXPY."""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import Workdiv, check

_i64, _vp, _sz, _st, _dbl = ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
_lib.extra_signatures({
    "gb_enqueue": (_st, [_vp, ctypes.POINTER(Workdiv), _vp, ctypes.POINTER(_vp), _sz]),
    "gb_kernel_handle": (_vp, [ctypes.c_char_p]),
    "gb_daxpy": (_st, [_vp, ctypes.POINTER(Workdiv), _i64, _dbl, _vp, _vp]),
})


def kernel_handle(name: str):
    h = _lib.load().gb_kernel_handle(name.encode())
    if not h:
        raise KeyError(f"no library kernel named {name!r}")
    return h


def enqueue(kernel, workdiv: Workdiv, args, queue=None, shared_bytes: int = 0):
    """Enqueue `kernel` with `workdiv`; args: list of ctypes scalars (kept alive)."""
    from .gemm import default_queue
    q = queue or default_queue()
    ptrs = (_vp * max(1, len(args)))(*[ctypes.cast(ctypes.pointer(a), _vp) for a in args])
    check(_lib.load().gb_enqueue(q.handle, ctypes.byref(workdiv), _vp(kernel), ptrs,
                                 shared_bytes), "gb_enqueue")


def daxpy(alpha: float, x, y, workdiv: Workdiv | None = None, queue=None):
    """y <- alpha * x + y on the GPU (float64 CUDA tensors of equal length)."""
    from .gemm import default_queue
    if x.numel() != y.numel():
        raise ValueError("x and y differ in length")
    q = queue or default_queue()
    wd = ctypes.byref(workdiv) if workdiv is not None else None
    check(_lib.load().gb_daxpy(q.handle, wd, x.numel(), alpha, _vp(x.data_ptr()),
                               _vp(y.data_ptr())), "gb_daxpy")
    return y
