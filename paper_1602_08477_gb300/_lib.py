"""ctypes loader of libgbgemm.so and the C signatures of include/gb_gemm.h.

Argument marshalling only: no arithmetic of the GEMM happens in Python.  There
is no fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgbgemm.so")

GB_OK = 0
STATUS_NAMES = {
    0: "GB_OK", 1: "GB_ERR_INVALID_ARG", 2: "GB_ERR_INVALID_WORKDIV", 3: "GB_ERR_UNSUPPORTED",
    4: "GB_ERR_NO_DEVICE", 5: "GB_ERR_CUDA", 6: "GB_ERR_OUT_OF_BUDGET", 7: "GB_ERR_TIMEOUT",
    8: "GB_ERR_NONFINITE", 9: "GB_ERR_BUSY", 10: "GB_ERR_WORKSPACE",
}

GB_PREC_NATIVE, GB_PREC_EMULATED, GB_PREC_EMULATED_BF16, GB_PREC_EMULATED_CRT = 0, 1, 2, 3
#: precision names of the Python API -> gb_precision
PRECISIONS = {"native": GB_PREC_NATIVE, "emulated": GB_PREC_EMULATED,
              "emulated_bf16": GB_PREC_EMULATED_BF16, "emulated_crt": GB_PREC_EMULATED_CRT}


def precision_code(name: str) -> int:
    """gb_precision value of a precision name ("native", "emulated", "emulated_bf16",
    "emulated_crt")."""
    try:
        return PRECISIONS[name]
    except KeyError:
        raise ValueError(f"unknown precision {name!r}; one of {sorted(PRECISIONS)}") from None
KERNELS = {"auto": 0, "naive": 1, "tiled": 2, "dfma": 3, "dmma": 4}
GB_BAD_LINE = 0x40000000


class GbError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {message}")


class Workdiv(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_uint32),
                ("grid_blocks", ctypes.c_uint64 * 3),
                ("block_threads", ctypes.c_uint64 * 3),
                ("thread_elems", ctypes.c_uint64 * 3)]

    @classmethod
    def make(cls, grid, block, elems):
        wd = cls()
        wd.dim = len(grid)
        for d in range(3):
            wd.grid_blocks[d] = grid[d] if d < len(grid) else 1
            wd.block_threads[d] = block[d] if d < len(block) else 1
            wd.thread_elems[d] = elems[d] if d < len(elems) else 1
        return wd

    def as_tuple(self):
        n = self.dim
        return (tuple(self.grid_blocks[:n]), tuple(self.block_threads[:n]),
                tuple(self.thread_elems[:n]))


class EmulatedLayout(ctypes.Structure):
    _fields_ = [("kp", ctypes.c_int64), ("a_digits", ctypes.c_size_t),
                ("b_digits", ctypes.c_size_t), ("a_exp", ctypes.c_size_t),
                ("b_exp", ctypes.c_size_t), ("total", ctypes.c_size_t),
                ("a_tile_rows", ctypes.c_int32), ("b_tile_rows", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

_i64, _int, _dbl, _vp, _sz = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_st = ctypes.c_int

# name -> (restype, argtypes); mirrors include/*.h
SIGNATURES = {
    "gb_version": (_int, []),
    "gb_last_error": (ctypes.c_char_p, []),
    "gb_device_count": (_st, [ctypes.POINTER(_int)]),
    "gb_device_get": (_st, [_int, ctypes.POINTER(_vp)]),
    "gb_device_info": (_st, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "gb_device_release": (_st, [_vp]),
    "gb_queue_create": (_st, [_vp, _vp, _int, ctypes.POINTER(_vp)]),
    "gb_queue_wait": (_st, [_vp]),
    "gb_queue_stream": (_vp, [_vp]),
    "gb_queue_destroy": (_st, [_vp]),
    "gb_workdiv_suggest": (_st, [_vp, _int, _i64, _i64, _i64, ctypes.POINTER(Workdiv),
                                 ctypes.POINTER(_int)]),
    "gb_dgemm": (_st, [_vp, ctypes.POINTER(Workdiv), _int, _int, _int, _i64, _i64, _i64, _dbl,
                       _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _vp, _sz]),
    "gb_dgemm_workspace_size": (_st, [_int, _int, _i64, _i64, _i64, ctypes.POINTER(_sz)]),
    "gb_emulated_layout_get": (_st, [_int, _i64, _i64, _i64, ctypes.POINTER(EmulatedLayout)]),
    "gb_emulated_split_a": (_st, [_vp, _int, _i64, _i64, _i64, _vp, _i64, _vp, _sz]),
    "gb_emulated_split_b": (_st, [_vp, _int, _i64, _i64, _i64, _vp, _i64, _vp, _sz]),
    "gb_emulated_products": (_st, [_vp, _int, _i64, _i64, _i64, _dbl, _dbl, _vp, _i64, _vp, _sz]),
    "gb_emulated_crt_step": (_st, [_vp, _int, _int, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64,
                                   _dbl, _vp, _i64, _vp, _sz]),
    "gb_selftest_wait_timeout": (_st, [_vp, ctypes.c_uint32]),
    "gb_dgemm_emulated_noalloc": (_st, [_vp, _int, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64,
                                        _dbl, _vp, _i64]),
    "gb_dgemm_host": (_st, [_vp, _int, _int, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl,
                            _vp, _i64, _vp, _sz]),
    "gb_dgemm_host_workspace_size": (_st, [_int, _int, _i64, _i64, _i64, ctypes.POINTER(_sz)]),
    "gb_dgemm_host_schedule": (_st, [_int, _i64, _i64, _i64, _dbl, _int, ctypes.POINTER(_i64),
                                     _int, ctypes.POINTER(_int)]),
}


def extra_signatures(table: dict):
    """Register signatures of further entry points (used by the other modules)."""
    SIGNATURES.update(table)
    if _lib is not None:
        _apply(_lib, table)


def _apply(lib, table):
    for name, (res, args) in table.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def load():
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"the CUDA library is not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            # PyTorch loads its CUDA runtime (libcudart.so.13) by path; loading it
            # first lets the library bind to that same copy, so one runtime holds
            # every module's kernels (the library's, PyTorch's, and a caller's own
            # kernels launched through gb_enqueue)
            try:
                import torch  # noqa: F401
            except ImportError:
                pass
            lib = ctypes.CDLL(LIB_PATH)
            _apply(lib, SIGNATURES)
            _lib = lib
    return _lib


def last_error() -> str:
    msg = load().gb_last_error()
    return msg.decode() if msg else ""


def check(status: int, where: str):
    if status != GB_OK:
        raise GbError(status, where, last_error())
