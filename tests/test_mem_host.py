"""Pitched buffers and copies (include/gb_mem.h): argument checks and layout
rules on the host, with no device work."""
import ctypes

import pytest

import paper_1602_08477_gb300 as gb
from paper_1602_08477_gb300 import _lib, mem


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return _lib.load()


def u64s(*v):
    return (ctypes.c_uint64 * 3)(*(list(v) + [1] * (3 - len(v))))


def test_alloc_rejects_bad_arguments(lib):
    b = mem.GbBuf()
    assert lib.gb_buf_alloc(None, 0, u64s(4, 4), 8, ctypes.byref(b)) == 1
    assert lib.gb_buf_alloc(None, 4, u64s(4, 4), 8, ctypes.byref(b)) == 1
    assert lib.gb_buf_alloc(None, 2, u64s(4, 4), 0, ctypes.byref(b)) == 1
    assert lib.gb_buf_alloc(None, 2, None, 8, ctypes.byref(b)) == 1
    assert lib.gb_buf_alloc(None, 2, u64s(4, 4), 8, None) == 1
    # 2^40 rows x 2^30 elements x 8 B overflows 64 bits
    assert lib.gb_buf_alloc(None, 2, u64s(1 << 40, 1 << 30), 1 << 30, ctypes.byref(b)) == 1
    assert b"overflow" in lib.gb_last_error()


def test_empty_buffer_needs_no_memory(lib):
    b = mem.GbBuf()
    assert lib.gb_buf_alloc(None, 2, u64s(0, 7), 8, ctypes.byref(b)) == 0
    assert not b.ptr and b.dim == 2 and tuple(b.extent) == (0, 7, 1) and b.device == -1
    assert b.pitch_bytes == 64  # 56 B rounded up to 16
    ld = ctypes.c_int64()
    assert lib.gb_buf_ld(ctypes.byref(b), ctypes.byref(ld)) == 0 and ld.value == 8
    assert lib.gb_buf_free(ctypes.byref(b)) == 0


def test_ld_needs_a_pitch_multiple_of_the_element(lib):
    b = mem.GbBuf()
    b.elem_bytes, b.pitch_bytes, b.dim = 24, 64, 2
    ld = ctypes.c_int64()
    assert lib.gb_buf_ld(ctypes.byref(b), ctypes.byref(ld)) == 3  # GB_ERR_UNSUPPORTED


def test_copy_rejects_mismatches_before_any_device_work(lib):
    a, b = mem.GbBuf(), mem.GbBuf()
    a.dim, b.dim = 2, 3
    a.elem_bytes = b.elem_bytes = 8
    fake_queue = ctypes.c_void_p(1)  # never dereferenced: the checks come first
    assert lib.gb_buf_copy(None, ctypes.byref(a), ctypes.byref(b), None) == 1
    assert lib.gb_buf_copy(fake_queue, ctypes.byref(a), ctypes.byref(b), None) == 1
    b.dim = 2
    b.elem_bytes = 4
    assert lib.gb_buf_copy(fake_queue, ctypes.byref(a), ctypes.byref(b), None) == 1
    b.elem_bytes = 8
    a.extent[0], a.extent[1] = 4, 4
    b.extent[0], b.extent[1] = 8, 4
    # whole-src copy does not fit dst
    assert lib.gb_buf_copy(fake_queue, ctypes.byref(a), ctypes.byref(b), None) == 1
    assert b"exceeds" in lib.gb_last_error()


def test_host_alloc_without_a_device_is_an_error(lib):
    n = ctypes.c_int(-1)
    if lib.gb_device_count(ctypes.byref(n)) == 0:
        pytest.skip("a CUDA device is present")
    b = mem.GbBuf()
    assert lib.gb_buf_alloc(None, 2, u64s(4, 4), 8, ctypes.byref(b)) == 4  # GB_ERR_NO_DEVICE
    assert not b.ptr
