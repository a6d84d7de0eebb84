"""The C-ABI library: builds, loads, exports every declared symbol, and rejects bad
arguments on the host before any device work (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1602_08477_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def declared_functions():
    names = set()
    pat = re.compile(r"^\s*(?:gb_status|int|const char\s*\*|const void\s*\*|void\s*\*)\s*(gb_\w+)\s*\(", re.M)
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names.update(pat.findall(open(h).read()))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for must in ("gb_dgemm", "gb_queue_create", "gb_device_get", "gb_workdiv_suggest",
                 "gb_dgemm_workspace_size", "gb_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_every_declared_symbol_has_a_binding_signature(lib):
    missing = [n for n in declared_functions() if n not in _lib.SIGNATURES]
    assert not missing, missing


def test_version_and_error_string(lib):
    assert lib.gb_version() >= 100
    assert isinstance(lib.gb_last_error(), bytes)


def test_null_queue_rejected_on_host(lib):
    st = lib.gb_dgemm(None, None, 0, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, 0)
    assert st == 1  # GB_ERR_INVALID_ARG
    assert b"NULL" in lib.gb_last_error()


def test_workspace_size_and_layout(lib):
    out = ctypes.c_size_t()
    assert lib.gb_dgemm_workspace_size(0, 0, 100, 100, 100, ctypes.byref(out)) == 0
    assert out.value == 0
    assert lib.gb_dgemm_workspace_size(1, 11, 100, 70, 45, ctypes.byref(out)) == 0
    lay = _lib.EmulatedLayout()
    assert lib.gb_emulated_layout_get(11, 100, 70, 45, ctypes.byref(lay)) == 0
    assert lay.kp == 64
    assert lay.a_digits == 0 and lay.b_digits >= 11 * 100 * 64
    assert lay.a_exp >= lay.b_digits + 11 * 70 * 64 and lay.b_exp >= lay.a_exp + 400
    assert all(x % 1024 == 0 for x in (lay.b_digits, lay.a_exp, lay.b_exp))
    assert out.value == lay.total
    # slices out of range
    assert lib.gb_dgemm_workspace_size(1, 17, 8, 8, 8, ctypes.byref(out)) == 1
    assert lib.gb_dgemm_workspace_size(1, -1, 8, 8, 8, ctypes.byref(out)) == 1
    assert lib.gb_dgemm_workspace_size(0, 0, -1, 8, 8, ctypes.byref(out)) == 1


def test_workdiv_suggest_follows_table2_cuda_row(lib):
    # blocks = N / (B * V) per dimension (Table 2, CUDA row)
    wd = _lib.Workdiv()
    chosen = ctypes.c_int()
    for kernel, (B, V) in {1: (16, 1), 2: (16, 1), 3: (16, 4)}.items():
        assert lib.gb_workdiv_suggest(None, kernel, 1000, 700, 64, ctypes.byref(wd),
                                      ctypes.byref(chosen)) == 0
        assert chosen.value == kernel
        assert wd.dim == 2
        assert tuple(wd.block_threads[:2]) == (B, B)
        assert tuple(wd.thread_elems[:2]) == (V, V)
        assert wd.grid_blocks[0] == -(-1000 // (B * V))
        assert wd.grid_blocks[1] == -(-700 // (B * V))
    assert lib.gb_workdiv_suggest(None, 0, 4096, 4096, 4096, ctypes.byref(wd),
                                  ctypes.byref(chosen)) == 0
    assert chosen.value == 3  # DFMA: 16 x 16 threads, 4 x 4 elements each
    assert tuple(wd.block_threads[:2]) == (16, 16) and tuple(wd.thread_elems[:2]) == (4, 4)
    assert lib.gb_workdiv_suggest(None, 0, 1024, 1024, 1024, ctypes.byref(wd),
                                  ctypes.byref(chosen)) == 0
    assert chosen.value == 2  # smem tiles, one element per thread
    assert tuple(wd.block_threads[:2]) == (16, 16)
    # fewer than ~4 tiles of 16 x 16 per SM: 8 x 8 tiles spread the work evenly
    assert lib.gb_workdiv_suggest(None, 0, 256, 256, 256, ctypes.byref(wd),
                                  ctypes.byref(chosen)) == 0
    assert chosen.value == 2 and tuple(wd.block_threads[:2]) == (8, 8)
    assert tuple(wd.grid_blocks[:2]) == (32, 32)
    assert lib.gb_workdiv_suggest(None, 4, 4096, 4096, 4096, ctypes.byref(wd),
                                  ctypes.byref(chosen)) == 0
    assert tuple(wd.block_threads[:2]) == (2, 2) and tuple(wd.thread_elems[:2]) == (32, 32)
    assert lib.gb_workdiv_suggest(None, 9, 8, 8, 8, ctypes.byref(wd), None) == 1


def test_device_count_without_gpu_is_an_error_not_a_crash(lib):
    n = ctypes.c_int(-1)
    st = lib.gb_device_count(ctypes.byref(n))
    if st == 0:
        pytest.skip("a CUDA device is present")
    assert st == 4 and n.value == 0  # GB_ERR_NO_DEVICE
    h = ctypes.c_void_p()
    assert lib.gb_device_get(0, ctypes.byref(h)) == 4


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_host_buffer_workspace_size(lib):
    # gb_dgemm_host stages dense device copies of A, B, C (256-byte aligned each)
    # after the emulated workspace; native precision needs only the copies
    out = ctypes.c_size_t()
    up = lambda x: (x + 255) // 256 * 256
    m, n, k = 300, 200, 129
    assert lib.gb_dgemm_host_workspace_size(0, 0, m, n, k, ctypes.byref(out)) == 0
    assert out.value == up(8 * m * k) + up(8 * k * n) + up(8 * m * n)
    emu = ctypes.c_size_t()
    assert lib.gb_dgemm_workspace_size(1, 10, m, n, k, ctypes.byref(emu)) == 0
    assert lib.gb_dgemm_host_workspace_size(1, 10, m, n, k, ctypes.byref(out)) == 0
    assert out.value == up(emu.value) + up(8 * m * k) + up(8 * k * n) + up(8 * m * n)
    assert lib.gb_dgemm_host_workspace_size(1, 17, m, n, k, ctypes.byref(out)) == 1
    assert lib.gb_dgemm_host_workspace_size(5, 0, m, n, k, ctypes.byref(out)) == 1
    assert lib.gb_dgemm_host_workspace_size(0, 0, -1, n, k, ctypes.byref(out)) == 1


def test_host_buffer_gemm_rejects_bad_arguments_before_any_device_work(lib):
    # argument errors come back before the queue or the device is touched
    P = ctypes.c_void_p
    buf = (ctypes.c_double * 16)()
    p = ctypes.cast(buf, P)
    assert lib.gb_dgemm_host(None, 1, 10, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None, 0) == 1
    fake_q = P(1)  # never dereferenced: the leading dimension check fails first
    assert lib.gb_dgemm_host(fake_q, 1, 10, 4, 4, 4, 1.0, p, 3, p, 4, 0.0, p, 4, None, 0) == 1
    assert lib.gb_dgemm_host(fake_q, 7, 10, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None, 0) == 1
    assert lib.gb_dgemm_host(fake_q, 1, 99, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None, 0) == 1


def test_library_binds_the_shared_cuda_runtime(lib):
    # the library links libcudart.so (not a private static runtime), so a caller's
    # own kernels, compiled against the same shared runtime, launch through
    # gb_enqueue; loaded alone (no PyTorch) it brings that runtime in itself
    import subprocess
    import sys
    code = ("import ctypes, sys; ctypes.CDLL(sys.argv[1]); "
            "print(any('libcudart.so' in l for l in open('/proc/self/maps')))")
    r = subprocess.run([sys.executable, "-c", code, _lib.LIB_PATH], capture_output=True,
                       text=True, check=True)
    assert r.stdout.strip() == "True"


def test_residue_workspace_pads_k_to_whole_exact_units(lib):
    # the residue precision stores its residues over K padded to whole units of
    # 256 (the products kernel's exact FP32 units, four full pipeline stages
    # each): the workspace is constant within a unit and grows by the residue
    # planes of A and B (2 bytes x 13 moduli x padded lines) per unit
    from paper_1602_08477_gb300 import workspace_size
    m, n, N = 300, 260, 13
    size = {k: workspace_size("emulated_crt", N, m, n, k) for k in (1, 17, 255, 256, 257, 511,
                                                                     512, 513)}
    assert size[1] == size[17] == size[255] == size[256]
    assert size[257] == size[511] == size[512] > size[256]
    mp, np_ = 384, 512  # rows of A padded to 128-row tiles, columns of B to 256
    assert size[257] - size[256] == 2 * N * (mp + np_) * 256
    assert size[513] - size[512] == 2 * N * (mp + np_) * 256
