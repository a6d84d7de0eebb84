"""The emulated GEMM entry point that allocates nothing (static device scratch).

Callers that cannot allocate device memory (inside an allocation-free stream
capture, under a memory pool that owns the device, or as a plug-in handed only
its buffers) use gb_dgemm_emulated_noalloc.  This test calls it through the C
ABI twice in a row and checks each result against gb_dgemm with a caller
workspace, with the same tolerance as the other parity tests (bit-exact: the
two run the same kernels on the same digits).  It lives in a file collected
last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from synth import generators as g

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    lib = gb.load()
    stream = torch.cuda.current_stream()
    cases = [(300, 200, 129, 11, "uniform", 1.5, 0.5), (513, 257, 1000, 13, "hard", 1.0, 0.0),
             (130, 97, 70, 10, "uniform", -0.75, 2.0)]
    for (m, n, k, s, kind, alpha, beta) in cases:
        A = torch.from_numpy(g.matrix(kind, m, k, 91, 0)).cuda()
        B = torch.from_numpy(g.matrix(kind, k, n, 91, 1)).cuda()
        C0 = torch.from_numpy(g.matrix(kind, m, n, 91, 2)).cuda()
        want = C0.clone()
        gb.dgemm(A, B, want, alpha, beta, precision="emulated", slices=s)
        for _ in range(2):                 # two calls in a row share the scratch
            got = C0.clone()
            st = lib.gb_dgemm_emulated_noalloc(ctypes.c_void_p(stream.cuda_stream), s, m, n, k,
                                               alpha, _ptr(A), k, _ptr(B), n, beta, _ptr(got), n)
            assert st == 0, gb._lib.last_error()
            torch.cuda.synchronize()
            assert torch.equal(got, want)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    lib = gb.load()
    n = 4096  # 2 * 11 * 4096 * 4096 bytes of digits > 64 MiB
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = lib.gb_dgemm_emulated_noalloc(None, 11, n, n, n, 1.0, _ptr(A), n, _ptr(A), n, 0.0,
                                       _ptr(C), n)
    assert st == 3  # GB_ERR_UNSUPPORTED
    assert b"scratch" in lib.gb_last_error()
