"""The emulated GEMM entry point that allocates nothing (static device scratch).

Callers that cannot allocate device memory (a memory pool that owns the device,
a plug-in handed only its buffers, a loop that cannot pay for cudaMalloc's
device synchronization) use gb_dgemm_emulated_noalloc.  This test calls it
through the C ABI twice in a row and checks each result against gb_dgemm with a
caller workspace, bit for bit (the two run the same kernels on the same
digits), and against the CPU model of the split-precision steps, also bit for
bit; the cases include the default slice count (slices = 0) and operands that
are views with leading dimensions wider than the matrix, and one call captured
in a CUDA graph and replayed twice.  It lives in a file
collected last so that a failure here leaves every other test already run.
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
    from oracle import ozaki
    gb.build()
    lib = gb.load()
    stream = torch.cuda.current_stream()
    # (m, n, k, slices, kind, alpha, beta, pad): pad > 0 makes A, B and C views
    # into wider buffers (lda = k + pad, ldb = ldc = n + pad)
    cases = [(300, 200, 129, 11, "uniform", 1.5, 0.5, 0), (513, 257, 1000, 13, "hard", 1.0, 0.0, 0),
             (130, 97, 70, 10, "uniform", -0.75, 2.0, 0), (200, 75, 90, 0, "uniform", 1.0, 0.5, 0),
             (150, 61, 77, 9, "hard", 2.0, -1.0, 5)]
    for (m, n, k, s, kind, alpha, beta, pad) in cases:
        A_h = g.matrix(kind, m, k, 91, 0)
        B_h = g.matrix(kind, k, n, 91, 1)
        C_h = g.matrix(kind, m, n, 91, 2)
        Abuf = torch.full((m, k + pad), float("nan"), dtype=torch.float64, device="cuda")
        Bbuf = torch.full((k, n + pad), float("nan"), dtype=torch.float64, device="cuda")
        A, B = Abuf[:, :k], Bbuf[:, :n]
        A.copy_(torch.from_numpy(A_h))
        B.copy_(torch.from_numpy(B_h))
        C0 = torch.from_numpy(C_h).cuda()
        want = C0.clone()
        gb.dgemm(A, B, want, alpha, beta, precision="emulated", slices=s or 11)
        model = ozaki.emulated_gemm(alpha, A_h, B_h, beta, C_h, s=s or 11)
        assert np.array_equal(want.cpu().numpy(), model)
        for _ in range(2):                 # two calls in a row share the scratch
            Cbuf = torch.full((m, n + pad), -7.0, dtype=torch.float64, device="cuda")
            got = Cbuf[:, :n]
            got.copy_(C0)
            st = lib.gb_dgemm_emulated_noalloc(ctypes.c_void_p(stream.cuda_stream), s, m, n, k,
                                               alpha, _ptr(A), k + pad, _ptr(B), n + pad, beta,
                                               _ptr(got), n + pad)
            assert st == 0, gb._lib.last_error()
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            assert bool(torch.all(Cbuf[:, n:] == -7.0))   # nothing beyond the n columns


def test_noalloc_call_captured_in_a_cuda_graph_and_replayed():
    # the case the entry point exists for: a call recorded into a CUDA graph
    # (no allocation may happen inside the capture) and replayed later
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    lib = gb.load()
    m, n, k, s, alpha, beta = 257, 190, 300, 11, 1.25, 0.5
    A = torch.from_numpy(g.matrix("uniform", m, k, 92, 0)).cuda()
    B = torch.from_numpy(g.matrix("uniform", k, n, 92, 1)).cuda()
    C0 = torch.from_numpy(g.matrix("uniform", m, n, 92, 2)).cuda()
    want = C0.clone()
    gb.dgemm(A, B, want, alpha, beta, precision="emulated", slices=s)
    C = C0.clone()
    # one plain call first: it loads the module that holds the static scratch
    st = lib.gb_dgemm_emulated_noalloc(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                       s, m, n, k, alpha, _ptr(A), k, _ptr(B), n, beta, _ptr(C), n)
    assert st == 0, gb._lib.last_error()
    torch.cuda.synchronize()
    assert torch.equal(C, want)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = lib.gb_dgemm_emulated_noalloc(
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), s, m, n, k, alpha, _ptr(A),
            k, _ptr(B), n, beta, _ptr(C), n)
    assert st == 0, gb._lib.last_error()
    for _ in range(2):
        C.copy_(C0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(C, want)


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
