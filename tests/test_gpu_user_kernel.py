"""The generic executor launches a kernel the caller compiled itself.

The paper's executor binds any kernel, a work division and the kernel's
arguments and enqueues them on a queue (Section 3.4.6, "Kernel Execution"); the
kernel reads its indices through the work-division index functions (Section
3.4.3, "Work Division and Index Retrieval").  Here a caller-side CUDA source,
unknown to the library, is compiled by nvcc into its own shared library (linked
against the shared CUDA runtime, like the library), and its kernel handle is
enqueued through gb_enqueue with two-dimensional work divisions whose element
level is the kernel's own loop over thread_elems.  The results are integers,
so they are checked bit-exactly against NumPy.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from synth import generators as g

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

USER_SOURCE = r"""
#include <stdint.h>
#include "gb_gemm.h"
#include "gb_workdiv_device.cuh"

// out[i][j] = 2 in[i][j] + (i * cols + j) over a rows x cols matrix; every
// thread covers thread_elems[0] x thread_elems[1] elements, and records its
// linear thread index (the 1-dimensional map of its 2-dimensional index) at
// its row-major position in the grid of threads.
__global__ void user_scale_add_2d(gb_workdiv wd, int64_t rows, int64_t cols,
                                  const double* in, double* out, int64_t* lin) {
    const gb_idx3 t = gb_get_idx_grid_threads(2);
    const gb_idx3 ext = gb_get_workdiv_grid_threads(2);
    lin[t.v[0] * ext.v[1] + t.v[1]] = (int64_t)gb_map_idx_1(t, ext, 2);
    for (uint64_t e0 = 0; e0 < wd.thread_elems[0]; ++e0) {
        for (uint64_t e1 = 0; e1 < wd.thread_elems[1]; ++e1) {
            const uint64_t i = t.v[0] * wd.thread_elems[0] + e0;
            const uint64_t j = t.v[1] * wd.thread_elems[1] + e1;
            if (i < (uint64_t)rows && j < (uint64_t)cols)
                out[i * cols + j] = 2.0 * in[i * cols + j] + (double)(i * cols + j);
        }
    }
}

extern "C" const void* user_kernel_handle(void) {
    return (const void*)&user_scale_add_2d;
}
"""


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    import paper_1602_08477_gb300 as gb
    from paper_1602_08477_gb300 import compile_lib
    gb.build()
    gb.load()
    d = tmp_path_factory.mktemp("userkernel")
    src = d / "user.cu"
    src.write_text(USER_SOURCE)
    so = d / "libuser.so"
    nvcc = compile_lib._nvcc()
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "--cudart", "shared", "-I",
                    os.path.join(ROOT, "include"), "-o", str(so), str(src)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.user_kernel_handle.restype = ctypes.c_void_p
    return lib


@pytest.mark.parametrize("rows,cols,grid,block,elems", [
    (37, 100, (3, 2), (4, 32), (4, 2)),     # 48 x 128 threads-by-elements cover 37 x 100
    (5, 1000, (5, 1), (1, 256), (1, 4)),    # one row per block
    (64, 64, (2, 4), (8, 16), (4, 1)),      # exact cover
])
def test_user_kernel_through_gb_enqueue(user_lib, rows, cols, grid, block, elems):
    import torch
    import paper_1602_08477_gb300 as gb
    handle = user_lib.user_kernel_handle()
    assert handle
    x = g.matrix("int8", rows, cols, 77, 0)
    dx = torch.from_numpy(x).cuda()
    dout = torch.full((rows, cols), float("nan"), dtype=torch.float64, device="cuda")
    nthreads = [grid[d] * block[d] for d in range(2)]
    dlin = torch.full((nthreads[0] * nthreads[1],), -1, dtype=torch.int64, device="cuda")
    wd = gb.Workdiv.make(list(grid), list(block), list(elems))
    P = ctypes.c_void_p
    gb.enqueue(handle, wd, [wd, ctypes.c_int64(rows), ctypes.c_int64(cols), P(dx.data_ptr()),
                            P(dout.data_ptr()), P(dlin.data_ptr())])
    torch.cuda.synchronize()
    want = 2.0 * x + np.arange(rows * cols, dtype=np.float64).reshape(rows, cols)
    assert np.array_equal(dout.cpu().numpy(), want)
    # every thread of the work division ran once, at its row-major linear index
    assert np.array_equal(dlin.cpu().numpy(), np.arange(nthreads[0] * nthreads[1]))
