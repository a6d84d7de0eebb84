// The generic work-division executor (gb_enqueue) and DAXPY (include/gb_exec.h).
//
// DAXPY Y <- alpha X + Y (Section 4.1) with the CUDA row of Table 2: a block of B
// threads covers B * V consecutive elements, thread t the V elements
// [t V, t V + V) of its block's span (V-wide vector loads when aligned), one
// fused multiply-add per element.  On GB300 a separate multiply and add would
// take ~90% of the FP64 pipe at HBM speed; the fused form keeps it memory-bound.
#include <cuda_runtime.h>

#include <cstring>

#include "gb_exec.h"
#include "gb_workdiv_device.cuh"
#include "handles.h"
#include "internal.h"

namespace gb {
namespace {

template <int V>
__global__ void daxpy_kernel(int64_t n, double alpha, const double* __restrict__ x,
                             double* __restrict__ y) {
    const gb_idx3 t = gb_get_idx_grid_threads(1);
    const gb_idx3 ext = gb_get_workdiv_grid_threads(1);
    const bool vec = V % 2 == 0 && ((reinterpret_cast<uintptr_t>(x) |
                                     reinterpret_cast<uintptr_t>(y)) & 15) == 0;
    // element level: V consecutive elements per thread; the grid-stride loop lets
    // a work division smaller than n / V still cover every element
    for (int64_t i0 = (int64_t)gb_map_idx_1(t, ext, 1) * V; i0 < n;
         i0 += (int64_t)ext.v[0] * V) {
        if (vec && i0 + V <= n) {
#pragma unroll
            for (int u = 0; u < V; u += 2) {
                const double2 a = *reinterpret_cast<const double2*>(x + i0 + u);
                double2 b = *reinterpret_cast<const double2*>(y + i0 + u);
                b.x = fma(alpha, a.x, b.x);
                b.y = fma(alpha, a.y, b.y);
                *reinterpret_cast<double2*>(y + i0 + u) = b;
            }
        } else {
#pragma unroll
            for (int u = 0; u < V; ++u)
                if (i0 + u < n) y[i0 + u] = fma(alpha, x[i0 + u], y[i0 + u]);
        }
    }
}

const void* daxpy_handle(int V) {
    switch (V) {
        case 1: return reinterpret_cast<const void*>(&daxpy_kernel<1>);
        case 2: return reinterpret_cast<const void*>(&daxpy_kernel<2>);
        case 4: return reinterpret_cast<const void*>(&daxpy_kernel<4>);
        case 8: return reinterpret_cast<const void*>(&daxpy_kernel<8>);
        default: return nullptr;
    }
}

gb_status bad_wd(const char* msg) {
    set_error("work division: %s", msg);
    return GB_ERR_INVALID_WORKDIV;
}

// CUDA launch shape of a work division (dimension d on axis D-1-d).
gb_status launch_shape(const gb_workdiv* wd, dim3* grid, dim3* block) {
    if (wd->dim < 1 || wd->dim > 3) return bad_wd("dim must be 1, 2 or 3");
    uint64_t g[3] = {1, 1, 1}, b[3] = {1, 1, 1};
    for (uint32_t d = 0; d < wd->dim; ++d) {
        if (wd->grid_blocks[d] == 0 || wd->block_threads[d] == 0 || wd->thread_elems[d] == 0)
            return bad_wd("every extent must be at least 1");
        const int a = (int)wd->dim - 1 - (int)d;
        g[a] = wd->grid_blocks[d];
        b[a] = wd->block_threads[d];
    }
    if (b[0] * b[1] * b[2] > 1024) return bad_wd("more than 1024 threads per block");
    if (b[2] > 64) return bad_wd("block z extent above 64");
    if (g[0] > 2147483647ull || g[1] > 65535 || g[2] > 65535) return bad_wd("grid extent above the CUDA limit");
    *grid = dim3((unsigned)g[0], (unsigned)g[1], (unsigned)g[2]);
    *block = dim3((unsigned)b[0], (unsigned)b[1], (unsigned)b[2]);
    return GB_OK;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

const void* gb_kernel_handle(const char* name) {
    if (!name) return nullptr;
    if (!std::strcmp(name, "daxpy_v1")) return daxpy_handle(1);
    if (!std::strcmp(name, "daxpy_v2")) return daxpy_handle(2);
    if (!std::strcmp(name, "daxpy_v4")) return daxpy_handle(4);
    if (!std::strcmp(name, "daxpy_v8")) return daxpy_handle(8);
    return native_kernel_handle(name);
}

gb_status gb_enqueue(gb_queue* q, const gb_workdiv* wd, const void* kernel, void** args,
                     size_t shared_bytes) {
    if (!q || !wd || !kernel) {
        set_error("gb_enqueue: queue, work division or kernel is NULL");
        return GB_ERR_INVALID_ARG;
    }
    dim3 grid, block;
    gb_status st = launch_shape(wd, &grid, &block);
    if (st != GB_OK) return st;
    DeviceScope scope(q->dev->idx);
    cudaError_t e = cudaLaunchKernel(kernel, grid, block, args, shared_bytes, q->stream);
    return finish_call(q, e, "gb_enqueue");
}

gb_status gb_daxpy(gb_queue* q, const gb_workdiv* wd, int64_t n, double alpha, const double* x,
                   double* y) {
    if (!q) {
        set_error("queue is NULL");
        return GB_ERR_INVALID_ARG;
    }
    if (n < 0) {
        set_error("n must be >= 0");
        return GB_ERR_INVALID_ARG;
    }
    if (n == 0 || alpha == 0.0) return GB_OK;
    if (!x || !y || (reinterpret_cast<uintptr_t>(x) & 7) || (reinterpret_cast<uintptr_t>(y) & 7)) {
        set_error("x or y is NULL or not 8-byte aligned");
        return GB_ERR_INVALID_ARG;
    }
    if (!(alpha == alpha)) {
        set_error("alpha is NaN");
        return GB_ERR_INVALID_ARG;
    }
    gb_workdiv w;
    if (wd) {
        w = *wd;
        if (w.dim != 1) return bad_wd("DAXPY takes a 1-dimensional work division");
        const uint64_t B = w.block_threads[0], V = w.thread_elems[0];
        if (B == 0 || B % 32 || B > 1024 || !daxpy_handle((int)V) || w.grid_blocks[0] == 0)
            return bad_wd("DAXPY needs B a multiple of 32 up to 1024 and V in {1, 2, 4, 8}");
        if (w.grid_blocks[0] * B * V < (uint64_t)n) return bad_wd("does not cover n");
    } else {
        std::memset(&w, 0, sizeof(w));
        w.dim = 1;
        w.block_threads[0] = 256;
        w.thread_elems[0] = 4;
        w.grid_blocks[0] = (uint64_t)((n + 1023) / 1024);
        for (int d = 1; d < 3; ++d) w.grid_blocks[d] = w.block_threads[d] = w.thread_elems[d] = 1;
    }
    const void* k = daxpy_handle((int)w.thread_elems[0]);
    void* args[4] = {&n, &alpha, const_cast<double**>(&x), &y};
    return gb_enqueue(q, &w, k, args, 0);
}

}  // extern "C"
