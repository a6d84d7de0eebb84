/*
 * gb_workdiv_device.cuh -- device-side index retrieval for kernels written
 * against the grid / block / thread / element work division (Section 3.4.3,
 * "Work Division and Index Retrieval": the global n-dimensional thread index,
 * the n-dimensional thread extent and their row-major linearisation).
 *
 * Header-only CUDA; include it in kernels launched with gb_enqueue().  A work
 * division of dimension D (1..3) maps its dimension d to the CUDA axis
 * x for d = D-1 (the fastest-varying, as in row-major linearisation), y for
 * d = D-2 and z for d = D-3.  The element level (thread_elems) is the kernel's
 * own loop: pass the gb_workdiv as a kernel argument to read it.
 */
#ifndef GB_WORKDIV_DEVICE_CUH
#define GB_WORKDIV_DEVICE_CUH

#include <stdint.h>

struct gb_idx3 {
    uint64_t v[3];
};

/* CUDA axis (0 = x, 1 = y, 2 = z) of work-division dimension d out of D. */
__host__ __device__ inline int gb_axis_of_dim(int d, int D) { return D - 1 - d; }

/* Global index of the calling thread in the grid of threads, per dimension. */
__device__ inline gb_idx3 gb_get_idx_grid_threads(int D) {
    const uint64_t b[3] = {blockIdx.x, blockIdx.y, blockIdx.z};
    const uint64_t n[3] = {blockDim.x, blockDim.y, blockDim.z};
    const uint64_t t[3] = {threadIdx.x, threadIdx.y, threadIdx.z};
    gb_idx3 r = {{0, 0, 0}};
    for (int d = 0; d < D; ++d) {
        const int a = gb_axis_of_dim(d, D);
        r.v[d] = b[a] * n[a] + t[a];
    }
    return r;
}

/* Extent of the grid of threads (blocks per grid x threads per block), per dimension. */
__device__ inline gb_idx3 gb_get_workdiv_grid_threads(int D) {
    const uint64_t g[3] = {gridDim.x, gridDim.y, gridDim.z};
    const uint64_t n[3] = {blockDim.x, blockDim.y, blockDim.z};
    gb_idx3 r = {{1, 1, 1}};
    for (int d = 0; d < D; ++d) {
        const int a = gb_axis_of_dim(d, D);
        r.v[d] = g[a] * n[a];
    }
    return r;
}

/* Row-major linearisation of an index within an extent (the 1-dimensional map). */
__host__ __device__ inline uint64_t gb_map_idx_1(gb_idx3 idx, gb_idx3 extent, int D) {
    uint64_t lin = 0;
    for (int d = 0; d < D; ++d) lin = lin * extent.v[d] + idx.v[d];
    return lin;
}

#endif /* GB_WORKDIV_DEVICE_CUH */
