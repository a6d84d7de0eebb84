/*
 * gb_exec.h -- the generic work-division executor and DAXPY (C ABI).
 *
 * gb_enqueue binds a work division, a kernel and its arguments and enqueues the
 * execution on a queue (Section 3.4.6, "Kernel Execution": an executor binds an
 * accelerator, a work division, a kernel and its parameters and is enqueued
 * into a stream).  gb_daxpy is the paper's vector workload Y <- alpha X + Y
 * (Section 4.1, "Conceptual Comparison") over the same work division: blocks =
 * N / (B V), threads per block B, elements per thread V (Table 2, CUDA row).
 * Conventions and errors as in gb_gemm.h.
 */
#ifndef GB_EXEC_H
#define GB_EXEC_H

#include "gb_gemm.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Enqueue `kernel` (the host-side handle of a __global__ function of this
 * process: a CUDA runtime kernel pointer, or one returned by gb_kernel_handle)
 * on q with the work division wd and the argument array `args` (one pointer per
 * kernel parameter, as cudaLaunchKernel takes them) and `shared_bytes` of
 * dynamic shared memory.  The library uses the shared CUDA runtime
 * (libcudart.so.13): a kernel compiled into the caller's own module is found
 * when that module links the same shared runtime (nvcc --cudart shared), so
 * that its kernels register where the library launches them.  Dimension d of a D-dimensional work division runs on
 * the CUDA axis x for d = D-1, y for d = D-2, z for d = D-3
 * (include/gb_workdiv_device.cuh gives the matching device-side index
 * functions); the element level is the kernel's own loop.
 * Errors: GB_ERR_INVALID_ARG (NULL queue, kernel or args with parameters),
 * GB_ERR_INVALID_WORKDIV (dim not 1..3, a zero extent, more than 1024 threads
 * per block, block z > 64, grid y or z > 65535), GB_ERR_CUDA (launch failure).
 */
gb_status gb_enqueue(gb_queue* q, const gb_workdiv* wd, const void* kernel, void** args,
                     size_t shared_bytes);

/* Host-side handle of one of the library's own kernels usable with gb_enqueue,
 * or NULL.  Names: "daxpy_v1", "daxpy_v2", "daxpy_v4", "daxpy_v8" -- the DAXPY
 * kernel with V elements per thread, parameters
 * (int64_t n, double alpha, const double* x, double* y);  "dgemm_naive"
 * (16 x 16 threads, 1 element each), "dgemm_tiled16" (16 x 16 threads, 16 x 16
 * shared-memory tiles), "dgemm_dfma4" (16 x 16 threads, 4 x 4 elements each) --
 * the native DGEMM kernels, parameters (int64_t m, n, k, double alpha,
 * const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
 * double* C, int64_t ldc), grid (ceil(n / tile), ceil(m / tile)) on x, y. */
const void* gb_kernel_handle(const char* name);

/*
 * Y <- alpha X + Y for n doubles (x, y device pointers, 8-byte aligned; the
 * vector path needs 16-byte alignment), each element with one rounding
 * (fused multiply-add).  alpha == 0 leaves Y unread and unchanged; n == 0 is a
 * no-op.  wd: 1-dimensional work division (block threads a multiple of 32 up to
 * 1024, elements per thread 1, 2, 4 or 8, covering n), or NULL for the
 * library's (B = 256, V = 4).
 */
gb_status gb_daxpy(gb_queue* q, const gb_workdiv* wd, int64_t n, double alpha, const double* x,
                   double* y);

#ifdef __cplusplus
}
#endif

#endif /* GB_EXEC_H */
