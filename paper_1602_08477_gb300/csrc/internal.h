// Internal launcher interface between the C ABI (api.cpp) and the kernels.
// Not installed; the public interface is include/gb_gemm.h.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace gb {

// Bits of the per-queue device status word.
enum : unsigned {
    kStatusTimeout = 1u,    // a bounded device-side wait gave up
    kStatusNonfinite = 2u,  // the emulated path saw NaN/Inf input
};

struct Launch {
    cudaStream_t stream;
    unsigned* status;  // device status word (may be null)
    int sm_count;
};

struct Gemm {
    int64_t m, n, k;
    double alpha, beta;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
};

// ---- native FP64 kernels (dgemm_native.cu) ----
// C <- beta * C (alpha == 0 or k == 0).
cudaError_t launch_scale(const Launch& L, const Gemm& g);
// One thread per element; block by x bx threads (rows x cols).
cudaError_t launch_naive(const Launch& L, const Gemm& g, int by, int bx);
// Square shared-memory tiles of T x T (T in {8, 16, 32}), one element per thread.
cudaError_t launch_tiled(const Launch& L, const Gemm& g, int T);
// Register-tiled FP64 FMA: 16 x 16 threads with V x V elements (V in {2, 4, 8}).
cudaError_t launch_dfma(const Launch& L, const Gemm& g, int V);
// Warp-tiled DMMA: warps_m x warps_n warps, each wt_m x wt_n elements
// (supported: (2,2,32,32), (2,2,16,16), (4,2,32,32)).
cudaError_t launch_dmma(const Launch& L, const Gemm& g, int warps_m, int warps_n, int wt_m,
                        int wt_n);
bool dmma_variant_exists(int warps_m, int warps_n, int wt_m, int wt_n);

// ---- emulated FP64 (ozaki_split.cu, ozaki_gemm.cu) ----
struct EmuLayout {
    int64_t kp;
    size_t a_digits, b_digits, a_exp, b_exp, total;
};
EmuLayout emu_layout(int s, int64_t m, int64_t n, int64_t k);

cudaError_t launch_split_rows(const Launch& L, int s, int64_t m, int64_t k, const double* A,
                              int64_t lda, uint8_t* digits, int64_t kp, int32_t* exps);
cudaError_t launch_split_cols(const Launch& L, int s, int64_t n, int64_t k, const double* B,
                              int64_t ldb, uint8_t* digits, int64_t kp, int32_t* exps);
cudaError_t launch_emu_products(const Launch& L, int s, int64_t m, int64_t n, int64_t k,
                                double alpha, double beta, double* C, int64_t ldc,
                                const uint8_t* a_digits, const uint8_t* b_digits, int64_t kp,
                                const int32_t* a_exp, const int32_t* b_exp);

// Last error text helper used by launchers (thread-local in api.cpp).
void set_error(const char* fmt, ...);

}  // namespace gb
