// Emulated FP64 GEMM for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a GEMM:
// programs whose custom allocator or memory pool owns every byte of the
// device, plug-ins that are handed only the buffers of their inputs and
// outputs, and latency-bound loops that cannot afford cudaMalloc / cudaFree,
// which may synchronize the device.  The emulated path needs scratch memory for
// its digit planes and exponents, so this entry point takes that scratch from
// one file-scope __device__ array of fixed size instead of a caller workspace.
//
// The array is kNoAllocScratchBytes (64 MiB) per GPU, held until the process
// exits; with lazy module loading it is reserved when the first call on a
// device loads this file's module.  Host code cannot pass the array's name to
// a kernel (on the host it names a stand-in, not device memory), so the first
// call on each device, with that device current, looks up its device address
// once with cudaGetSymbolAddress and keeps it.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "gb_gemm.h"
#include "internal.h"

namespace gb {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
std::atomic<void*> g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(int dev, void** out) {
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" gb_status gb_dgemm_emulated_noalloc(void* cuda_stream, int slices, int64_t m,
                                               int64_t n, int64_t k, double alpha,
                                               const double* A, int64_t lda, const double* B,
                                               int64_t ldb, double beta, double* C,
                                               int64_t ldc) {
    const int v = validate_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    if (v != GB_OK) return (gb_status)v;
    const int s = slices == 0 ? 11 : slices;
    if (s < 1 || s > 16) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    if (m == 0 || n == 0) return GB_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("no usable current device: %s", cudaGetErrorString(e));
        return GB_ERR_NO_DEVICE;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_error("cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        return GB_ERR_CUDA;
    }
    const Launch L{static_cast<cudaStream_t>(cuda_stream), nullptr, sms};
    const Gemm g{m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
    if (alpha == 0.0 || k == 0) {
        e = launch_scale(L, g);
        if (e != cudaSuccess) {
            set_error("C <- beta C: %s", cudaGetErrorString(e));
            return GB_ERR_CUDA;
        }
        return GB_OK;
    }
    const EmuLayout lay = emu_layout(s, m, n, k);
    if (lay.total > kNoAllocScratchBytes) {
        set_error("this GEMM needs %zu bytes of scratch (s = %d, m = %lld, n = %lld, k = %lld); "
                  "the static scratch holds %zu bytes: use gb_dgemm with a workspace",
                  lay.total, s, (long long)m, (long long)n, (long long)k, kNoAllocScratchBytes);
        return GB_ERR_UNSUPPORTED;
    }
    void* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) {
        set_error("cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        return GB_ERR_CUDA;
    }
    uint8_t* ws = static_cast<uint8_t*>(base);
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    // The split kernels write every byte of the layout (digit padding included),
    // so nothing left by an earlier call needs clearing.
    e = launch_split_rows(L, s, m, k, A, lda, ws + lay.a_digits, lay.kp, ea);
    if (e == cudaSuccess)
        e = launch_split_cols(L, s, n, k, B, ldb, ws + lay.b_digits, lay.kp, fb,
                              reinterpret_cast<uint64_t*>(ws + lay.b_part));
    if (e == cudaSuccess)
        e = launch_emu_products(L, s, m, n, k, alpha, beta, C, ldc, ws + lay.a_digits,
                                ws + lay.b_digits, lay.kp, ea, fb);
    if (e != cudaSuccess) {
        set_error("emulated dgemm (static scratch): %s", cudaGetErrorString(e));
        return GB_ERR_CUDA;
    }
    return GB_OK;
}
