// C ABI of the library (include/gb_gemm.h): devices, queues, work divisions and
// the FP64 GEMM.  Every argument is validated here, on the host, before anything
// is enqueued; no call throws or aborts across the ABI.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "gb_gemm.h"
#include "handles.h"
#include "internal.h"

namespace gb {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

gb_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return GB_ERR_CUDA;
}

namespace {

gb_status invalid(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return GB_ERR_INVALID_ARG;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// Reads and clears the queue's device status word (after the stream finished).
gb_status drain_status(gb_queue* q) {
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, q->status, sizeof(h), cudaMemcpyDeviceToHost, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the queue status");
    if (h == 0) return GB_OK;
    e = cudaMemsetAsync(q->status, 0, sizeof(unsigned), q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the queue status");
    if (h & kStatusTimeout) {
        set_error("a device-side wait timed out");
        return GB_ERR_TIMEOUT;
    }
    set_error("the emulated path found NaN/Inf in A or B; affected outputs are NaN");
    return GB_ERR_NONFINITE;
}

gb_status finish_call(gb_queue* q, cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!q->blocking) return GB_OK;
    e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return drain_status(q);
}

namespace {

Launch launch_of(const gb_queue* q) { return Launch{q->stream, q->status, q->dev->sm_count}; }

// ---- work divisions ----------------------------------------------------------------
struct Variant {
    gb_kernel kernel;
    uint64_t bt0, bt1;  // block_threads (rows, cols)
    uint64_t te0, te1;  // thread_elems (rows, cols)
};

uint64_t cdiv(int64_t a, uint64_t b) { return (uint64_t)((a + (int64_t)b - 1) / (int64_t)b); }

void fill_workdiv(gb_workdiv* wd, const Variant& v, int64_t m, int64_t n) {
    std::memset(wd, 0, sizeof(*wd));
    wd->dim = 2;
    wd->block_threads[0] = v.bt0;
    wd->block_threads[1] = v.bt1;
    wd->thread_elems[0] = v.te0;
    wd->thread_elems[1] = v.te1;
    wd->grid_blocks[0] = cdiv(m > 0 ? m : 1, v.bt0 * v.te0);
    wd->grid_blocks[1] = cdiv(n > 0 ? n : 1, v.bt1 * v.te1);
    for (int d = 2; d < 3; ++d) wd->grid_blocks[d] = wd->block_threads[d] = wd->thread_elems[d] = 1;
}

// The library's default variant per kernel family and size.
Variant default_variant(gb_kernel kernel, int64_t m, int64_t n, int64_t k) {
    (void)k;
    const int64_t mn = m < n ? m : n;
    switch (kernel) {
        case GB_KERNEL_NAIVE: return {kernel, 16, 16, 1, 1};
        case GB_KERNEL_TILED: return {kernel, 16, 16, 1, 1};
        case GB_KERNEL_DFMA: return {kernel, 16, 16, 4, 4};
        case GB_KERNEL_DMMA:
            // a warp is one "thread"; its 32 x 32 (or 16 x 16) register tile the elements
            if (mn <= 1024) return {GB_KERNEL_DMMA, 2, 2, 16, 16};
            return {GB_KERNEL_DMMA, 2, 2, 32, 32};
        case GB_KERNEL_AUTO:
        default: {
            // measured on GB300: one element per thread in 16 x 16 smem tiles is
            // fastest up to 2048 (finest load balance over 152 SMs); above it the
            // 4 x 4 register tiles run the FP64 FMA pipe at its peak.  With fewer
            // than ~4 tiles of 16 x 16 per SM the SMs get unequal tile counts
            // (n = 256: 256 tiles, 2 or 1 per SM), so 8 x 8 tiles even them out
            // (n = 256: 36.9 -> 32.9 us; n = 512 stays faster with 16 x 16).
            const int64_t tiles16 = ((m + 15) / 16) * ((n + 15) / 16);
            if (tiles16 < 600) return {GB_KERNEL_TILED, 8, 8, 1, 1};
            if (mn <= 2048) return {GB_KERNEL_TILED, 16, 16, 1, 1};
            return {GB_KERNEL_DFMA, 16, 16, 4, 4};
        }
    }
}

gb_status check_workdiv(const gb_workdiv* wd, gb_kernel kernel, int64_t m, int64_t n) {
    if (wd->dim != 2) {
        set_error("work division: dim must be 2 (rows, cols), got %u", wd->dim);
        return GB_ERR_INVALID_WORKDIV;
    }
    for (int d = 0; d < 2; ++d) {
        if (wd->grid_blocks[d] == 0 || wd->block_threads[d] == 0 || wd->thread_elems[d] == 0) {
            set_error("work division: zero extent in dimension %d", d);
            return GB_ERR_INVALID_WORKDIV;
        }
    }
    const uint64_t ext[2] = {(uint64_t)m, (uint64_t)n};
    for (int d = 0; d < 2; ++d) {
        const uint64_t cover = wd->grid_blocks[d] * wd->block_threads[d] * wd->thread_elems[d];
        if (cover < ext[d]) {
            set_error("work division does not cover C: dimension %d covers %llu < %llu", d,
                      (unsigned long long)cover, (unsigned long long)ext[d]);
            return GB_ERR_INVALID_WORKDIV;
        }
    }
    const uint64_t by = wd->block_threads[0], bx = wd->block_threads[1];
    const uint64_t ey = wd->thread_elems[0], ex = wd->thread_elems[1];
    bool ok = false;
    switch (kernel) {
        case GB_KERNEL_NAIVE:
            ok = ey == 1 && ex == 1 && by * bx <= 1024 && bx <= 1024 && by <= 1024 &&
                 wd->grid_blocks[0] <= 65535;
            break;
        case GB_KERNEL_TILED:
            ok = ey == 1 && ex == 1 && by == bx && (bx == 8 || bx == 16 || bx == 32) &&
                 wd->grid_blocks[0] <= 65535;
            break;
        case GB_KERNEL_DFMA:
            ok = by == 16 && bx == 16 && ey == ex && (ex == 2 || ex == 4 || ex == 8) &&
                 wd->grid_blocks[0] <= 65535;
            break;
        case GB_KERNEL_DMMA:
            ok = dmma_variant_exists((int)by, (int)bx, (int)ey, (int)ex) &&
                 wd->grid_blocks[0] <= 65535;
            break;
        default: break;
    }
    if (!ok) {
        set_error("no compiled variant of kernel %d has block (%llu, %llu) x elements (%llu, %llu)",
                  (int)kernel, (unsigned long long)by, (unsigned long long)bx,
                  (unsigned long long)ey, (unsigned long long)ex);
        return GB_ERR_INVALID_WORKDIV;
    }
    return GB_OK;
}

gb_status check_gemm_args(int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                          int64_t lda, const double* B, int64_t ldb, double beta,
                          const double* C, int64_t ldc) {
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0 (got %lld, %lld, %lld)",
                                                 (long long)m, (long long)n, (long long)k);
    if (lda < (k > 1 ? k : 1)) return invalid("lda = %lld < max(1, k = %lld)", (long long)lda, (long long)k);
    if (ldb < (n > 1 ? n : 1)) return invalid("ldb = %lld < max(1, n = %lld)", (long long)ldb, (long long)n);
    if (ldc < (n > 1 ? n : 1)) return invalid("ldc = %lld < max(1, n = %lld)", (long long)ldc, (long long)n);
    if (m == 0 || n == 0) return GB_OK;
    if (!C) return invalid("C is NULL");
    if (!aligned(C, 8)) return invalid("C is not 8-byte aligned");
    const bool reads_ab = alpha != 0.0 && k > 0;
    if (reads_ab && (!A || !B)) return invalid("A or B is NULL while alpha != 0 and k > 0");
    if (reads_ab && (!aligned(A, 8) || !aligned(B, 8))) return invalid("A or B is not 8-byte aligned");
    if (!(alpha == alpha) || !(beta == beta)) return invalid("alpha or beta is NaN");
    (void)beta;
    return GB_OK;
}

int resolve_slices(int slices) { return slices == 0 ? 11 : slices; }

}  // namespace

int validate_gemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, const double* C, int64_t ldc) {
    return (int)check_gemm_args(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

bool emu_group_trans(int s, int64_t m, int64_t n) {
    const int64_t bn = emu_bn(s);
    auto pad = [](int64_t x, int64_t r) { return (x + r - 1) / r * r; };
    return pad(n, kEmuBM) * pad(m, bn) < pad(m, kEmuBM) * pad(n, bn);
}

EmuLayout emu_group_layout(int s, int64_t m, int64_t n, int64_t k, bool trans) {
    return trans ? emu_layout(s, n, m, k, false) : emu_layout(s, m, n, k, false);
}

void emu_group_assign(EmuProb& e, uint8_t* base, const EmuLayout& w) {
    uint8_t* row_side = base + w.a_digits;  // 128-line tiles
    uint8_t* col_side = base + w.b_digits;  // emu_bn(s)-line tiles
    int32_t* row_exp = reinterpret_cast<int32_t*>(base + w.a_exp);
    int32_t* col_exp = reinterpret_cast<int32_t*>(base + w.b_exp);
    e.a_digits = e.trans ? col_side : row_side;
    e.b_digits = e.trans ? row_side : col_side;
    e.a_exp = e.trans ? col_exp : row_exp;
    e.b_exp = e.trans ? row_exp : col_exp;
    e.ra = e.trans ? emu_bn(e.s) : kEmuBM;
    e.rb = e.trans ? kEmuBM : emu_bn(e.s);
}

EmuLayout emu_layout(int s, int64_t m, int64_t n, int64_t k, bool colmax_scratch) {
    EmuLayout L{};
    L.kp = ((k + 31) / 32) * 32;
    if (L.kp == 0) L.kp = 32;
    auto up = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t off = 0;
    const size_t mp = (size_t)((m + kEmuBM - 1) / kEmuBM) * kEmuBM;
    L.bn = emu_bn(s);
    const size_t np = (size_t)((n + L.bn - 1) / L.bn) * L.bn;
    L.a_digits = off;
    off = up(off + (size_t)s * mp * (size_t)L.kp);
    L.b_digits = off;
    off = up(off + (size_t)s * np * (size_t)L.kp);
    L.a_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)m);
    L.b_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)n);
    L.b_part = off;
    if (colmax_scratch) off = up(off + sizeof(uint64_t) * (size_t)kColmaxParts * (size_t)n);
    L.total = off;
    return L;
}


EmuLayout emu_layout_bf16(int s, int64_t m, int64_t n, int64_t k) {
    EmuLayout L{};
    L.kp = ((k + 15) / 16) * 16;
    if (L.kp == 0) L.kp = 16;
    auto up = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t off = 0;
    const size_t mp = (size_t)((m + kEmuBM - 1) / kEmuBM) * kEmuBM;
    L.bn = kBf16BN;
    const size_t np = (size_t)((n + L.bn - 1) / L.bn) * L.bn;
    L.a_digits = off;
    off = up(off + 2 * (size_t)s * mp * (size_t)L.kp);
    L.b_digits = off;
    off = up(off + 2 * (size_t)s * np * (size_t)L.kp);
    L.a_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)m);
    L.b_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)n);
    L.b_part = off;
    off = up(off + sizeof(uint64_t) * (size_t)kColmaxParts * (size_t)n);
    L.total = off;
    return L;
}

}  // namespace gb

using namespace gb;

// Slice count of the BF16-digit precision: 0 selects 7 (55 bits of each line).
static int resolve_bf16_slices(int slices) { return slices == 0 ? 7 : slices; }
// Moduli of the residue precision: 0 selects 13.
static int resolve_crt_moduli(int slices) { return slices == 0 ? kCrtDefaultModuli : slices; }

extern "C" {

int gb_version(void) { return 100; }

const char* gb_last_error(void) { return gb::g_err; }

gb_status gb_device_count(int* n) {
    if (!n) return invalid("n is NULL");
    int c = 0;
    cudaError_t e = cudaGetDeviceCount(&c);
    if (e != cudaSuccess || c == 0) {
        *n = 0;
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        return GB_ERR_NO_DEVICE;
    }
    *n = c;
    return GB_OK;
}

gb_status gb_device_get(int idx, gb_device** out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    int c = 0;
    if (cudaGetDeviceCount(&c) != cudaSuccess || idx < 0 || idx >= c) {
        set_error("device index %d out of range (count %d)", idx, c);
        return GB_ERR_NO_DEVICE;
    }
    cudaDeviceProp p;
    cudaError_t e = cudaGetDeviceProperties(&p, idx);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    gb_device* d = new (std::nothrow) gb_device{idx, p.multiProcessorCount, p.major, p.minor};
    if (!d) return invalid("out of host memory");
    *out = d;
    return GB_OK;
}

gb_status gb_device_info(const gb_device* dev, int* sm_count, int* cc_major, int* cc_minor) {
    if (!dev) return invalid("dev is NULL");
    if (sm_count) *sm_count = dev->sm_count;
    if (cc_major) *cc_major = dev->cc_major;
    if (cc_minor) *cc_minor = dev->cc_minor;
    return GB_OK;
}

gb_status gb_device_release(gb_device* dev) {
    delete dev;
    return GB_OK;
}

gb_status gb_queue_create(gb_device* dev, void* cuda_stream, int blocking, gb_queue** out) {
    if (!dev || !out) return invalid("dev or out is NULL");
    *out = nullptr;
    DeviceScope scope(dev->idx);
    if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    unsigned* st = nullptr;
    cudaError_t e = cudaMalloc(&st, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "allocating the queue status word");
    e = cudaMemset(st, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(st);
        return cuda_fail(e, "clearing the queue status word");
    }
    gb_queue* q = new (std::nothrow) gb_queue{dev, (cudaStream_t)cuda_stream, blocking, st, false};
    if (!q) {
        cudaFree(st);
        return invalid("out of host memory");
    }
    *out = q;
    return GB_OK;
}

gb_status gb_queue_wait(gb_queue* q) {
    if (!q) return invalid("q is NULL");
    DeviceScope scope(q->dev->idx);
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return drain_status(q);
}

void* gb_queue_stream(const gb_queue* q) { return q ? (void*)q->stream : nullptr; }

gb_status gb_queue_destroy(gb_queue* q) {
    if (!q) return GB_OK;
    DeviceScope scope(q->dev->idx);
    cudaStreamSynchronize(q->stream);
    release_aux(q);
    cudaFree(q->status);
    if (q->owns_stream) cudaStreamDestroy(q->stream);
    delete q;
    return GB_OK;
}

gb_status gb_workdiv_suggest(const gb_device* dev, gb_kernel kernel, int64_t m, int64_t n,
                             int64_t k, gb_workdiv* out, gb_kernel* chosen) {
    if (!out) return invalid("out is NULL");
    (void)dev;
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    if (kernel < GB_KERNEL_AUTO || kernel > GB_KERNEL_DMMA) return invalid("unknown kernel %d", (int)kernel);
    const Variant v = default_variant(kernel, m, n, k);
    fill_workdiv(out, v, m, n);
    if (chosen) *chosen = v.kernel;
    return GB_OK;
}

gb_status gb_dgemm_workspace_size(gb_precision prec, int slices, int64_t m, int64_t n,
                                  int64_t k, size_t* out) {
    if (!out) return invalid("out is NULL");
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    if (prec == GB_PREC_NATIVE) {
        *out = 0;
        return GB_OK;
    }
    if (prec == GB_PREC_EMULATED_BF16) {
        const int s = resolve_bf16_slices(slices);
        if (s < 1 || s > kBf16MaxSlices)
            return invalid("BF16-digit slices must be in [1, %d] (or 0 for the default), got %d",
                           kBf16MaxSlices, slices);
        *out = emu_layout_bf16(s, m, n, k).total;
        return GB_OK;
    }
    if (prec == GB_PREC_EMULATED_CRT) {
        const int N = resolve_crt_moduli(slices);
        if (N < 1 || N > kCrtMaxModuli)
            return invalid("the number of moduli must be in [1, %d] (or 0 for the default), got %d",
                           kCrtMaxModuli, slices);
        *out = crt_layout(N, m, n, k).total;
        return GB_OK;
    }
    if (prec != GB_PREC_EMULATED) return invalid("unknown precision %d", (int)prec);
    const int s = resolve_slices(slices);
    if (s < 1 || s > 16) return invalid("slices must be in [1, 16] (or 0 for the default), got %d", slices);
    *out = emu_layout(s, m, n, k).total;
    return GB_OK;
}

gb_status gb_emulated_layout_get(int slices, int64_t m, int64_t n, int64_t k,
                                 gb_emulated_layout* out) {
    if (!out) return invalid("out is NULL");
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    const int s = resolve_slices(slices);
    if (s < 1 || s > 16) return invalid("slices must be in [1, 16], got %d", slices);
    const EmuLayout L = emu_layout(s, m, n, k);
    out->kp = L.kp;
    out->a_digits = L.a_digits;
    out->b_digits = L.b_digits;
    out->a_exp = L.a_exp;
    out->b_exp = L.b_exp;
    out->total = L.total;
    out->a_tile_rows = kEmuBM;
    out->b_tile_rows = L.bn;
    return GB_OK;
}

static gb_status check_workspace_layout(const EmuLayout& L, void* ws, size_t bytes) {
    if (!ws) {
        set_error("the emulated path needs a workspace of %zu bytes", L.total);
        return GB_ERR_WORKSPACE;
    }
    if (!aligned(ws, 256)) {
        set_error("workspace must be 256-byte aligned");
        return GB_ERR_WORKSPACE;
    }
    if (bytes < L.total) {
        set_error("workspace of %zu bytes < required %zu", bytes, L.total);
        return GB_ERR_WORKSPACE;
    }
    return GB_OK;
}

static gb_status check_workspace(int s, int64_t m, int64_t n, int64_t k, void* ws, size_t bytes) {
    return check_workspace_layout(emu_layout(s, m, n, k), ws, bytes);
}

gb_status gb_emulated_split_a(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                              const double* A, int64_t lda, void* workspace,
                              size_t workspace_bytes) {
    if (!q) return invalid("q is NULL");
    const int s = resolve_slices(slices);
    if (s < 1 || s > 16) return invalid("slices must be in [1, 16], got %d", slices);
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    if (lda < (k > 1 ? k : 1)) return invalid("lda < max(1, k)");
    if (m > 0 && k > 0 && (!A || !aligned(A, 8))) return invalid("A is NULL or misaligned");
    gb_status st = check_workspace(s, m, n, k, workspace, workspace_bytes);
    if (st != GB_OK) return st;
    DeviceScope scope(q->dev->idx);
    const EmuLayout L = emu_layout(s, m, n, k);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e = launch_split_rows(launch_of(q), s, m, k, A, lda, ws + L.a_digits, L.kp,
                                      reinterpret_cast<int32_t*>(ws + L.a_exp));
    return finish_call(q, e, "split of A");
}

gb_status gb_emulated_split_b(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                              const double* B, int64_t ldb, void* workspace,
                              size_t workspace_bytes) {
    if (!q) return invalid("q is NULL");
    const int s = resolve_slices(slices);
    if (s < 1 || s > 16) return invalid("slices must be in [1, 16], got %d", slices);
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    if (ldb < (n > 1 ? n : 1)) return invalid("ldb < max(1, n)");
    if (n > 0 && k > 0 && (!B || !aligned(B, 8))) return invalid("B is NULL or misaligned");
    gb_status st = check_workspace(s, m, n, k, workspace, workspace_bytes);
    if (st != GB_OK) return st;
    DeviceScope scope(q->dev->idx);
    const EmuLayout L = emu_layout(s, m, n, k);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e = launch_split_cols(launch_of(q), s, n, k, B, ldb, ws + L.b_digits, L.kp,
                                      reinterpret_cast<int32_t*>(ws + L.b_exp),
                                      reinterpret_cast<uint64_t*>(ws + L.b_part));
    return finish_call(q, e, "split of B");
}

gb_status gb_emulated_products(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                               double alpha, double beta, double* C, int64_t ldc,
                               void* workspace, size_t workspace_bytes) {
    if (!q) return invalid("q is NULL");
    const int s = resolve_slices(slices);
    if (s < 1 || s > 16) return invalid("slices must be in [1, 16], got %d", slices);
    if (m < 0 || n < 0 || k < 0) return invalid("m, n, k must be >= 0");
    if (ldc < (n > 1 ? n : 1)) return invalid("ldc < max(1, n)");
    if (m > 0 && n > 0 && (!C || !aligned(C, 8))) return invalid("C is NULL or misaligned");
    gb_status st = check_workspace(s, m, n, k, workspace, workspace_bytes);
    if (st != GB_OK) return st;
    DeviceScope scope(q->dev->idx);
    const EmuLayout L = emu_layout(s, m, n, k);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    cudaError_t e = launch_emu_products(launch_of(q), s, m, n, k, alpha, beta, C, ldc,
                                        ws + L.a_digits, ws + L.b_digits, L.kp,
                                        reinterpret_cast<int32_t*>(ws + L.a_exp),
                                        reinterpret_cast<int32_t*>(ws + L.b_exp));
    return finish_call(q, e, "emulated products");
}

gb_status gb_emulated_crt_step(gb_queue* q, int step, int moduli, int64_t m, int64_t n,
                               int64_t k, double alpha, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double beta, double* C,
                               int64_t ldc, void* workspace, size_t workspace_bytes) {
    if (!q) return invalid("q is NULL");
    if (step < 0 || step > 3) return invalid("step must be 0 - 3, got %d", step);
    if (m < 0 || n < 0 || k < 1) return invalid("m, n >= 0 and k >= 1 for the steps");
    const int N = resolve_crt_moduli(moduli);
    if (N < 1 || N > kCrtMaxModuli)
        return invalid("the number of moduli must be in [1, %d] (or 0), got %d", kCrtMaxModuli,
                       moduli);
    if (crt_scale_bits(N, k) < 1) {
        set_error("k = %lld is too long for %d moduli", (long long)k, N);
        return GB_ERR_UNSUPPORTED;
    }
    if (step == 0 && (!A || lda < k || !aligned(A, 8)))
        return invalid("A missing, misaligned or lda < k");
    if (step == 1 && (!B || ldb < (n > 1 ? n : 1) || !aligned(B, 8)))
        return invalid("B missing, misaligned or ldb < n");
    if (step == 3 && (!C || ldc < (n > 1 ? n : 1) || !aligned(C, 8)))
        return invalid("C missing, misaligned or ldc < n");
    const CrtLayout lay = crt_layout(N, m, n, k);
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < lay.total) {
        set_error("the residue steps need a 256-byte aligned workspace of %zu bytes", lay.total);
        return GB_ERR_WORKSPACE;
    }
    if (m == 0 || n == 0) return GB_OK;
    DeviceScope scope(q->dev->idx);
    if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    const Launch L = launch_of(q);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    int16_t* cres = reinterpret_cast<int16_t*>(ws + lay.c_res);
    cudaError_t e = cudaSuccess;
    switch (step) {
        case 0: e = crt_split_a(L, N, lay.b, m, k, A, lda, ws + lay.a_res, lay.kp, ea); break;
        case 1:
            e = crt_split_b(L, N, lay.b, n, k, B, ldb, ws + lay.b_res, lay.kp, fb,
                            reinterpret_cast<uint64_t*>(ws + lay.b_part));
            break;
        case 2: e = crt_residue_products(L, N, m, n, lay.kp, ws + lay.a_res, ws + lay.b_res, cres); break;
        default: e = crt_combine(L, N, lay.b, m, n, alpha, beta, C, ldc, cres, ea, fb); break;
    }
    return finish_call(q, e, "emulated (residues) step");
}

gb_status gb_dgemm(gb_queue* q, const gb_workdiv* wd, gb_kernel kernel, gb_precision prec,
                   int slices, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                   int64_t ldc, void* workspace, size_t workspace_bytes) {
    if (!q) return invalid("q is NULL");
    gb_status st = check_gemm_args(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    if (st != GB_OK) return st;
    if (prec != GB_PREC_NATIVE && prec != GB_PREC_EMULATED && prec != GB_PREC_EMULATED_BF16 &&
        prec != GB_PREC_EMULATED_CRT)
        return invalid("unknown precision %d", (int)prec);
    if (kernel < GB_KERNEL_AUTO || kernel > GB_KERNEL_DMMA) return invalid("unknown kernel %d", (int)kernel);
    int s = 0;
    if (prec == GB_PREC_EMULATED) {
        s = resolve_slices(slices);
        if (s < 1 || s > 16) return invalid("slices must be in [1, 16] (or 0), got %d", slices);
    } else if (prec == GB_PREC_EMULATED_BF16) {
        s = resolve_bf16_slices(slices);
        if (s < 1 || s > kBf16MaxSlices)
            return invalid("BF16-digit slices must be in [1, %d] (or 0), got %d", kBf16MaxSlices,
                           slices);
        if (k > kBf16MaxK) {
            set_error("the BF16-digit precision supports k <= %lld, got %lld",
                      (long long)kBf16MaxK, (long long)k);
            return GB_ERR_UNSUPPORTED;
        }
    } else if (prec == GB_PREC_EMULATED_CRT) {
        s = resolve_crt_moduli(slices);
        if (s < 1 || s > kCrtMaxModuli)
            return invalid("the number of moduli must be in [1, %d] (or 0), got %d", kCrtMaxModuli,
                           slices);
        if (crt_scale_bits(s, k) < 1) {
            set_error("k = %lld is too long for %d moduli (the exact product would not fit)",
                      (long long)k, s);
            return GB_ERR_UNSUPPORTED;
        }
    }
    if (prec != GB_PREC_NATIVE && wd) {
        set_error("the emulated precisions take no work division (pass NULL)");
        return GB_ERR_INVALID_WORKDIV;
    }
    Variant v{};
    gb_workdiv resolved;
    if (prec == GB_PREC_NATIVE) {
        if (wd) {
            const gb_kernel kk = kernel == GB_KERNEL_AUTO ? GB_KERNEL_DFMA : kernel;
            st = check_workdiv(wd, kk, m, n);
            if (st != GB_OK) return st;
            resolved = *wd;
            v = Variant{kk, wd->block_threads[0], wd->block_threads[1], wd->thread_elems[0],
                        wd->thread_elems[1]};
        } else {
            v = default_variant(kernel, m, n, k);
            fill_workdiv(&resolved, v, m, n);
            st = check_workdiv(&resolved, v.kernel, m, n);
            if (st != GB_OK) return st;
        }
    }
    if (m == 0 || n == 0) return GB_OK;
    DeviceScope scope(q->dev->idx);
    if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    const Launch L = launch_of(q);
    const Gemm g{m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
    if (alpha == 0.0 || k == 0) return finish_call(q, launch_scale(L, g), "C <- beta C");

    if (prec == GB_PREC_EMULATED) {
        st = check_workspace(s, m, n, k, workspace, workspace_bytes);
        if (st != GB_OK) return st;
        const EmuLayout lay = emu_layout(s, m, n, k);
        uint8_t* ws = static_cast<uint8_t*>(workspace);
        int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
        int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
        cudaError_t e = launch_split_rows(L, s, m, k, A, lda, ws + lay.a_digits, lay.kp, ea);
        if (e == cudaSuccess)
            e = launch_split_cols(L, s, n, k, B, ldb, ws + lay.b_digits, lay.kp, fb,
                                  reinterpret_cast<uint64_t*>(ws + lay.b_part));
        if (e == cudaSuccess)
            e = launch_emu_products(L, s, m, n, k, alpha, beta, C, ldc, ws + lay.a_digits,
                                    ws + lay.b_digits, lay.kp, ea, fb);
        return finish_call(q, e, "emulated dgemm");
    }
    if (prec == GB_PREC_EMULATED_BF16) {
        const EmuLayout lay = emu_layout_bf16(s, m, n, k);
        st = check_workspace_layout(lay, workspace, workspace_bytes);
        if (st != GB_OK) return st;
        uint8_t* ws = static_cast<uint8_t*>(workspace);
        int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
        int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
        cudaError_t e = launch_bf16_split_rows(L, s, m, k, A, lda, ws + lay.a_digits, lay.kp, ea);
        if (e == cudaSuccess)
            e = launch_bf16_split_cols(L, s, n, k, B, ldb, ws + lay.b_digits, lay.kp, fb,
                                       reinterpret_cast<uint64_t*>(ws + lay.b_part));
        if (e == cudaSuccess)
            e = launch_bf16_products(L, s, m, n, alpha, beta, C, ldc, ws + lay.a_digits,
                                     ws + lay.b_digits, lay.kp, ea, fb);
        return finish_call(q, e, "emulated (BF16 digits) dgemm");
    }
    if (prec == GB_PREC_EMULATED_CRT) {
        const CrtLayout lay = crt_layout(s, m, n, k);
        if (!workspace) {
            set_error("the emulated path needs a workspace of %zu bytes", lay.total);
            return GB_ERR_WORKSPACE;
        }
        if (!aligned(workspace, 256)) {
            set_error("workspace must be 256-byte aligned");
            return GB_ERR_WORKSPACE;
        }
        if (workspace_bytes < lay.total) {
            set_error("workspace of %zu bytes < required %zu", workspace_bytes, lay.total);
            return GB_ERR_WORKSPACE;
        }
        const cudaError_t e = launch_crt_gemm(L, g, static_cast<uint8_t*>(workspace), lay);
        return finish_call(q, e, "emulated (residues) dgemm");
    }

    cudaError_t e = cudaSuccess;
    switch (v.kernel) {
        case GB_KERNEL_NAIVE: e = launch_naive(L, g, (int)v.bt0, (int)v.bt1); break;
        case GB_KERNEL_TILED: e = launch_tiled(L, g, (int)v.bt0); break;
        case GB_KERNEL_DFMA: e = launch_dfma(L, g, (int)v.te0); break;
        case GB_KERNEL_DMMA:
        default: e = launch_dmma(L, g, (int)v.bt0, (int)v.bt1, (int)v.te0, (int)v.te1); break;
    }
    return finish_call(q, e, "native dgemm");
}

}  // extern "C"
