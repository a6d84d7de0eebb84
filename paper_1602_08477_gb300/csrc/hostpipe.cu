// FP64 GEMM on operands in host memory, with the transfers overlapped.
//
// The paper's memory model (Section 3.4.4) keeps host and device buffers apart and
// moves data only by explicit copies enqueued on a queue; a caller whose A, B and
// C live in host memory would copy A and B in, run the GEMM and copy C out, one
// after the other.  This entry point enqueues the same copies itself and overlaps
// them with the computation, on the queue's stream plus two streams of its own
// (one per copy direction), ordered by events:
//
//   h2d stream : B, then A and (beta != 0) C in bands of rows
//   queue      : split of B once B has arrived; per band: split of the band's rows
//                of A, the band's slice products into its rows of C
//   d2h stream : each band's rows of C as soon as its products are done
//
// so the copies of A after the first band and of C before the last band run
// under the tensor-core products.  The native precision copies everything first
// and C last (its FP64 compute outweighs the transfers by two orders of
// magnitude).  The device side is a caller workspace: the emulated workspace
// followed by dense device copies of A, B and C.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "gb_gemm.h"
#include "handles.h"
#include "internal.h"

namespace gb {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct HostLayout {
    size_t emu = 0;  // emulated workspace bytes (0 for native)
    size_t a = 0, b = 0, c = 0, total = 0;
};

HostLayout host_layout(gb_precision prec, int s, int64_t m, int64_t n, int64_t k) {
    HostLayout h;
    size_t off = 0;
    if (prec == GB_PREC_EMULATED) off = up256(emu_layout(s, m, n, k).total);
    h.emu = off;
    h.a = off;
    off = up256(off + 8 * (size_t)m * (size_t)k);
    h.b = off;
    off = up256(off + 8 * (size_t)k * (size_t)n);
    h.c = off;
    off = up256(off + 8 * (size_t)m * (size_t)n);
    h.total = off;
    return h;
}

// Row bands of the emulated pipeline: whole 128-row tiles, at most kMaxBands
// bands, none smaller than kMinBandRows (each band is one launch of the split and
// of the products kernel, whose last wave is partly idle).
constexpr int kMaxBands = 4;
constexpr int64_t kMinBandRows = 1024;

int band_count(int64_t m) {
    int64_t nb = m / kMinBandRows;
    if (nb < 1) nb = 1;
    if (nb > kMaxBands) nb = kMaxBands;
    return (int)nb;
}

// Rows [r0, r1) of band i of nb over m rows (band edges on 128-row tiles).
void band_rows(int64_t m, int nb, int i, int64_t* r0, int64_t* r1) {
    const int64_t tiles = (m + kEmuBM - 1) / kEmuBM;
    const int64_t t0 = tiles * i / nb, t1 = tiles * (i + 1) / nb;
    *r0 = t0 * kEmuBM;
    *r1 = t1 * kEmuBM < m ? t1 * kEmuBM : m;
}

cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch,
                      int64_t cols, int64_t rows, cudaMemcpyKind kind, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, 8 * (size_t)cols, (size_t)rows, kind, s);
}

// The queue's copy streams and events, created on first use.
cudaError_t ensure_aux(gb_queue* q) {
    if (q->aux_h2d) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&q->aux_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->aux_d2h, cudaStreamNonBlocking);
    for (int i = 0; i < kAuxEvents && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&q->aux_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) release_aux(q);
    return e;
}

}  // namespace

void release_aux(gb_queue* q) {
    for (int i = 0; i < kAuxEvents; ++i) {
        if (q->aux_ev[i]) cudaEventDestroy(q->aux_ev[i]);
        q->aux_ev[i] = nullptr;
    }
    if (q->aux_h2d) cudaStreamDestroy(q->aux_h2d);
    if (q->aux_d2h) cudaStreamDestroy(q->aux_d2h);
    q->aux_h2d = q->aux_d2h = nullptr;
}

}  // namespace gb

using namespace gb;

extern "C" {

gb_status gb_dgemm_host_workspace_size(gb_precision prec, int slices, int64_t m, int64_t n,
                                       int64_t k, size_t* out) {
    if (!out) {
        set_error("out is NULL");
        return GB_ERR_INVALID_ARG;
    }
    if (m < 0 || n < 0 || k < 0) {
        set_error("m, n, k must be >= 0");
        return GB_ERR_INVALID_ARG;
    }
    if (prec != GB_PREC_NATIVE && prec != GB_PREC_EMULATED) {
        set_error("unknown precision %d", (int)prec);
        return GB_ERR_INVALID_ARG;
    }
    const int s = slices == 0 ? 11 : slices;
    if (prec == GB_PREC_EMULATED && (s < 1 || s > 16)) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    *out = host_layout(prec, s, m, n, k).total;
    return GB_OK;
}

gb_status gb_dgemm_host(gb_queue* q, gb_precision prec, int slices, int64_t m, int64_t n,
                        int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double beta, double* C, int64_t ldc, void* workspace,
                        size_t workspace_bytes) {
    if (!q) {
        set_error("q is NULL");
        return GB_ERR_INVALID_ARG;
    }
    const int v = validate_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    if (v != GB_OK) return (gb_status)v;
    if (prec != GB_PREC_NATIVE && prec != GB_PREC_EMULATED) {
        set_error("unknown precision %d", (int)prec);
        return GB_ERR_INVALID_ARG;
    }
    const int s = slices == 0 ? 11 : slices;
    if (prec == GB_PREC_EMULATED && (s < 1 || s > 16)) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    if (m == 0 || n == 0) return GB_OK;
    const HostLayout h = host_layout(prec, s, m, n, k);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
        workspace_bytes < h.total) {
        set_error("gb_dgemm_host needs a 256-byte aligned device workspace of %zu bytes "
                  "(got %zu)", h.total, workspace ? workspace_bytes : (size_t)0);
        return GB_ERR_WORKSPACE;
    }
    DeviceScope scope(q->dev->idx);
    if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    cudaError_t e = ensure_aux(q);
    if (e != cudaSuccess) return cuda_fail(e, "creating the copy streams");

    uint8_t* ws = static_cast<uint8_t*>(workspace);
    double* dA = reinterpret_cast<double*>(ws + h.a);
    double* dB = reinterpret_cast<double*>(ws + h.b);
    double* dC = reinterpret_cast<double*>(ws + h.c);
    const bool reads_ab = alpha != 0.0 && k > 0;
    const bool reads_c = beta != 0.0;
    const int64_t kk = k > 0 ? k : 1;  // device leading dimensions (dense rows)
    cudaStream_t qs = q->stream, hs = q->aux_h2d, ds = q->aux_d2h;
    cudaEvent_t* ev = q->aux_ev;  // [0] start, [1] B in, [2 + 2i] band i in, [3 + 2i] band i done
    const Launch L{qs, q->status, q->dev->sm_count};

    // the copies must not overtake work already on the queue that uses the workspace
    e = cudaEventRecord(ev[0], qs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, ev[0], 0);

    if (prec == GB_PREC_NATIVE || !reads_ab) {
        // copy in, compute with gb_dgemm on the queue (non-blocking view), copy out
        if (e == cudaSuccess && reads_ab)
            e = copy_rows(dA, 8 * (size_t)kk, A, 8 * (size_t)lda, k, m, cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess && reads_ab)
            e = copy_rows(dB, 8 * (size_t)n, B, 8 * (size_t)ldb, n, k, cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess && reads_c)
            e = copy_rows(dC, 8 * (size_t)n, C, 8 * (size_t)ldc, n, m, cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], hs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[1], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host-buffer dgemm: copies in");
        gb_queue view = *q;
        view.blocking = 0;
        gb_status st = gb_dgemm(&view, nullptr, GB_KERNEL_AUTO, prec, s, m, n, k, alpha, dA, kk, dB,
                                n, beta, dC, n, ws, h.emu);
        if (st != GB_OK) return st;
        e = cudaEventRecord(ev[3], qs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, ev[3], 0);
        if (e == cudaSuccess)
            e = copy_rows(C, 8 * (size_t)ldc, dC, 8 * (size_t)n, n, m, cudaMemcpyDeviceToHost, ds);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], ds);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[2], 0);
        return finish_call(q, e, "host-buffer dgemm: copy out");
    }

    const EmuLayout lay = emu_layout(s, m, n, k);
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    const int nb = band_count(m);
    // h2d: B first (every band's products need all of B), then the bands of A (and C)
    if (e == cudaSuccess)
        e = copy_rows(dB, 8 * (size_t)n, B, 8 * (size_t)ldb, n, k, cudaMemcpyHostToDevice, hs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], hs);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        int64_t r0, r1;
        band_rows(m, nb, i, &r0, &r1);
        e = copy_rows(dA + r0 * kk, 8 * (size_t)kk, A + r0 * lda, 8 * (size_t)lda, k, r1 - r0,
                      cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess && reads_c)
            e = copy_rows(dC + r0 * n, 8 * (size_t)n, C + r0 * ldc, 8 * (size_t)ldc, n, r1 - r0,
                          cudaMemcpyHostToDevice, hs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 + 2 * i], hs);
    }
    // queue: split of B, then per band the split of its rows of A and its products
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[1], 0);
    if (e == cudaSuccess)
        e = launch_split_cols(L, s, n, k, dB, n, ws + lay.b_digits, lay.kp, fb);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        int64_t r0, r1;
        band_rows(m, nb, i, &r0, &r1);
        // a band starts on a 128-row tile: its digit tiles start r0 * kp * s bytes in
        const size_t doff = (size_t)r0 * (size_t)lay.kp * (size_t)s;
        e = cudaStreamWaitEvent(qs, ev[2 + 2 * i], 0);
        if (e == cudaSuccess)
            e = launch_split_rows(L, s, r1 - r0, k, dA + r0 * kk, kk, ws + lay.a_digits + doff,
                                  lay.kp, ea + r0);
        if (e == cudaSuccess)
            e = launch_emu_products(L, s, r1 - r0, n, k, alpha, beta, dC + r0 * n, n,
                                    ws + lay.a_digits + doff, ws + lay.b_digits, lay.kp, ea + r0,
                                    fb);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 + 2 * i], qs);
        // d2h: this band's rows of C while the next bands compute
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, ev[3 + 2 * i], 0);
        if (e == cudaSuccess)
            e = copy_rows(C + r0 * ldc, 8 * (size_t)ldc, dC + r0 * n, 8 * (size_t)n, n, r1 - r0,
                          cudaMemcpyDeviceToHost, ds);
    }
    // the queue completes when C is back in host memory
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], ds);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[0], 0);
    return finish_call(q, e, "host-buffer emulated dgemm");
}

}  // extern "C"
