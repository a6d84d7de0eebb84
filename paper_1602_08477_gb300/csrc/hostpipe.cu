// FP64 GEMM on operands in host memory, with the transfers overlapped.
//
// The paper's memory model (Section 3.4.4) keeps host and device buffers apart and
// moves data only by explicit copies enqueued on a queue; a caller whose A, B and
// C live in host memory would copy A and B in, run the GEMM and copy C out, one
// after the other.  This entry point enqueues the same copies itself and overlaps
// them with the computation, on the queue's stream plus two streams of its own
// (one per copy direction), ordered by events:
//
//   h2d stream : B in one or two blocks of columns and A (and, beta != 0, C) in
//                bands of rows, in the order the launches below need them
//   queue      : per row band: split of its rows of A, then its slice products
//                into its rows of C; the first band in two column blocks, each
//                block of B split just before its first use
//   d2h stream : each block of C as soon as its products are done
//
// so the first products start once part of B and the first band of A have
// arrived, and the other copies run under the tensor-core products.  Band and
// block sizes are chosen so that each products launch fills whole waves of the
// SMs where possible.  The native
// precision copies everything first and C last (its FP64 compute outweighs the
// transfers by two orders of magnitude).  The device side is a caller workspace: the emulated workspace
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

// Row bands of the emulated pipeline, on whole 128-row tiles: at most kMaxBands,
// each with at least kMinWaves waves of output tiles over the SMs (every band is
// one products launch, whose last wave is partly idle).
constexpr int kMaxBands = 4;
constexpr int kMinWaves = 8;
static_assert(1 + 2 + kMaxBands + (kMaxBands + 1) <= kAuxEvents, "events of the pipeline");

int band_count(int64_t tile_rows, int64_t tile_cols, int sms) {
    int64_t nb = tile_rows * tile_cols / ((int64_t)kMinWaves * sms);
    if (nb > tile_rows) nb = tile_rows;
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

// Idle tile slots of a launch of `tiles` tiles in its last wave over `sms` SMs.
int64_t tail_slots(int64_t tiles, int sms) { return (tiles + sms - 1) / sms * sms - tiles; }

// The first row band (R tile rows) runs as two launches, over tile columns [0, c)
// and [c, T), so its products start once the first c tile columns of B have
// arrived.  c lies in [0.4 T, 0.5 T] (the second part of B must arrive while the
// first block computes) and leaves the fewest idle slots in the two last waves
// (n = 8192, s = 10: c = 76 of 171, 8 and 10 full waves).  0: no split.
int64_t first_band_split(int nb, int64_t R, int64_t T, int sms) {
    if (nb < 2 || T < 16) return 0;
    int64_t best = 0, best_idle = 0;
    for (int64_t c = (4 * T + 9) / 10; c <= T / 2; ++c) {
        const int64_t idle = tail_slots(R * c, sms) + tail_slots(R * (T - c), sms);
        if (best == 0 || idle < best_idle) {
            best = c;
            best_idle = idle;
        }
    }
    return best;
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
    const int bn = lay.bn;
    const int64_t tile_rows = (m + kEmuBM - 1) / kEmuBM, tile_cols = (n + bn - 1) / bn;
    const int nb = band_count(tile_rows, tile_cols, q->dev->sm_count);
    int64_t fr0, fr1;
    band_rows(m, nb, 0, &fr0, &fr1);
    const int64_t csplit_tiles =
        first_band_split(nb, (fr1 - fr0 + kEmuBM - 1) / kEmuBM, tile_cols, q->dev->sm_count);
    // column blocks of B: [0, csplit) and [csplit, n), or one block
    const int64_t csplit = csplit_tiles > 0 ? csplit_tiles * bn : n;
    const int ncb = csplit < n ? 2 : 1;
    const int64_t cb0[2] = {0, csplit}, cb1[2] = {csplit, n};
    // events: [1, 3) column blocks of B in, [3, 3 + nb) row bands of A (and C) in,
    // [3 + nb, ...) one per products launch
    cudaEvent_t* ev_b = ev + 1;
    cudaEvent_t* ev_a = ev + 3;
    cudaEvent_t* ev_p = ev + 3 + nb;
    auto copy_b = [&](int j) {
        cudaError_t r = copy_rows(dB + cb0[j], 8 * (size_t)n, B + cb0[j], 8 * (size_t)ldb,
                                  cb1[j] - cb0[j], k, cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_b[j], hs) : r;
    };
    auto copy_a = [&](int i) {
        int64_t r0, r1;
        band_rows(m, nb, i, &r0, &r1);
        cudaError_t r = copy_rows(dA + r0 * kk, 8 * (size_t)kk, A + r0 * lda, 8 * (size_t)lda, k,
                                  r1 - r0, cudaMemcpyHostToDevice, hs);
        if (r == cudaSuccess && reads_c)
            r = copy_rows(dC + r0 * n, 8 * (size_t)n, C + r0 * ldc, 8 * (size_t)ldc, n, r1 - r0,
                          cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_a[i], hs) : r;
    };
    // h2d in the order the launches need it: B's first column block, A's first row
    // band, the rest of B, A's other row bands (each with C's rows)
    if (e == cudaSuccess) e = copy_b(0);
    if (e == cudaSuccess) e = copy_a(0);
    if (ncb == 2 && e == cudaSuccess) e = copy_b(1);
    for (int i = 1; i < nb && e == cudaSuccess; ++i) e = copy_a(i);
    // queue: per row band the split of its rows of A, then its products (the first
    // band in two column blocks, each block of B split just before its first use);
    // d2h: each block of C as soon as it is computed.  Band edges sit on tile
    // edges (128 rows, bn columns), so a band's digit tiles start r0 * kp * s
    // (c0 * kp * s) bytes into the planes.
    int launch = 0;
    auto products = [&](int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
        const size_t aoff = (size_t)r0 * (size_t)lay.kp * (size_t)s;
        const size_t boff = (size_t)c0 * (size_t)lay.kp * (size_t)s;
        cudaError_t r = launch_emu_products(L, s, r1 - r0, c1 - c0, k, alpha, beta,
                                            dC + r0 * n + c0, n, ws + lay.a_digits + aoff,
                                            ws + lay.b_digits + boff, lay.kp, ea + r0, fb + c0);
        cudaEvent_t done = ev_p[launch++];
        if (r == cudaSuccess) r = cudaEventRecord(done, qs);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(ds, done, 0);
        if (r == cudaSuccess)
            r = copy_rows(C + r0 * ldc + c0, 8 * (size_t)ldc, dC + r0 * n + c0, 8 * (size_t)n,
                          c1 - c0, r1 - r0, cudaMemcpyDeviceToHost, ds);
        return r;
    };
    auto split_b = [&](int j) {
        const size_t boff = (size_t)cb0[j] * (size_t)lay.kp * (size_t)s;
        cudaError_t r = cudaStreamWaitEvent(qs, ev_b[j], 0);
        if (r == cudaSuccess)
            r = launch_split_cols(L, s, cb1[j] - cb0[j], k, dB + cb0[j], n,
                                  ws + lay.b_digits + boff, lay.kp, fb + cb0[j]);
        return r;
    };
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        int64_t r0, r1;
        band_rows(m, nb, i, &r0, &r1);
        const size_t aoff = (size_t)r0 * (size_t)lay.kp * (size_t)s;
        e = cudaStreamWaitEvent(qs, ev_a[i], 0);
        if (e == cudaSuccess)
            e = launch_split_rows(L, s, r1 - r0, k, dA + r0 * kk, kk, ws + lay.a_digits + aoff,
                                  lay.kp, ea + r0);
        if (i == 0) {
            for (int j = 0; j < ncb && e == cudaSuccess; ++j) {
                e = split_b(j);
                if (e == cudaSuccess) e = products(r0, r1, cb0[j], cb1[j]);
            }
        } else if (e == cudaSuccess) {
            e = products(r0, r1, 0, n);
        }
    }
    // the queue completes when C is back in host memory
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], ds);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[0], 0);
    return finish_call(q, e, "host-buffer emulated dgemm");
}

}  // extern "C"
