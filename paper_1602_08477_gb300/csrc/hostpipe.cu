// FP64 GEMM on operands in host memory, with the transfers overlapped.
//
// The paper's memory model (Section 3.4.4) keeps host and device buffers apart and
// moves data only by explicit copies enqueued on a queue; a caller whose A, B and
// C live in host memory would copy A and B in, run the GEMM and copy C out, one
// after the other.  This entry point enqueues the same copies itself and overlaps
// them with the computation, on the queue's stream plus two streams of its own
// (one per copy direction), ordered by events:
//
//   h2d stream : B in column blocks and A (and, beta != 0, C) in bands of rows,
//                in the order the launches below need them
//   queue      : per row band: split of its rows of A, then its slice products
//                into its rows of C; the first band one launch per column block
//                of B, each block split just before its first use; the last band
//                in two launches
//   d2h stream : each block of C as soon as its products are done
//
// (the residue precision follows the same plan with its own steps and pieces,
// crt_host_pipeline), so the first products start once a small first block of B
// and the first band of A have arrived, the blocks of B grow as fast as the link keeps ahead of the
// products, the other copies run under the tensor-core products, and only a small
// last block of C is copied back after the last launch.  Launch sizes are chosen
// so that each fills whole waves of the SMs where possible.  The native
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
    if (prec == GB_PREC_EMULATED_CRT) off = up256(crt_layout(s, m, n, k).total);
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
// one products launch or a few, the last wave of each partly idle).
constexpr int kMaxBands = 4;
constexpr int kMinWaves = 8;
constexpr int kMaxBBlocks = 6;                       // column blocks of B (first band)
constexpr int kMaxPieces = kMaxBBlocks + kMaxBands;  // products launches
static_assert(1 + kMaxBBlocks + kMaxBands + kMaxPieces <= kAuxEvents, "events of the pipeline");

// Planning estimates (they order the copies and size the launches; the result does
// not depend on them): FP8 tensor-core flop of the slice products per SM and
// second, and bytes per second of the host link in either direction.
constexpr double kPlanSmFlops = 25e12;
constexpr double kPlanLinkBytes = 180e9;

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
int64_t waves(int64_t tiles, int sms) { return (tiles + sms - 1) / sms; }
int64_t gcd64(int64_t a, int64_t b) { return b ? gcd64(b, a % b) : a; }

// The launches of one host-buffer GEMM, in enqueue order.  Band 0 runs one launch
// per column block of B (B arrives block by block, the first small); bands
// 1 .. nb-2 one launch each; the last band two when that hides the copy-back of
// its first part under the second.
struct Piece {
    int64_t r0, r1, c0, c1;  // rows of A / C, columns of B / C
    int band, bblock;        // row band; column block of B (band 0), else -1
};
struct HostSchedule {
    int nb = 1;     // row bands of A (and C)
    int nbb = 1;    // column blocks of B, = launches of band 0
    int64_t bcut[kMaxBBlocks + 1] = {};  // column edges of the blocks of B
    int np = 0;
    Piece piece[kMaxPieces] = {};
};

// Column blocks of B for band 0 (R tile rows, T tile columns; cut[] in tile
// columns).  Blocks are whole waves of band 0 where the wave quantum allows: the
// first is one quantum (so the products start after a small part of B), each next
// the largest number of quanta whose copy ends before the previous block's
// products do (t_col per tile column of B, t_tile per tile and SM, t_head for the
// copies that precede the first launch), the last takes the remaining columns.
// Without a usable quantum: two blocks, [0, c) and [c, T), c in [0.4 T, 0.5 T]
// leaving the fewest idle slots.
int b_blocks(int nb, int64_t R, int64_t T, int sms, double t_tile, double t_col,
             double t_head, int64_t* cut) {
    cut[0] = 0;
    if (nb < 2 || T < 16) {
        cut[1] = T;
        return 1;
    }
    const int64_t q = sms / gcd64(R, (int64_t)sms);  // tile columns per whole wave count
    if (3 * q > T) {
        int64_t best = 0, best_idle = 0;
        for (int64_t c = (4 * T + 9) / 10; c <= T / 2; ++c) {
            const int64_t idle = tail_slots(R * c, sms) + tail_slots(R * (T - c), sms);
            if (best == 0 || idle < best_idle) {
                best = c;
                best_idle = idle;
            }
        }
        cut[1] = best;
        cut[2] = T;
        return 2;
    }
    int n = 0;
    int64_t c = q, used = q;
    double link = t_head + (double)c * t_col;  // B's block 0 and A's band 0 are in
    double gpu = link;                          // the first launch starts
    cut[++n] = used;
    while (used < T && n < kMaxBBlocks - 1) {
        const double gpu_end = gpu + (double)waves(R * c, sms) * t_tile;
        const int64_t cmax = (int64_t)((gpu_end - link) / t_col);
        c = cmax / q * q;
        if (c < q) c = q;
        if (T - used - c < q) c = T - used;  // no room for a further whole block
        link += (double)c * t_col;
        gpu = gpu_end > link ? gpu_end : link;
        used += c;
        cut[++n] = used;
    }
    if (used < T) cut[++n] = T;
    return n;
}

// First tile column of the last band's second launch (R tile rows): the split
// whose first part's copy back runs under the second part's products and saves
// the most time after the last launch, net of the waves the second launch adds;
// T (one launch) when no split saves time.
int64_t last_band_split(int64_t R, int64_t rows, int64_t T, int bn, int sms, double t_tile) {
    if (T < 16) return T;
    int64_t best = T;
    double best_gain = 0.0;
    for (int64_t c = T - 1; 2 * c >= T; --c) {
        const double back = 8.0 * (double)rows * (double)(c * bn) / kPlanLinkBytes;
        if (back > (double)waves(R * (T - c), sms) * t_tile) continue;
        const int64_t extra = waves(R * c, sms) + waves(R * (T - c), sms) - waves(R * T, sms);
        const double gain = back - (double)extra * t_tile;
        if (gain > best_gain) {
            best = c;
            best_gain = gain;
        }
    }
    return best;
}

HostSchedule host_schedule(int s, int64_t m, int64_t n, int64_t k, bool reads_c, int sms) {
    HostSchedule h;
    const EmuLayout lay = emu_layout(s, m, n, k);
    const int bn = lay.bn;
    const int64_t tile_rows = (m + kEmuBM - 1) / kEmuBM, tile_cols = (n + bn - 1) / bn;
    h.nb = band_count(tile_rows, tile_cols, sms);
    const double t_tile =
        (double)s * (s + 1) * kEmuBM * bn * (double)lay.kp / kPlanSmFlops;  // s(s+1)/2 pairs
    const double t_col = 8.0 * (double)k * bn / kPlanLinkBytes;
    int64_t r0, r1;
    band_rows(m, h.nb, 0, &r0, &r1);
    const double t_head = 8.0 * (double)(r1 - r0) * (double)(k + (reads_c ? n : 0)) / kPlanLinkBytes;
    int64_t cut[kMaxBBlocks + 1];
    h.nbb = b_blocks(h.nb, (r1 - r0 + kEmuBM - 1) / kEmuBM, tile_cols, sms, t_tile, t_col,
                     t_head, cut);
    for (int j = 0; j <= h.nbb; ++j) h.bcut[j] = cut[j] * bn < n ? cut[j] * bn : n;
    for (int j = 0; j < h.nbb; ++j) h.piece[h.np++] = Piece{r0, r1, h.bcut[j], h.bcut[j + 1], 0, j};
    for (int i = 1; i < h.nb; ++i) {
        band_rows(m, h.nb, i, &r0, &r1);
        const int64_t c = i + 1 == h.nb
                              ? last_band_split((r1 - r0 + kEmuBM - 1) / kEmuBM, r1 - r0,
                                                tile_cols, bn, sms, t_tile) * bn
                              : n;
        if (c < n) {
            h.piece[h.np++] = Piece{r0, r1, 0, c, i, -1};
            h.piece[h.np++] = Piece{r0, r1, c, n, i, -1};
        } else {
            h.piece[h.np++] = Piece{r0, r1, 0, n, i, -1};
        }
    }
    return h;
}

cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch,
                      int64_t cols, int64_t rows, cudaMemcpyKind kind, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, 8 * (size_t)cols, (size_t)rows, kind, s);
}

// Residue precision: the launches of one host-buffer GEMM.  A in nb equal row
// bands of whole 128-row tiles (at most kMaxBands, each with at least two waves
// of (modulus, tile) products).  The first band runs one launch per column block
// of B, kCrtBBlocks equal blocks of whole 256-column tiles: narrower blocks would
// start the products sooner, but a column block is a strided copy whose rows are
// the block's width, and the host link moves rows narrower than 16 KiB far below
// its rate (measured pinned -> device: 75 GB/s at 2 KiB, 109 at 8 KiB, 188 at
// 16 KiB, 210 at 32 KiB).  The last band runs two launches when that shortens the
// time after its products: the first part's copy back then runs under the second
// part's products (planning estimates below; the result does not depend on them).
constexpr int kCrtBBlocks = 4;
constexpr double kPlanItemFlopsPerSm = 10.5e12;  // BF16 residue products, per SM and second
constexpr double kPlanLinkBack = 190e9;         // device -> host bytes per second

HostSchedule crt_host_schedule(int N, int64_t m, int64_t n, int64_t kp, int sms) {
    HostSchedule h;
    const int64_t tiles_m = (m + kCrtTileRows - 1) / kCrtTileRows;
    const int64_t tiles_n = (n + kCrtTileCols - 1) / kCrtTileCols;
    int64_t nb = (int64_t)N * tiles_m * tiles_n / (2 * (int64_t)sms);
    if (nb > kMaxBands) nb = kMaxBands;
    if (nb > tiles_m) nb = tiles_m;
    if (nb < 1) nb = 1;
    h.nb = (int)nb;
    auto band = [&](int64_t i, int64_t* r0, int64_t* r1) {
        *r0 = tiles_m * i / nb * kCrtTileRows;
        const int64_t e = tiles_m * (i + 1) / nb * kCrtTileRows;
        *r1 = e < m ? e : m;
    };
    // column blocks of B for the first band, in tile columns
    int64_t cut[kMaxBBlocks + 1];
    int nbb = 0;
    cut[0] = 0;
    {
        const int64_t q = tiles_n < kCrtBBlocks ? tiles_n : kCrtBBlocks;
        for (int64_t j = 1; j < q; ++j) cut[++nbb] = tiles_n * j / q;
    }
    cut[++nbb] = tiles_n;
    h.nbb = nbb;
    for (int j = 0; j <= nbb; ++j) h.bcut[j] = cut[j] * kCrtTileCols < n ? cut[j] * kCrtTileCols : n;
    int64_t r0, r1;
    band(0, &r0, &r1);
    for (int j = 0; j < nbb; ++j) h.piece[h.np++] = Piece{r0, r1, h.bcut[j], h.bcut[j + 1], 0, j};
    const double t_item = 2.0 * kCrtTileRows * kCrtTileCols * (double)kp / kPlanItemFlopsPerSm;
    for (int64_t i = 1; i < nb; ++i) {
        band(i, &r0, &r1);
        int64_t split = tiles_n;
        if (i + 1 == nb && tiles_n >= 4) {
            // time from the band's start to the end of its copy back, one launch or two
            const int64_t R = (r1 - r0 + kCrtTileRows - 1) / kCrtTileRows;
            const double row_back = 8.0 * (double)(r1 - r0) / kPlanLinkBack;  // per column of C
            const double whole = (double)waves(N * R * tiles_n, sms) * t_item +
                                 row_back * (double)n;
            double best = whole;
            for (int64_t c = tiles_n - 1; 2 * c >= tiles_n; --c) {
                const int64_t c_cols = c * kCrtTileCols < n ? c * kCrtTileCols : n;
                const double t1 = (double)waves(N * R * c, sms) * t_item;
                const double t2 = t1 + (double)waves(N * R * (tiles_n - c), sms) * t_item;
                const double back1 = t1 + row_back * (double)c_cols;
                const double end = (t2 > back1 ? t2 : back1) + row_back * (double)(n - c_cols);
                if (end < best) {
                    best = end;
                    split = c;
                }
            }
        }
        if (split < tiles_n) {
            h.piece[h.np++] = Piece{r0, r1, 0, split * kCrtTileCols, (int)i, -1};
            h.piece[h.np++] = Piece{r0, r1, split * kCrtTileCols, n, (int)i, -1};
        } else {
            h.piece[h.np++] = Piece{r0, r1, 0, n, (int)i, -1};
        }
    }
    return h;
}

// Residue precision on host buffers, on the schedule above.  h2d: A's first band,
// B's blocks, A's other bands (each with C's rows when beta != 0); queue: the
// first band's residues, then per block of B its residues, the products of the
// first band with it and their reconstruction into C, then per further band its
// residues and its launches with all of B; d2h: each piece of C as soon as it is
// reconstructed.
cudaError_t crt_host_pipeline(const Launch& L, cudaStream_t hs, cudaStream_t ds, cudaEvent_t* ev,
                              int N, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb,
                              double beta, double* C, int64_t ldc, uint8_t* ws,
                              const CrtLayout& lay, double* dA, double* dB, double* dC) {
    const HostSchedule sch = crt_host_schedule(N, m, n, lay.kp, L.sm_count);
    const int64_t tiles_m = (m + kCrtTileRows - 1) / kCrtTileRows;
    const int64_t nb = sch.nb, nbb = sch.nbb;
    auto band = [&](int64_t i, int64_t* r0, int64_t* r1) {
        *r0 = tiles_m * i / nb * kCrtTileRows;
        const int64_t e = tiles_m * (i + 1) / nb * kCrtTileRows;
        *r1 = e < m ? e : m;
    };
    auto block = [&](int64_t j, int64_t* c0, int64_t* c1) {
        *c0 = sch.bcut[j];
        *c1 = sch.bcut[j + 1];
    };
    const bool reads_c = beta != 0.0;
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    uint8_t* ares = ws + lay.a_res;
    uint8_t* bres = ws + lay.b_res;
    int16_t* cres = reinterpret_cast<int16_t*>(ws + lay.c_res);
    uint64_t* part = reinterpret_cast<uint64_t*>(ws + lay.b_part);
    const size_t row_bytes = 2 * (size_t)N * (size_t)lay.kp;  // residues of one row or column
    cudaEvent_t* ev_b = ev + 1;                // column blocks of B in
    cudaEvent_t* ev_a = ev + 1 + kMaxBBlocks;  // row bands of A (and C) in
    cudaEvent_t* ev_p = ev_a + kMaxBands;      // pieces reconstructed
    auto copy_b = [&](int64_t j) {
        int64_t c0, c1;
        block(j, &c0, &c1);
        cudaError_t r = copy_rows(dB + c0, 8 * (size_t)n, B + c0, 8 * (size_t)ldb, c1 - c0, k,
                                  cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_b[j], hs) : r;
    };
    auto copy_a = [&](int64_t i) {
        int64_t r0, r1;
        band(i, &r0, &r1);
        cudaError_t r = copy_rows(dA + r0 * k, 8 * (size_t)k, A + r0 * lda, 8 * (size_t)lda, k,
                                  r1 - r0, cudaMemcpyHostToDevice, hs);
        if (r == cudaSuccess && reads_c)
            r = copy_rows(dC + r0 * n, 8 * (size_t)n, C + r0 * ldc, 8 * (size_t)ldc, n, r1 - r0,
                          cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_a[i], hs) : r;
    };
    auto split_a = [&](int64_t i) {
        int64_t r0, r1;
        band(i, &r0, &r1);
        cudaError_t r = cudaStreamWaitEvent(L.stream, ev_a[i], 0);
        if (r == cudaSuccess)
            r = crt_split_a(L, N, lay.b, r1 - r0, k, dA + r0 * k, k, ares + (size_t)r0 * row_bytes,
                            lay.kp, ea + r0);
        return r;
    };
    auto split_b = [&](int64_t j) {
        int64_t c0, c1;
        block(j, &c0, &c1);
        cudaError_t r = cudaStreamWaitEvent(L.stream, ev_b[j], 0);
        if (r == cudaSuccess)
            r = crt_split_b(L, N, lay.b, c1 - c0, k, dB + c0, n, bres + (size_t)c0 * row_bytes,
                            lay.kp, fb + c0, part);
        return r;
    };
    int np = 0;
    auto piece = [&](int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
        cudaError_t r = crt_products(L, N, lay.b, r1 - r0, c1 - c0, lay.kp, alpha, beta,
                                     dC + r0 * n + c0, n, ares + (size_t)r0 * row_bytes,
                                     bres + (size_t)c0 * row_bytes, cres, ea + r0, fb + c0);
        if (r == cudaSuccess) r = cudaEventRecord(ev_p[np], L.stream);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(ds, ev_p[np], 0);
        if (r == cudaSuccess)
            r = copy_rows(C + r0 * ldc + c0, 8 * (size_t)ldc, dC + r0 * n + c0, 8 * (size_t)n,
                          c1 - c0, r1 - r0, cudaMemcpyDeviceToHost, ds);
        ++np;
        return r;
    };
    cudaError_t e = copy_a(0);
    for (int64_t j = 0; j < nbb && e == cudaSuccess; ++j) e = copy_b(j);
    for (int64_t i = 1; i < nb && e == cudaSuccess; ++i) e = copy_a(i);
    int split_band = -1;
    for (int p = 0; p < sch.np && e == cudaSuccess; ++p) {
        const Piece& pc = sch.piece[p];
        if (pc.band != split_band) {
            e = split_a(pc.band);
            split_band = pc.band;
        }
        if (e == cudaSuccess && pc.bblock >= 0) e = split_b(pc.bblock);
        if (e == cudaSuccess) e = piece(pc.r0, pc.r1, pc.c0, pc.c1);
    }
    return e;
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
    if (prec == GB_PREC_EMULATED_BF16) {
        set_error("the host-buffer GEMM takes native, E4M3-digit or residue precision");
        return GB_ERR_UNSUPPORTED;
    }
    if (prec != GB_PREC_NATIVE && prec != GB_PREC_EMULATED && prec != GB_PREC_EMULATED_CRT) {
        set_error("unknown precision %d", (int)prec);
        return GB_ERR_INVALID_ARG;
    }
    const int s = slices == 0 ? (prec == GB_PREC_EMULATED_CRT ? kCrtDefaultModuli : 11) : slices;
    if (prec == GB_PREC_EMULATED && (s < 1 || s > 16)) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    if (prec == GB_PREC_EMULATED_CRT && (s < 1 || s > kCrtMaxModuli)) {
        set_error("the number of moduli must be in [1, %d] (or 0), got %d", kCrtMaxModuli, slices);
        return GB_ERR_INVALID_ARG;
    }
    *out = host_layout(prec, s, m, n, k).total;
    return GB_OK;
}

gb_status gb_dgemm_host_schedule(int slices, int64_t m, int64_t n, int64_t k, double beta,
                                 int sm_count, int64_t* pieces, int max_pieces, int* count) {
    if (!count || (max_pieces > 0 && !pieces)) {
        set_error("count is NULL, or pieces is NULL with max_pieces > 0");
        return GB_ERR_INVALID_ARG;
    }
    *count = 0;
    if (m < 0 || n < 0 || k < 0 || sm_count < 1) {
        set_error("m, n, k must be >= 0 and sm_count >= 1");
        return GB_ERR_INVALID_ARG;
    }
    const int s = slices == 0 ? 11 : slices;
    if (s < 1 || s > 16) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    if (m == 0 || n == 0 || k == 0) return GB_OK;
    const HostSchedule sch = host_schedule(s, m, n, k, beta != 0.0, sm_count);
    *count = sch.np;
    if (max_pieces < sch.np) {
        set_error("%d launches do not fit max_pieces = %d", sch.np, max_pieces);
        return GB_ERR_INVALID_ARG;
    }
    for (int p = 0; p < sch.np; ++p) {
        pieces[4 * p + 0] = sch.piece[p].r0;
        pieces[4 * p + 1] = sch.piece[p].r1;
        pieces[4 * p + 2] = sch.piece[p].c0;
        pieces[4 * p + 3] = sch.piece[p].c1;
    }
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
    if (prec == GB_PREC_EMULATED_BF16) {
        set_error("the host-buffer GEMM takes native, E4M3-digit or residue precision");
        return GB_ERR_UNSUPPORTED;
    }
    if (prec != GB_PREC_NATIVE && prec != GB_PREC_EMULATED && prec != GB_PREC_EMULATED_CRT) {
        set_error("unknown precision %d", (int)prec);
        return GB_ERR_INVALID_ARG;
    }
    const bool crt = prec == GB_PREC_EMULATED_CRT;
    const int s = slices == 0 ? (crt ? kCrtDefaultModuli : 11) : slices;
    if (prec == GB_PREC_EMULATED && (s < 1 || s > 16)) {
        set_error("slices must be in [1, 16] (or 0 for the default), got %d", slices);
        return GB_ERR_INVALID_ARG;
    }
    if (crt && (s < 1 || s > kCrtMaxModuli)) {
        set_error("the number of moduli must be in [1, %d] (or 0), got %d", kCrtMaxModuli, slices);
        return GB_ERR_INVALID_ARG;
    }
    if (crt && k > 0 && crt_scale_bits(s, k) < 1) {
        set_error("k = %lld is too long for %d moduli", (long long)k, s);
        return GB_ERR_UNSUPPORTED;
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

    if (crt) {
        e = crt_host_pipeline(L, hs, ds, ev, s, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                              crt_layout(s, m, n, k), dA, dB, dC);
        // the queue completes when C is back in host memory
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], ds);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[0], 0);
        return finish_call(q, e, "host-buffer emulated (residues) dgemm");
    }
    const EmuLayout lay = emu_layout(s, m, n, k);
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    const HostSchedule sch = host_schedule(s, m, n, k, reads_c, q->dev->sm_count);
    cudaEvent_t* ev_b = ev + 1;                // column blocks of B in
    cudaEvent_t* ev_a = ev + 1 + kMaxBBlocks;  // row bands of A (and C) in
    cudaEvent_t* ev_p = ev_a + kMaxBands;      // products launches done
    auto copy_b = [&](int j) {
        const int64_t c0 = sch.bcut[j], c1 = sch.bcut[j + 1];
        cudaError_t r = copy_rows(dB + c0, 8 * (size_t)n, B + c0, 8 * (size_t)ldb, c1 - c0, k,
                                  cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_b[j], hs) : r;
    };
    auto copy_a = [&](int i) {
        int64_t r0, r1;
        band_rows(m, sch.nb, i, &r0, &r1);
        cudaError_t r = copy_rows(dA + r0 * kk, 8 * (size_t)kk, A + r0 * lda, 8 * (size_t)lda, k,
                                  r1 - r0, cudaMemcpyHostToDevice, hs);
        if (r == cudaSuccess && reads_c)
            r = copy_rows(dC + r0 * n, 8 * (size_t)n, C + r0 * ldc, 8 * (size_t)ldc, n, r1 - r0,
                          cudaMemcpyHostToDevice, hs);
        return r == cudaSuccess ? cudaEventRecord(ev_a[i], hs) : r;
    };
    // h2d in the order the launches need it: B's first column block, A's first row
    // band, B's other blocks, A's other row bands (each with C's rows)
    if (e == cudaSuccess) e = copy_b(0);
    if (e == cudaSuccess) e = copy_a(0);
    for (int j = 1; j < sch.nbb && e == cudaSuccess; ++j) e = copy_b(j);
    for (int i = 1; i < sch.nb && e == cudaSuccess; ++i) e = copy_a(i);
    // queue: each block of B split as it arrives, each band of A split before its
    // first launch, then the launches in schedule order; d2h: each block of C as soon
    // as it is computed.  Band and block edges sit on tile edges (128 rows, bn
    // columns), so a piece's digit tiles start r0 * kp * s (c0 * kp * s) bytes into
    // the planes.
    auto split_b = [&](int j) {
        const int64_t c0 = sch.bcut[j], c1 = sch.bcut[j + 1];
        const size_t boff = (size_t)c0 * (size_t)lay.kp * (size_t)s;
        cudaError_t r = cudaStreamWaitEvent(qs, ev_b[j], 0);
        if (r == cudaSuccess)
            r = launch_split_cols(L, s, c1 - c0, k, dB + c0, n, ws + lay.b_digits + boff, lay.kp,
                                  fb + c0, reinterpret_cast<uint64_t*>(ws + lay.b_part));
        return r;
    };
    auto split_a = [&](int i) {
        int64_t r0, r1;
        band_rows(m, sch.nb, i, &r0, &r1);
        const size_t aoff = (size_t)r0 * (size_t)lay.kp * (size_t)s;
        cudaError_t r = cudaStreamWaitEvent(qs, ev_a[i], 0);
        if (r == cudaSuccess)
            r = launch_split_rows(L, s, r1 - r0, k, dA + r0 * kk, kk, ws + lay.a_digits + aoff,
                                  lay.kp, ea + r0);
        return r;
    };
    int band = -1;
    for (int p = 0; p < sch.np && e == cudaSuccess; ++p) {
        const Piece& pc = sch.piece[p];
        if (pc.bblock >= 0) e = split_b(pc.bblock);
        if (e == cudaSuccess && pc.band != band) {
            band = pc.band;
            e = split_a(band);
        }
        if (e != cudaSuccess) break;
        const size_t aoff = (size_t)pc.r0 * (size_t)lay.kp * (size_t)s;
        const size_t boff = (size_t)pc.c0 * (size_t)lay.kp * (size_t)s;
        e = launch_emu_products(L, s, pc.r1 - pc.r0, pc.c1 - pc.c0, k, alpha, beta,
                                dC + pc.r0 * n + pc.c0, n, ws + lay.a_digits + aoff,
                                ws + lay.b_digits + boff, lay.kp, ea + pc.r0, fb + pc.c0);
        if (e == cudaSuccess) e = cudaEventRecord(ev_p[p], qs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, ev_p[p], 0);
        if (e == cudaSuccess)
            e = copy_rows(C + pc.r0 * ldc + pc.c0, 8 * (size_t)ldc, dC + pc.r0 * n + pc.c0,
                          8 * (size_t)n, pc.c1 - pc.c0, pc.r1 - pc.r0, cudaMemcpyDeviceToHost, ds);
    }
    // the queue completes when C is back in host memory
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], ds);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qs, ev[0], 0);
    return finish_call(q, e, "host-buffer emulated dgemm");
}

}  // extern "C"
