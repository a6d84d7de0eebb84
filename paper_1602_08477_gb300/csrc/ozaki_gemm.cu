// Emulated FP64 GEMM, steps e3 + e4 on the tcgen05 tensor cores.
//
// e3: for an output tile of 128 rows x BN columns, the level sums
//       S_g = sum_{p + q = g} DA_p DB_q^T,  g = 2 .. s+1,
//     of the E4M3 digit planes (|digit| <= 16) are accumulated in tensor memory,
//     one FP32 accumulator of 128 lanes x BN columns per level (s * BN <= 512
//     columns).  Every digit product is an integer <= 256, so each partial sum is
//     an exact integer in FP32 while it stays below 2^24 (k * pairs * 256).
// e4: the epilogue reads the levels back, forms the exact integer
//       T = sum_g S_g 2^(5 (s+1-g))
//     in 128-bit integer arithmetic, rounds it once to FP64 (nearest, ties to
//     even), scales by the power of two 2^(e_i + f_j - 8 - 5 (s-1)) and writes
//     C = alpha t + beta C.  GB300 runs FP64 at a small fraction of its integer
//     rate, so only the alpha / beta step uses the FP64 pipe.
//
// Pipeline per CTA (one output tile, 192 threads):
//   warp 0 lane 0 : producer.  Stage = one 32-byte K block of all s digit planes
//                   of A (128 x 32 B each) and B (BN x 32 B each).  The split
//                   kernels store each such block pre-tiled and pre-swizzled
//                   (the 32-byte-swizzled K-major image the tensor core reads),
//                   so a stage is two contiguous 1-D bulk copies (s * 4 KiB and
//                   s * 1 KiB) instead of thousands of 32-byte row requests.
//   warp 1        : allocates 512 TMEM columns; lane 0 issues the pair
//                   products of a stage (M = 128, K = 32, N up to 256; all pairs
//                   sharing an A slice go into one MMA) and commits each stage
//                   back to the producer.
//   warps 2 - 17  : epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                   the 8 columns of group (w - 2) / 4 of every level.
// Every wait on an mbarrier is bounded (wall-clock); on a timeout the CTA records
// the timeout bit in the status word, skips its output and still frees TMEM.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

#define GB_BAD_LINE_DEV 0x40000000

namespace gb {
namespace {

constexpr int kBM = kEmuBM;
constexpr int kBN = kEmuGroupBN;
constexpr int kBKBytes = 32;
constexpr int kEpiWarps = 16;    // 4 TMEM lane quarters x 4 column groups of 8
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s
constexpr int kSmemLimit = 227 * 1024;

struct SmemTail {
    uint64_t bars[2 * 8 + 3];
    uint32_t tmem_holder;
    int abort;
};

// exact integer value of an FP32 that holds an integer (|v| < 2^63)
__device__ __forceinline__ int64_t f32_int_value(uint32_t b) {
    const uint32_t a = b & 0x7FFFFFFFu;
    if (a == 0) return 0;
    const int ex = (int)(a >> 23) - 127;
    if (ex < 0) return 0;  // not an integer: cannot occur for digit products
    const int64_t mant = (int64_t)((a & 0x7FFFFFu) | 0x800000u);
    const int64_t v = ex >= 23 ? (mant << (ex - 23)) : (mant >> (23 - ex));
    return (b >> 31) ? -v : v;
}

struct I128 {
    int64_t hi;
    uint64_t lo;
};

__device__ __forceinline__ void i128_horner(I128& x, int sh, int64_t v) {
    // x = x * 2^sh + v   (1 <= sh <= 63)
    x.hi = (int64_t)(((uint64_t)x.hi << sh) | (x.lo >> (64 - sh)));
    x.lo <<= sh;
    const uint64_t vlo = (uint64_t)v;
    const int64_t vhi = v < 0 ? -1 : 0;
    const uint64_t nlo = x.lo + vlo;
    x.hi += vhi + (nlo < x.lo ? 1 : 0);
    x.lo = nlo;
}

__device__ __forceinline__ double pow2(int e) {  // exact for -1022 <= e <= 1023
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// RN(T) * 2^E as an FP64 (T a signed 128-bit integer).  The scaling is exact
// when the result is a normal double; otherwise RN(T) is multiplied by powers
// of two in the normal range (one multiplication, or two when E is out of it).
__device__ __forceinline__ double i128_to_double_scaled(I128 x, int E) {
    const bool neg = x.hi < 0;
    uint64_t hi = (uint64_t)x.hi, lo = x.lo;
    if (neg) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0 ? 1 : 0);
    }
    if (hi == 0 && lo == 0) return 0.0;
    int p = hi ? 64 + 63 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    uint64_t M;
    if (p <= 52) {
        M = lo << (52 - p);
    } else {
        const int sh = p - 52;  // 1 .. 74
        uint64_t rem_hi, rem_lo, half_hi, half_lo;
        if (sh < 64) {
            M = (lo >> sh) | (sh ? (hi << (64 - sh)) : 0);
            rem_hi = 0;
            rem_lo = lo & ((1ull << sh) - 1);
            half_hi = 0;
            half_lo = 1ull << (sh - 1);
        } else {
            const int s2 = sh - 64;
            M = hi >> s2;
            rem_hi = s2 ? (hi & ((1ull << s2) - 1)) : 0;
            rem_lo = lo;
            half_hi = s2 ? (1ull << (s2 - 1)) : 0;
            half_lo = s2 ? 0 : (1ull << 63);
        }
        const bool gt = rem_hi > half_hi || (rem_hi == half_hi && rem_lo > half_lo);
        const bool eq = rem_hi == half_hi && rem_lo == half_lo;
        if (gt || (eq && (M & 1))) {
            M += 1;
            if (M == (1ull << 53)) {
                M >>= 1;
                p += 1;
            }
        }
    }
    const int biased = p + E + 1023;
    double r;
    if (biased >= 1 && biased <= 2046) {
        r = __longlong_as_double((long long)(((uint64_t)biased << 52) | (M & 0xFFFFFFFFFFFFFull)));
    } else {
        double t = __longlong_as_double(
            (long long)(((uint64_t)(p + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull)));
        if (E >= -1022 && E <= 1023) {
            t = __dmul_rn(t, pow2(E));
        } else {
            const int E1 = (E >= 0) ? E / 2 : -((-E + 1) / 2);  // floor(E / 2)
            t = __dmul_rn(__dmul_rn(t, pow2(E1)), pow2(E - E1));
        }
        r = t;
    }
    return neg ? -r : r;
}

// Arguments of one output tile (row0, col0) of one problem.
struct TileArgs {
    const uint8_t* a_src;  // A digit tiles of this tile row, K block 0 (s * 4 KiB per block)
    const uint8_t* b_src;  // B digit tiles of this tile column, K block 0 (s * 1 KiB per block)
    int s, nkb;
    int64_t m, n, ldc, row0, col0;
    double alpha, beta;
    double* C;
    const int32_t* eA;  // row exponents (indexed by row)
    const int32_t* fB;  // column exponents (indexed by column)
};

// One 128 x BN output tile: level sums on the tensor cores, recombination into
// C.  All 192 threads call it; `smem` is 1024-byte aligned and holds `stages`
// ring slots of `slot_bytes` plus a SmemTail.
// The MMAs of one K block (32 bytes) of all slice pairs, with compile-time slice
// count S: for a fixed A slice p the pairs (p, q), q = 1 .. S+1-p, land in the
// consecutive levels p-1 .. S-1, whose accumulators are consecutive TMEM column
// blocks, and the B slices q are consecutive in shared memory.  So one MMA with
// N = 32 (S+1-p) (split at the 256-column limit) covers them all, reading the A
// tile once.  Fully unrolled: descriptor offsets are immediates, so the single
// issuing thread spends a few instructions per MMA.
template <int S>
__device__ __forceinline__ void issue_kblock(uint64_t adesc, uint64_t bdesc, uint32_t tmem_base,
                                             bool first) {
#pragma unroll
    for (int p = 1; p <= S; ++p) {
        const uint64_t ad = adesc + (uint64_t)(((p - 1) * kBM * kBKBytes) >> 4);
        const uint32_t acc = (first && p == 1) ? 0u : 1u;
        constexpr int kUnused = 0;
        (void)kUnused;
        const int rows = kBN * (S + 1 - p);
#pragma unroll
        for (int r0 = 0; r0 < kBN * S; r0 += 256) {
            if (r0 < rows) {
                const int nn = rows - r0 < 256 ? rows - r0 : 256;
                const uint64_t bd = bdesc + (uint64_t)((r0 * kBKBytes) >> 4);
                ptx::mma_e4m3(tmem_base + (uint32_t)((p - 1) * kBN + r0), ad, bd,
                              ptx::idesc_e4m3_f32(kBM, nn), acc);
            }
        }
    }
}

// K blocks per pipeline stage for S slices: as many as keep two stages in 227 KB
// (at most 4), so the per-stage wait / fence / commit of the issuing thread is
// shared by KB K blocks.
__host__ __device__ constexpr int kblocks_per_stage(int S) {
    return ((kSmemLimit - 2048) / (2 * S * (kBM + kBN) * kBKBytes)) < 1
               ? 1
               : ((kSmemLimit - 2048) / (2 * S * (kBM + kBN) * kBKBytes)) > 4
                     ? 4
                     : ((kSmemLimit - 2048) / (2 * S * (kBM + kBN) * kBKBytes));
}

// Persistent CTA over output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (tile_of(t) gives a tile's arguments; every role walks the same sequence).
// Barriers and the TMEM allocation live for the whole CTA: the producer runs
// ahead into the next tile's stages, and the epilogue hands TMEM back (tmem_empty)
// as soon as it has read the level sums, so the next tile's MMAs overlap its
// rounding and stores.  `smem` is 1024-byte aligned and holds `stages` ring slots
// of `slot_bytes` (>= KB * S * 5 KiB) plus a SmemTail.  A stage holds KB
// consecutive K blocks: their A tiles (KB * S * 4 KiB, contiguous in the
// workspace) then their B tiles (KB * S * 1 KiB).
template <int S, int KB, class TileFn>
__device__ __forceinline__ void products_persistent(const TileFn& tile_of, int64_t t_begin,
                                                    int64_t t_end, uint8_t* smem, int stages,
                                                    uint32_t slot_bytes, unsigned* status) {
    constexpr int BN = kBN;
    SmemTail* tail = reinterpret_cast<SmemTail*>(smem + (size_t)stages * slot_bytes);
    uint64_t* full = tail->bars;
    uint64_t* empty = tail->bars + stages;
    uint64_t* tmem_full = tail->bars + 2 * stages;
    uint64_t* tmem_empty = tail->bars + 2 * stages + 1;
    uint64_t* drain = tail->bars + 2 * stages + 2;
    volatile int* abort = &tail->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = t_begin + blockIdx.x, dt = gridDim.x;

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        ptx::mbar_init(tmem_full, 1);
        ptx::mbar_init(tmem_empty, kEpiWarps);
        ptx::mbar_init(drain, 1);
        tail->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 1) {
        ptx::tmem_alloc(&tail->tmem_holder, kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = tail->tmem_holder;
    constexpr uint32_t a_bytes = (uint32_t)S * kBM * kBKBytes;  // one K block
    constexpr uint32_t b_bytes = (uint32_t)S * BN * kBKBytes;

    if (warp == 0 && lane == 0) {
        // ---- producer: two contiguous bulk copies per stage, across tiles ----
        uint32_t it = 0;
        for (int64_t t = t0; t < t_end && !*abort; t += dt) {
            const TileArgs a = tile_of(t);
            const int nst = (a.nkb + KB - 1) / KB;
            for (int j = 0; j < nst; ++j, ++it) {
                const int st = (int)(it % (uint32_t)stages);
                const uint32_t ph = (it / (uint32_t)stages) & 1u;
                if (!ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs))
                    break;
                const int kb0 = j * KB;
                const int kc = a.nkb - kb0 < KB ? a.nkb - kb0 : KB;
                uint8_t* sa = smem + (size_t)st * slot_bytes;
                ptx::mbar_arrive_expect_tx(&full[st], (uint32_t)kc * (a_bytes + b_bytes));
                ptx::bulk_load(sa, a.a_src + (size_t)kb0 * a_bytes, (uint32_t)kc * a_bytes,
                               &full[st]);
                ptx::bulk_load(sa + KB * a_bytes, a.b_src + (size_t)kb0 * b_bytes,
                               (uint32_t)kc * b_bytes, &full[st]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        uint32_t it = 0, tile_iter = 0;
        for (int64_t t = t0; t < t_end && !*abort; t += dt, ++tile_iter) {
            const TileArgs a = tile_of(t);
            const int nst = (a.nkb + KB - 1) / KB;
            if (tile_iter > 0) {
                // the epilogue has read the previous tile's accumulators
                if (!ptx::mbar_wait_bounded(tmem_empty, (tile_iter - 1) & 1u, abort, status,
                                            kStatusTimeout, kWaitTimeoutNs))
                    break;
                ptx::tc_fence_after();
            }
            for (int j = 0; j < nst; ++j, ++it) {
                const int st = (int)(it % (uint32_t)stages);
                const uint32_t ph = (it / (uint32_t)stages) & 1u;
                if (!ptx::mbar_wait_bounded(&full[st], ph, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs))
                    break;
                ptx::tc_fence_after();
                const uint32_t a0 = ptx::smem_u32(smem + (size_t)st * slot_bytes);
                const uint64_t adesc = ptx::umma_desc_sw32(a0);
                const uint64_t bdesc = ptx::umma_desc_sw32(a0 + KB * a_bytes);
                const int kc = a.nkb - j * KB < KB ? a.nkb - j * KB : KB;
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    if (kk < kc)
                        issue_kblock<S>(adesc + (uint64_t)((kk * a_bytes) >> 4),
                                        bdesc + (uint64_t)((kk * b_bytes) >> 4), tmem_base,
                                        j == 0 && kk == 0);
                }
                ptx::mma_commit(&empty[st]);
            }
            ptx::mma_commit(tmem_full);
        }
    } else if (warp >= 2) {
        // ---- epilogue ----
        // T = sum_g S_g 2^(5 (s+1-g)) exactly: Horner in int64 over groups of at
        // most 6 levels (each group stays below 2^53 for k * pairs * 256 < 2^28),
        // folded into a 128-bit integer at group ends; one rounding to FP64.
        const int quarter = warp & 3;
        const int cgroup = (warp - 2) >> 2;
        const uint32_t col_addr = tmem_base + ((uint32_t)(quarter * 32) << 16) + cgroup * 8;
        uint32_t tile_iter = 0;
        for (int64_t t = t0; t < t_end; t += dt, ++tile_iter) {
            const TileArgs a = tile_of(t);
            const bool ok = ptx::mbar_wait_bounded(tmem_full, tile_iter & 1u, abort, status,
                                                   kStatusTimeout, kWaitTimeoutNs);
            ptx::tc_fence_after();
            if (!ok || *abort) break;
            I128 T[8];
            int64_t G[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                T[j] = I128{0, 0};
                G[j] = 0;
            }
            int in_group = 0;
#pragma unroll 1
            for (int g = 2; g <= S + 1; ++g) {
                uint32_t v[8];
                ptx::tmem_ld_32x32b_x8(col_addr + (uint32_t)(g - 2) * BN, v);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 8; ++j) G[j] = G[j] * 32 + f32_int_value(v[j]);
                ++in_group;
                if (in_group == 6 || g == S + 1) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        i128_horner(T[j], 5 * in_group, G[j]);
                        G[j] = 0;
                    }
                    in_group = 0;
                }
            }
            // accumulators read: hand TMEM to the next tile's MMAs
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(tmem_empty);
            const int64_t row = a.row0 + quarter * 32 + lane;
            if (row < a.m) {
                const int32_t ei = a.eA[row];
                const bool bad_row = ei == GB_BAD_LINE_DEV;
                const int Ebase = -8 - 5 * (S - 1);
                const bool plain = (a.alpha == 1.0 && a.beta == 0.0);
                double* crow = a.C + row * a.ldc;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t col = a.col0 + cgroup * 8 + j;
                    if (col < a.n) {
                        const int32_t fj = a.fB[col];
                        double out;
                        if (bad_row || fj == GB_BAD_LINE_DEV) {
                            out = __longlong_as_double(0x7FF8000000000000ll);
                        } else {
                            const double tv = i128_to_double_scaled(T[j], ei + fj + Ebase);
                            if (plain) {
                                out = tv;
                            } else {
                                out = __dmul_rn(a.alpha, tv);
                                if (a.beta != 0.0) out = __dadd_rn(out, __dmul_rn(a.beta, crow[col]));
                            }
                        }
                        crow[col] = out;
                    }
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        if (lane == 0 && *abort) {
            // make sure no MMA is still writing the accumulators before freeing them
            volatile int dummy = 0;
            ptx::mma_commit(drain);
            ptx::mbar_wait_bounded(drain, 0, &dummy, nullptr, 0, kWaitTimeoutNs);
        }
        __syncwarp();
        ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

__device__ __forceinline__ uint8_t* aligned_smem(uint8_t* raw) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
}

// One GEMM: persistent CTAs over its tiles in the rasterised order (groups of 8
// tile rows sweep the tile columns, so concurrent CTAs share A and B strips in L2).
template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    emu_products_kernel(const uint8_t* __restrict__ ad, const uint8_t* __restrict__ bd,
                        int64_t m, int64_t n, int nkb, double alpha, double beta,
                        double* __restrict__ C, int64_t ldc, const int32_t* __restrict__ eA,
                        const int32_t* __restrict__ fB, int tiles_m, int tiles_n, int stages,
                        uint32_t slot_bytes, unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    auto tile_of = [&](int64_t t) {
        const int bid = (int)t;
        const int group_size = 8 * tiles_n;
        const int first_m = (bid / group_size) * 8;
        const int gm = min(tiles_m - first_m, 8);
        const int tm = first_m + (bid % group_size) % gm;
        const int tn = (bid % group_size) / gm;
        TileArgs a;
        a.a_src = ad + (size_t)tm * nkb * S * kBM * kBKBytes;
        a.b_src = bd + (size_t)tn * nkb * S * kBN * kBKBytes;
        a.s = S;
        a.nkb = nkb;
        a.m = m;
        a.n = n;
        a.ldc = ldc;
        a.row0 = (int64_t)tm * kBM;
        a.col0 = (int64_t)tn * kBN;
        a.alpha = alpha;
        a.beta = beta;
        a.C = C;
        a.eA = eA;
        a.fB = fB;
        return a;
    };
    products_persistent<S, kblocks_per_stage(S)>(tile_of, 0, (int64_t)tiles_m * tiles_n, smem,
                                                  stages, slot_bytes, status);
}

// Grouped: persistent CTAs over the tiles [t_begin, t_end) of the problems of one
// slice count S (the table keeps problems of equal s together).
template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    grouped_products_kernel(const EmuProb* __restrict__ P, int np, int64_t t_begin,
                            int64_t t_end, int stages, uint32_t slot_bytes, unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    auto tile_of = [&](int64_t t) {
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P[mid].first_tile <= t) lo = mid; else hi = mid - 1;
        }
        const EmuProb& q = P[lo];
        const int64_t local = t - q.first_tile;
        const int64_t tm = local / q.tiles_n, tn = local % q.tiles_n;
        const int nkb = (int)(q.kp / kBKBytes);
        TileArgs a;
        a.a_src = q.a_digits + (size_t)tm * nkb * S * kBM * kBKBytes;
        a.b_src = q.b_digits + (size_t)tn * nkb * S * kBN * kBKBytes;
        a.s = S;
        a.nkb = nkb;
        a.m = q.m;
        a.n = q.n;
        a.ldc = q.ldc;
        a.row0 = tm * kBM;
        a.col0 = tn * kBN;
        a.alpha = q.alpha;
        a.beta = q.beta;
        a.C = q.C;
        a.eA = q.a_exp;
        a.fB = q.b_exp;
        return a;
    };
    products_persistent<S, kblocks_per_stage(S)>(tile_of, t_begin, t_end, smem, stages,
                                                  slot_bytes, status);
}

struct RingShape {
    int stages;
    uint32_t slot_bytes;
    size_t smem;
};

RingShape ring_for(int max_s, int kb_per_stage) {
    RingShape r{};
    r.slot_bytes = (uint32_t)kb_per_stage * max_s * (kBM + kBN) * kBKBytes;
    const int fixed = 1024 + (int)sizeof(SmemTail) + 64;
    r.stages = (kSmemLimit - fixed) / (int)r.slot_bytes;
    if (r.stages > 8) r.stages = 8;
    r.smem = (size_t)r.stages * r.slot_bytes + fixed;
    return r;
}

template <typename K>
cudaError_t allow_smem(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

template <int S>
cudaError_t launch_products_s(const Launch& L, int64_t m, int64_t n, int64_t kp, double alpha,
                              double beta, double* C, int64_t ldc, const uint8_t* ad,
                              const uint8_t* bd, const int32_t* ea, const int32_t* fb) {
    const RingShape r = ring_for(S, kblocks_per_stage(S));
    if (r.stages < 2) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(emu_products_kernel<S>);
    if (e != cudaSuccess) return e;
    const int tiles_m = (int)((m + kBM - 1) / kBM), tiles_n = (int)((n + kBN - 1) / kBN);
    const int nkb = (int)(kp / kBKBytes);
    const int64_t tiles = (int64_t)tiles_m * tiles_n;
    const int grid = (int)(tiles < L.sm_count ? tiles : L.sm_count);
    emu_products_kernel<S><<<grid, kThreads, r.smem, L.stream>>>(
        ad, bd, m, n, nkb, alpha, beta, C, ldc, ea, fb, tiles_m, tiles_n, r.stages,
        r.slot_bytes, L.status);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_grouped_s(const Launch& L, const EmuProb* probs, int np, int64_t t_begin,
                             int64_t t_end) {
    const RingShape r = ring_for(S, kblocks_per_stage(S));
    if (r.stages < 2) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(grouped_products_kernel<S>);
    if (e != cudaSuccess) return e;
    const int64_t tiles = t_end - t_begin;
    const int grid = (int)(tiles < L.sm_count ? tiles : L.sm_count);
    grouped_products_kernel<S><<<grid, kThreads, r.smem, L.stream>>>(probs, np, t_begin, t_end,
                                                                     r.stages, r.slot_bytes,
                                                                     L.status);
    return cudaGetLastError();
}

}  // namespace

#define GB_CASES(CALL)                                                                     \
    CALL(1) CALL(2) CALL(3) CALL(4) CALL(5) CALL(6) CALL(7) CALL(8) CALL(9) CALL(10)       \
        CALL(11) CALL(12) CALL(13) CALL(14) CALL(15) CALL(16)

cudaError_t launch_emu_products(const Launch& L, int s, int64_t m, int64_t n, int64_t k,
                                double alpha, double beta, double* C, int64_t ldc,
                                const uint8_t* a_digits, const uint8_t* b_digits, int64_t kp,
                                const int32_t* a_exp, const int32_t* b_exp) {
    (void)k;
    if (m == 0 || n == 0) return cudaSuccess;
    switch (s) {
#define GB_CASE(SS)                                                                          \
    case SS:                                                                                 \
        return launch_products_s<SS>(L, m, n, kp, alpha, beta, C, ldc, a_digits, b_digits, \
                                     a_exp, b_exp);
        GB_CASES(GB_CASE)
#undef GB_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grouped_products(const Launch& L, const EmuProb* probs, int np,
                                    int64_t t_begin, int64_t t_end, int s) {
    if (np == 0 || t_end <= t_begin) return cudaSuccess;
    switch (s) {
#define GB_CASE(SS) \
    case SS: return launch_grouped_s<SS>(L, probs, np, t_begin, t_end);
        GB_CASES(GB_CASE)
#undef GB_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
