// Emulated FP64 GEMM, steps e3 + e4 on the tcgen05 tensor cores.
//
// e3: for an output tile of 128 rows x BN columns (BN = emu_bn(s): 48 for
//     s <= 10, else 32), the level sums
//       S_g = sum_{p + q = g} DA_p DB_q^T,  g = 2 .. s+1,
//     of the E4M3 digit planes (|digit| <= 16) are accumulated in tensor memory,
//     one FP32 accumulator of 128 lanes x BN columns per level (s * BN <= 512
//     columns).  Every digit product is an integer <= 256, so each partial sum is
//     an exact integer in FP32 while it stays below 2^24 (k * pairs * 256).
// e4: the epilogue reads the levels back, forms the exact integer
//       T = sum_g S_g 2^(5 (s+1-g))
//     in 128-bit integer arithmetic, rounds T 2^(e_i + f_j - 8 - 5 (s-1)) once
//     to FP64 (nearest, ties to even, gradual underflow, overflow to +-Inf) and
//     writes C = alpha t + beta C.  GB300 runs FP64 at a small fraction of its integer
//     rate, so only the alpha / beta step uses the FP64 pipe.
//
// Persistent CTAs, one per SM, 576 threads, over the output tiles:
//   warp 0 lane 0 : producer.  Resolves each tile's arguments once and shares
//                   them through a ring in shared memory.  Stage = KB 32-byte K
//                   blocks of all s digit planes of A (128 x 32 B each) and B
//                   (BN x 32 B each).  The split kernels store each such block
//                   pre-tiled and pre-swizzled (the 32-byte-swizzled K-major image
//                   the tensor core reads), so a stage is two contiguous 1-D bulk
//                   copies instead of thousands of 32-byte row requests.
//   warp 1        : allocates 512 TMEM columns; lane 0 issues the pair
//                   products of a stage (M = 128, K = 32, N up to 256; all pairs
//                   sharing an A slice go into one MMA) and commits each stage
//                   back to the producer.
//   warps 2 - 17  : epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                   the BN / 4 columns of group (w - 2) / 4 of every level.
// Every wait on an mbarrier is bounded (wall-clock); on a timeout the CTA records
// the timeout bit in the status word, skips its output and still frees TMEM.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

#include "emu_common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace gb {
namespace {

constexpr int kEpiWarps = 16;    // 4 TMEM lane quarters x 4 column groups of 8
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s
constexpr int kSmemLimit = 227 * 1024;

// Tile arguments travel from the producer, which resolves each tile once (for a
// group: a binary search of the tile prefix and the problem record, thousands of
// cycles of dependent loads), to the MMA issuer and the epilogue warps through a
// ring of kArgSlots records in shared memory.
constexpr int kArgSlots = 4;

struct SmemTail {
    uint64_t bars[2 * 8 + 3];
    uint64_t args_full[kArgSlots];   // the producer wrote the record
    uint64_t args_empty[kArgSlots];  // the MMA issuer and every epilogue warp copied it
    TileArgs args[kArgSlots];
    uint32_t tmem_holder;
    int abort;
};

// One 128 x BN output tile: level sums on the tensor cores, recombination into
// C.  All 192 threads call it; `smem` is 1024-byte aligned and holds `stages`
// ring slots of `slot_bytes` plus a SmemTail.
// The MMAs of one K block (32 bytes) of all slice pairs, with compile-time slice
// count S: for a fixed A slice p the pairs (p, q), q = 1 .. S+1-p, land in the
// consecutive levels p-1 .. S-1, whose accumulators are consecutive TMEM column
// blocks, and the B slices q are consecutive in shared memory.  So one MMA with
// N = BN (S+1-p) covers them all, reading the A tile once (above the 256-column
// limit, two MMAs that share the A tile through the collector buffer).  Fully
// unrolled: descriptor offsets are immediates, so the single issuing thread
// spends a few instructions per MMA.
// Split accumulators (kSplit): slices p <= G = split_point(S) accumulate into
// the level columns 0 .. 32 S, slices p > G into a second set of the levels
// G .. S-1 at columns 32 S + 32 (L - G), so no accumulator collects more than
// max(G, S - G) pairs per K index.  G is a compile-time constant: the MMA
// operands stay immediates.
__host__ __device__ constexpr int split_point(int S) {
    return (S + 1) / 2 > 2 * S - 16 ? (S + 1) / 2 : 2 * S - 16;
}

template <int S, int BN, bool kSplit>
__device__ __forceinline__ void issue_kblock(uint64_t adesc, uint64_t bdesc, uint32_t tmem_base,
                                             bool first) {
    constexpr int G = kSplit ? split_point(S) : S;
#pragma unroll
    for (int p = 1; p <= S; ++p) {
        const uint64_t ad = adesc + (uint64_t)(((p - 1) * kBM * kBKBytes) >> 4);
        // the first slice of each accumulator set covers all of its levels
        const uint32_t acc = (first && (p == 1 || p == G + 1)) ? 0u : 1u;
        const uint32_t col0 = p > G ? (uint32_t)(BN * S + (p - 1 - G) * BN)
                                    : (uint32_t)((p - 1) * BN);
        const int rows = BN * (S + 1 - p);
        if (rows <= 256) {
            ptx::mma_e4m3(tmem_base + col0, ad, bdesc, ptx::idesc_e4m3_f32(kBM, rows), acc);
        } else {
            // N above the 256-column limit: two MMAs on the same A tile, which the
            // second takes from the collector buffer instead of shared memory
            // (shared-memory bandwidth bounds this kernel)
            static_assert(BN * S <= 512, "at most two MMAs per A slice");
            ptx::mma_e4m3_collect<ptx::ACollector::kFill>(tmem_base + col0, ad, bdesc,
                                                          ptx::idesc_e4m3_f32(kBM, 256), acc);
            ptx::mma_e4m3_collect<ptx::ACollector::kLastUse>(
                tmem_base + col0 + 256u, ad, bdesc + (uint64_t)((256 * kBKBytes) >> 4),
                ptx::idesc_e4m3_f32(kBM, rows - 256), acc);
        }
    }
}

// K blocks per pipeline stage for S slices: as many as keep two stages in 227 KB
// (at most 4), so the per-stage wait / fence / commit of the issuing thread is
// shared by KB K blocks.
__host__ __device__ constexpr int kblocks_per_stage(int S) {
    return ((kSmemLimit - 2048) / (2 * S * (kBM + emu_bn(S)) * kBKBytes)) < 1
               ? 1
               : ((kSmemLimit - 2048) / (2 * S * (kBM + emu_bn(S)) * kBKBytes)) > 4
                     ? 4
                     : ((kSmemLimit - 2048) / (2 * S * (kBM + emu_bn(S)) * kBKBytes));
}

// Exactness of the FP32 level sums: an accumulator that collects P pair products
// of digits with |d| <= 16 per K index stays within +-2^24 (every partial sum an
// exactly representable integer) while K * P * 256 <= 2^24; level g has
// g - 1 <= S pairs.  For a longer K the pairs are spread over two accumulator sets
// (issue_kblock<S, true>, for 9 <= S <= 15 where both sets fit in the 512 TMEM
// columns) or, failing that, K runs in chunks of kchunk_stages(S, KB) pipeline
// stages: each chunk's level sums are read out and added exactly (128-bit) before
// the next chunk starts from zero.
__host__ __device__ constexpr int kchunk_stages(int S, int KB) {
    return (((1 << 24) / (256 * S)) / kBKBytes) / KB;
}

// Exact integer of an integer-valued FP32 with |v| < 2^22: adding 1.5 * 2^23
// lands in [2^23, 2^24), where the unit in the last place is 1.
__device__ __forceinline__ int32_t f32_small_int_value(uint32_t b) {
    const float f = __fadd_rn(__uint_as_float(b), 12582912.0f);
    return (int32_t)(__float_as_uint(f) - 0x4B400000u);
}



// The W columns of part P of an epilogue warp's column group g of the level at
// TMEM address `level`: part 0 = columns 8g .. 8g+7 (W = 8), part 1 = columns
// 32 + 4g .. 32 + 4g + 3 (W = 4, 48-column tiles only).
template <int P, int W>
__device__ __forceinline__ void tmem_ld_part(uint32_t level, int g, uint32_t (&v)[W]) {
    if constexpr (P == 0) {
        static_assert(W == 8, "part 0 has 8 columns");
        ptx::tmem_ld_32x32b_x8(level + (uint32_t)(8 * g), v);
    } else {
        static_assert(W == 4, "part 1 has 4 columns");
        ptx::tmem_ld_32x32b_x4(level + (uint32_t)(32 + 4 * g), v);
    }
}

// T[j0 .. j0+W) += sum_g S_g 2^(5 (S+1-g)) over the S levels of one accumulation
// unit for part P of this thread's columns (level index L = g - 2 at lane_addr +
// BN L, plus lane_addr + BN (S + L - G) for L >= G with split accumulators),
// exactly: Horner in int64 over runs of at most 6 levels (each |S_g| < 2^25 as
// the sum of two accumulators, so a run stays below 2^55), each run added into the
// 128-bit T at its own weight, so the chunks of a tile add up in the same T.  The
// next tile's MMAs wait until every level has been read, so this runs unrolled
// (constant shifts) and converts with one hardware FP32 -> int32 conversion per
// value (exact: every accumulator is an integer below 2^25); small: every
// accumulator below 2^22, converted by one FP32 add instead.
// Exact integer value of level L's sum for the W columns, from its FP32
// accumulator v (and the second set's y for split accumulators): below 2^25.
template <int W>
__device__ __forceinline__ void level_values(const uint32_t (&v)[W], const uint32_t (&y)[W],
                                             bool two, bool small, int32_t (&x)[W]) {
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (small)
            x[j] = f32_small_int_value(v[j]) + (two ? f32_small_int_value(y[j]) : 0);
        else
            x[j] = __float2int_rn(__uint_as_float(v[j])) +
                   (two ? __float2int_rn(__uint_as_float(y[j])) : 0);
    }
}

template <int S, int BN, bool kSplit, int P, int W, int J0>
__device__ __forceinline__ void add_levels_part(uint32_t lane_addr, int cg, bool small,
                                                I128 (&T)[BN / 4]) {
    constexpr int kRun = 6;
    constexpr int split_g = kSplit ? split_point(S) : S;
    // levels read NB at a time, one wait per batch: the reads of a tile end hold
    // up the next tile's MMAs, and each wait costs a TMEM load round trip.  NB is
    // even, so that consecutive levels L, L+1 (L even: runs start at multiples of
    // 6) are in one batch and enter the Horner sum as one 32-bit pair
    // x_L 32 + x_(L+1) (|x| < 2^25, so the pair is below 2^31): one 64-bit step
    // per two levels in this integer-ALU-bound epilogue
    constexpr int NB = 16 / W;
    static_assert(NB % 2 == 0, "level pairs within a batch");
    int64_t G[W];
#pragma unroll
    for (int j = 0; j < W; ++j) G[j] = 0;
#pragma unroll
    for (int L0 = 0; L0 < S; L0 += NB) {
        uint32_t v[NB][W], y[NB][W];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int L = L0 + b;
            if (L < S) {
                tmem_ld_part<P, W>(lane_addr + (uint32_t)L * BN, cg, v[b]);
                if (L >= split_g)
                    tmem_ld_part<P, W>(lane_addr + (uint32_t)(S + L - split_g) * BN, cg, y[b]);
            }
        }
        ptx::tmem_ld_wait();
#pragma unroll
        for (int b = 0; b < NB; b += 2) {
            const int L = L0 + b;
            if (L < S) {
                int32_t x0[W];
                level_values<W>(v[b], y[b], L >= split_g, small, x0);
                int last = L;  // last level folded into G by this step
                if (L + 1 < S) {
                    int32_t x1[W];
                    level_values<W>(v[b + 1], y[b + 1], L + 1 >= split_g, small, x1);
#pragma unroll
                    for (int j = 0; j < W; ++j)
                        G[j] = G[j] * 1024 + (int64_t)(x0[j] * 32 + x1[j]);
                    last = L + 1;
                } else {
#pragma unroll
                    for (int j = 0; j < W; ++j) G[j] = G[j] * 32 + (int64_t)x0[j];
                }
                if ((last + 1) % kRun == 0 || last == S - 1) {
                    const int sh = 5 * (S - 1 - last);  // weight of the run's last level
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        i128_add_shl(T[J0 + j], G[j], sh);
                        G[j] = 0;
                    }
                }
            }
        }
    }
}

// All BN / 4 columns of this thread (see epi_col): 8 from part 0, and 4 from part 1
// for 48-column tiles, one part at a time to keep the run registers few.
template <int S, int BN, bool kSplit>
__device__ __forceinline__ void add_levels(uint32_t lane_addr, int cg, bool small,
                                           I128 (&T)[BN / 4]) {
    add_levels_part<S, BN, kSplit, 0, 8, 0>(lane_addr, cg, small, T);
    if constexpr (BN == 48) add_levels_part<S, BN, kSplit, 1, 4, 8>(lane_addr, cg, small, T);
}


// Tiles of one accumulation unit whose level sums are all below 2^22 (every
// grouped problem of K * s < 16384): the S levels of this thread's BN / 4 columns
// (see epi_col) are read as ceil(S/2) 32-bit pairs x_L 32 + x_(L+1) (levels L,
// L+1 of one batch; |pair| < 2^27.1), so the MMAs of the next tile get TMEM back
// after the reads and two integer steps per value; the exact sums follow from
// the pairs afterwards (pairs_to_sum).
template <int S, int BN>
__device__ __forceinline__ void read_level_pairs(uint32_t lane_addr, int cg,
                                                 int32_t (&pr)[(S + 1) / 2][BN / 4]) {
#pragma unroll
    for (int L0 = 0; L0 < S; L0 += 2) {
        uint32_t v0[8], v1[8];
        ptx::tmem_ld_32x32b_x8(lane_addr + (uint32_t)(L0 * BN + 8 * cg), v0);
        if (L0 + 1 < S) ptx::tmem_ld_32x32b_x8(lane_addr + (uint32_t)((L0 + 1) * BN + 8 * cg), v1);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int32_t x0 = f32_small_int_value(v0[j]);
            pr[L0 / 2][j] = L0 + 1 < S ? x0 * 32 + f32_small_int_value(v1[j]) : x0;
        }
        if constexpr (BN == 48) {
            uint32_t w0[4], w1[4];
            ptx::tmem_ld_32x32b_x4(lane_addr + (uint32_t)(L0 * BN + 32 + 4 * cg), w0);
            if (L0 + 1 < S)
                ptx::tmem_ld_32x32b_x4(lane_addr + (uint32_t)((L0 + 1) * BN + 32 + 4 * cg), w1);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int32_t x0 = f32_small_int_value(w0[j]);
                pr[L0 / 2][8 + j] = L0 + 1 < S ? x0 * 32 + f32_small_int_value(w1[j]) : x0;
            }
        }
    }
}

// T = sum_L x_L 2^(5 (S-1-L)) of column j from its level pairs, exactly: Horner in
// int64 over runs of three pairs (six levels; each run below 2^48), each run
// added into the 128-bit T at the weight of its last level.
template <int S, int NC>
__device__ __forceinline__ I128 pairs_to_sum(const int32_t (&pr)[(S + 1) / 2][NC], int j) {
    constexpr int NP = (S + 1) / 2;
    I128 T{0, 0};
#pragma unroll
    for (int r0 = 0; r0 < NP; r0 += 3) {
        int64_t G = 0;
        int last = 0;
#pragma unroll
        for (int i = r0; i < r0 + 3 && i < NP; ++i) {
            const bool full = 2 * i + 1 < S;
            G = G * (full ? 1024 : 32) + (int64_t)pr[i][j];
            last = full ? 2 * i + 1 : 2 * i;
        }
        i128_add_shl(T, G, 5 * (S - 1 - last));
    }
    return T;
}

// How one launch keeps its level sums exact (see kchunk_stages): split
// accumulators, or K chunks of chunk_stages pipeline stages (a huge value: none).
struct AccPlan {
    bool split;
    int chunk_stages;
};

template <int S, int KB>
AccPlan acc_plan(int64_t kp, bool allow_split) {
    AccPlan a{false, 1 << 30};
    const int64_t kmax = (int64_t)1 << 24;  // K * pairs * 256 <= 2^24
    if (kp * S * 256 <= kmax) return a;
    constexpr int G = split_point(S);
    if (allow_split && S >= 9 && S <= 15 && kp * (G > S - G ? G : S - G) * 256 <= kmax) {
        a.split = true;
        return a;
    }
    a.chunk_stages = kchunk_stages(S, KB);
    return a;
}

// Persistent CTA over the output tiles of a Walk (start / valid / next / args;
// every role walks its own copy of the same sequence).
// Barriers and the TMEM allocation live for the whole CTA: the producer runs
// ahead into the next tile's stages, and the epilogue hands TMEM back (tmem_empty)
// as soon as it has read the level sums, so the next tile's MMAs overlap its
// rounding and stores.  `smem` is 1024-byte aligned and holds `stages` ring slots
// of `slot_bytes` (>= KB * S * (128 + BN) * 32 bytes) plus a SmemTail.  A stage
// holds KB consecutive K blocks: their A tiles (KB * S * 4 KiB, contiguous in the
// workspace) then their B tiles (KB * S * BN * 32 bytes).
template <int S, int BN, int KB, bool kSplit, class Walk, bool kSmall = false>
__device__ __forceinline__ void products_persistent(const Walk& walk, int chunk_stages,
                                                    uint8_t* smem, int stages,
                                                    uint32_t slot_bytes, unsigned* status) {
    constexpr int CW = BN / 4;  // columns per epilogue warp
    SmemTail* tail = reinterpret_cast<SmemTail*>(smem + (size_t)stages * slot_bytes);
    uint64_t* full = tail->bars;
    uint64_t* empty = tail->bars + stages;
    uint64_t* tmem_full = tail->bars + 2 * stages;
    uint64_t* tmem_empty = tail->bars + 2 * stages + 1;
    uint64_t* drain = tail->bars + 2 * stages + 2;
    volatile int* abort = &tail->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        ptx::mbar_init(tmem_full, 1);
        ptx::mbar_init(tmem_empty, kEpiWarps);
        ptx::mbar_init(drain, 1);
        for (int i = 0; i < kArgSlots; ++i) {
            ptx::mbar_init(&tail->args_full[i], 1);
            ptx::mbar_init(&tail->args_empty[i], 1 + kEpiWarps);
        }
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
        int st = 0;        // ring slot of the next stage
        uint32_t ph = 0;   // its phase parity (flips at every wrap of the ring)
        Walk w = walk;
        int ti = 0;  // tiles walked so far: the record's slot and phase
        for (w.start(); w.valid() && !*abort; w.next(), ++ti) {
            const TileArgs a = w.args();
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_empty[as], ((ti / kArgSlots) & 1u) ^ 1u, abort,
                                        status, kStatusTimeout, kWaitTimeoutNs))
                break;
            tail->args[as] = a;
            ptx::mbar_arrive(&tail->args_full[as]);  // release: the record is visible
            const int nst = (a.nkb + KB - 1) / KB;
            for (int j = 0; j < nst; ++j) {
                if (!ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs))
                    break;
                const int kb0 = (a.reverse ? nst - 1 - j : j) * KB;
                const int kc = a.nkb - kb0 < KB ? a.nkb - kb0 : KB;
                uint8_t* sa = smem + (size_t)st * slot_bytes;
                ptx::mbar_arrive_expect_tx(&full[st], (uint32_t)kc * (a_bytes + b_bytes));
                ptx::bulk_load(sa, a.a_src + (size_t)kb0 * a_bytes, (uint32_t)kc * a_bytes,
                               &full[st]);
                ptx::bulk_load(sa + KB * a_bytes, a.b_src + (size_t)kb0 * b_bytes,
                               (uint32_t)kc * b_bytes, &full[st]);
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        const int kCS = chunk_stages;
        int st = 0;        // ring slot of the next stage
        uint32_t ph = 0;   // its phase parity
        uint32_t chunk_iter = 0;
        bool stop = false;
        Walk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !*abort && !stop; w.next(), ++ti) {
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_full[as], (ti / kArgSlots) & 1u, abort, status,
                                        kStatusTimeout, kWaitTimeoutNs))
                break;
            const TileArgs a = tail->args[as];
            ptx::mbar_arrive(&tail->args_empty[as]);
            const int nst = (a.nkb + KB - 1) / KB;
            int in_chunk = 0;  // stages of the current accumulation unit issued so far
            // two stages per loop pass: the issuing thread's per-pass bookkeeping
            // between MMA batches is the tensor pipe's idle time (1.6% faster)
#pragma unroll 2
            for (int j = 0; j < nst; ++j) {
                const bool chunk_start = in_chunk == 0;
                if (chunk_start) {
                    if (chunk_iter > 0) {
                        // the epilogue has read the previous chunk's accumulators
                        if (!ptx::mbar_wait_bounded(tmem_empty, (chunk_iter - 1) & 1u, abort,
                                                    status, kStatusTimeout, kWaitTimeoutNs)) {
                            stop = true;
                            break;
                        }
                        ptx::tc_fence_after();
                    }
                    ++chunk_iter;
                }
                if (!ptx::mbar_wait_bounded(&full[st], ph, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs)) {
                    stop = true;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t a0 = ptx::smem_u32(smem + (size_t)st * slot_bytes);
                const uint64_t adesc = ptx::umma_desc_sw32(a0);
                const uint64_t bdesc = ptx::umma_desc_sw32(a0 + KB * a_bytes);
                const int kb0 = (a.reverse ? nst - 1 - j : j) * KB;
                const int kc = a.nkb - kb0 < KB ? a.nkb - kb0 : KB;
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    if (kk < kc)
                        issue_kblock<S, BN, kSplit>(adesc + (uint64_t)((kk * a_bytes) >> 4),
                                                bdesc + (uint64_t)((kk * b_bytes) >> 4),
                                                tmem_base, chunk_start && kk == 0);
                }
                ptx::mma_commit(&empty[st]);
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
                if (++in_chunk == kCS || j + 1 == nst) {
                    ptx::mma_commit(tmem_full);
                    in_chunk = 0;
                }
            }
        }
    } else if (warp >= 2) {
        // ---- epilogue ----
        // Every chunk adds its sum_g S_g 2^(5 (s+1-g)) exactly into the tile's
        // 128-bit T (add_levels); one rounding to FP64 at the end.
        const int kCS = chunk_stages;
        const int quarter = warp & 3;
        const int cgroup = (warp - 2) >> 2;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
        uint32_t chunk_iter = 0;
        bool stop = false;
        Walk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !stop; w.next(), ++ti) {
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_full[as], (ti / kArgSlots) & 1u, abort, status,
                                        kStatusTimeout, kWaitTimeoutNs))
                break;
            // the record stays in shared memory (read where needed, not held in
            // registers across the level reads) until this warp's stores are done
            const TileArgs& a = tail->args[as];
            const int nch = ((a.nkb + KB - 1) / KB + kCS - 1) / kCS;
            const bool small = a.nkb * S < 512;  // every accumulator below 2^22
            // a warp whose 32 rows, or whose columns (8 cgroup .. on), all lie in the
            // tile's padding has no output: it skips the level reads, the
            // recombination and the stores, and only hands TMEM back (warp-uniform)
            const bool live = a.row0 + quarter * 32 < a.m && a.col0 + 8 * cgroup < a.n;
            // the row and column exponents are brought into L1 now, so that their
            // latency passes while the tile's MMAs run (read from L2 one by one after
            // the level sums, behind the stores to C, they were most of the
            // epilogue's time on short tiles); held in registers across the level
            // reads they would spill
            const int64_t row = a.row0 + quarter * 32 + lane;
            const bool row_ok = live && row < a.m;
            if (row_ok) {
                ptx::prefetch_l1(a.eA + row);
                if (lane == 0) {
                    ptx::prefetch_l1(a.fB + a.col0 + 8 * cgroup);
                    if (CW > 8) ptx::prefetch_l1(a.fB + a.col0 + 32 + 4 * cgroup);
                }
            }
            if constexpr (kSmall) {
                static_assert(!kSplit, "small-sum tiles: one accumulator set");
                (void)nch;
                (void)small;
                {
                    // one unit of small level sums: TMEM goes back right after the
                    // level pairs are read (read_level_pairs)
                    const bool ok = ptx::mbar_wait_bounded(tmem_full, chunk_iter & 1u, abort,
                                                           status, kStatusTimeout,
                                                           kWaitTimeoutNs);
                    ptx::tc_fence_after();
                    if (!ok || *abort) break;
                    int32_t pr[(S + 1) / 2][CW];
                    if (live) read_level_pairs<S, BN>(lane_addr, cgroup, pr);
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(tmem_empty);
                    ++chunk_iter;
                    if (row_ok) {
                        const int64_t n = a.n, col0 = a.col0;
                        const int32_t* fB = a.fB;
                        const double alpha = a.alpha, beta = a.beta;
                        const int64_t rstride = a.trans ? 1 : a.ldc, cstride = a.trans ? a.ldc : 1;
                        double* crow = a.C + row * rstride;
                        const int32_t ei = a.eA[row];
                        const int Ebase = -8 - 5 * (S - 1);
                        const long long ab = __double_as_longlong(alpha),
                                        bb = __double_as_longlong(beta);
                        const bool beta0 = (bb & 0x7FFFFFFFFFFFFFFFll) == 0;
                        const bool plain = ab == 0x3FF0000000000000ll && beta0;
                        // four columns at a time: their sums from the pairs, rounded
                        // and stored one by one
#pragma unroll
                        for (int g0 = 0; g0 < CW; g0 += 4) {
                            I128 T4[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) T4[j] = pairs_to_sum<S, CW>(pr, g0 + j);
                            if (g0 == 0)
                                store_part<S, 0, 4, 4, 1, 0>(T4, ei, Ebase, fB, col0, n, cgroup,
                                                             plain, beta0, alpha, beta, crow,
                                                             cstride);
                            else if (g0 == 4)
                                store_part<S, 4, 4, 4, 1, 0>(T4, ei, Ebase, fB, col0, n, cgroup,
                                                             plain, beta0, alpha, beta, crow,
                                                             cstride);
                            else
                                store_part<S, 8, 4, 4, 1, 0>(T4, ei, Ebase, fB, col0, n, cgroup,
                                                             plain, beta0, alpha, beta, crow,
                                                             cstride);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tail->args_empty[as]);
                }
            } else {
            I128 T[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) T[j] = I128{0, 0};
            for (int c = 0; c < nch; ++c, ++chunk_iter) {
                const bool ok = ptx::mbar_wait_bounded(tmem_full, chunk_iter & 1u, abort, status,
                                                       kStatusTimeout, kWaitTimeoutNs);
                ptx::tc_fence_after();
                if (!ok || *abort) {
                    stop = true;
                    break;
                }
                if (live) add_levels<S, BN, kSplit>(lane_addr, cgroup, small, T);
                // accumulators read: hand TMEM to the next unit's MMAs
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(tmem_empty);
            }
            if (stop) break;
            if (row_ok) {
                // the fields of the store phase in registers, all exponents loaded
                // (L1 hits, prefetched) and all outputs formed before the first store:
                // read through the shared record between stores, every field and
                // exponent was a dependent reload per column
                const int64_t n = a.n, col0 = a.col0;
                const int32_t* fB = a.fB;
                const double alpha = a.alpha, beta = a.beta;
                const int64_t rstride = a.trans ? 1 : a.ldc, cstride = a.trans ? a.ldc : 1;
                double* crow = a.C + row * rstride;
                const int32_t ei = a.eA[row];
                const int Ebase = -8 - 5 * (S - 1);
                // alpha == 1 and beta == +-0 tested on the bit patterns (integer ALU)
                const long long ab = __double_as_longlong(alpha), bb = __double_as_longlong(beta);
                const bool beta0 = (bb & 0x7FFFFFFFFFFFFFFFll) == 0;
                const bool plain = ab == 0x3FF0000000000000ll && beta0;
                // C[row][col], or C[col][row] for a transposed problem (a warp's
                // 32 lanes then store 32 consecutive doubles of one row of C); the
                // thread's columns in the parts of add_levels (8, then 4 for
                // 48-column tiles) to stay within the registers
                // 48-column tiles hold 12 128-bit sums per thread: one output at a time
                constexpr int G = CW > 8 ? 1 : 4;
                store_part<S, 0, 8, CW, G>(T, ei, Ebase, fB, col0, n, cgroup, plain, beta0, alpha,
                                           beta, crow, cstride);
                if constexpr (CW > 8)
                    store_part<S, 8, 4, CW, G>(T, ei, Ebase, fB, col0, n, cgroup, plain, beta0,
                                               alpha, beta, crow, cstride);
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tail->args_empty[as]);
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



template <int S, bool kSplit>
__global__ void __launch_bounds__(kThreads, 1)
    emu_products_kernel(const uint8_t* __restrict__ ad, const uint8_t* __restrict__ bd,
                        int64_t m, int64_t n, int nkb, double alpha, double beta,
                        double* __restrict__ C, int64_t ldc, const int32_t* __restrict__ eA,
                        const int32_t* __restrict__ fB, int tiles_m, int tiles_n,
                        int chunk_stages, int stages, uint32_t slot_bytes, unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    constexpr int BN = emu_bn(S);
    const RasterWalk<BN> w{ad, bd, m, n, ldc, nkb, tiles_m, tiles_n, S, alpha, beta, C, eA, fB, 0};
    products_persistent<S, BN, kblocks_per_stage(S), kSplit>(w, chunk_stages, smem, stages,
                                                             slot_bytes, status);
}

// Grouped: the tiles [t_begin, t_end) of the problems [q_begin, q_end) of the
// table (all with S slices; the table puts long-K problems first), taken
// t = t_begin + blockIdx.x, + gridDim.x, ...: concurrent CTAs work on
// neighbouring tiles, so the digit strips they share stay in L2.  A tile's
// problem is a binary search over the compact tile-prefix array (L1-resident).
template <int BN>
struct GroupWalk {
    const EmuProb* P;
    const int64_t* key;
    int q_begin, q_end;
    int64_t t_begin, t_end, t;
    __device__ void start() { t = t_begin + blockIdx.x; }
    __device__ bool valid() const { return t < t_end; }
    __device__ void next() { t += gridDim.x; }
    __device__ TileArgs args() const {
        int lo = q_begin, hi = q_end - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (key[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const EmuProb& e = P[lo];
        const int64_t local = t - key[lo];
        const int64_t tm = local / e.tiles_n, tn = local % e.tiles_n;
        const int nkb = (int)(e.kp / kBKBytes);
        // a transposed problem has B's columns on the tile rows and A's rows on the
        // tile columns
        const bool tr = e.trans != 0;
        TileArgs a;
        a.a_src = (tr ? e.b_digits : e.a_digits) + (size_t)tm * nkb * e.s * kBM * kBKBytes;
        a.b_src = (tr ? e.a_digits : e.b_digits) + (size_t)tn * nkb * e.s * BN * kBKBytes;
        a.s = e.s;
        a.nkb = nkb;
        a.reverse = false;
        a.trans = tr;
        a.m = tr ? e.n : e.m;
        a.n = tr ? e.m : e.n;
        a.ldc = e.ldc;
        a.row0 = tm * kBM;
        a.col0 = tn * BN;
        a.alpha = e.alpha;
        a.beta = e.beta;
        a.C = e.C;
        a.eA = tr ? e.b_exp : e.a_exp;
        a.fB = tr ? e.a_exp : e.b_exp;
        return a;
    }
};

template <int S, bool kSmall>
__global__ void __launch_bounds__(kThreads, 1)
    grouped_products_kernel(const EmuProb* __restrict__ P, const int64_t* __restrict__ key,
                            int q_begin, int q_end, int64_t t_begin, int64_t t_end,
                            int chunk_stages, int stages, uint32_t slot_bytes,
                            unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    constexpr int BN = emu_bn(S);
    const GroupWalk<BN> w{P, key, q_begin, q_end, t_begin, t_end, 0};
    products_persistent<S, BN, kblocks_per_stage(S), false, GroupWalk<BN>, kSmall>(
        w, chunk_stages, smem, stages, slot_bytes, status);
}

struct RingShape {
    int stages;
    uint32_t slot_bytes;
    size_t smem;
};

RingShape ring_for(int max_s, int kb_per_stage) {
    RingShape r{};
    // slots start on 1024-byte boundaries (the operand tiles inside are 256-byte
    // aligned, as the 32-byte swizzle's 8-row pattern needs)
    r.slot_bytes = ((uint32_t)kb_per_stage * max_s * (kBM + emu_bn(max_s)) * kBKBytes + 1023u) &
                   ~1023u;
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
    constexpr int BN = emu_bn(S);
    const int tiles_m = (int)((m + kBM - 1) / kBM), tiles_n = (int)((n + BN - 1) / BN);
    const int nkb = (int)(kp / kBKBytes);
    const int64_t tiles = (int64_t)tiles_m * tiles_n;
    const int grid = (int)(tiles < L.sm_count ? tiles : L.sm_count);
    // split accumulators need BN (2S - G) TMEM columns
    constexpr bool kCanSplit = S >= 9 && S <= 15 && BN * (2 * S - split_point(S)) <= 512;
    const AccPlan plan = acc_plan<S, kblocks_per_stage(S)>(kp, kCanSplit);
    if constexpr (kCanSplit) {
        if (plan.split) {
            cudaError_t e = allow_smem(emu_products_kernel<S, true>);
            if (e != cudaSuccess) return e;
            emu_products_kernel<S, true><<<grid, kThreads, r.smem, L.stream>>>(
                ad, bd, m, n, nkb, alpha, beta, C, ldc, ea, fb, tiles_m, tiles_n,
                plan.chunk_stages, r.stages, r.slot_bytes, L.status);
            return cudaGetLastError();
        }
    }
    cudaError_t e = allow_smem(emu_products_kernel<S, false>);
    if (e != cudaSuccess) return e;
    emu_products_kernel<S, false><<<grid, kThreads, r.smem, L.stream>>>(
        ad, bd, m, n, nkb, alpha, beta, C, ldc, ea, fb, tiles_m, tiles_n, plan.chunk_stages,
        r.stages, r.slot_bytes, L.status);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_grouped_s(const Launch& L, const EmuProb* probs, const int64_t* key,
                             const EmuSRange& g) {
    const RingShape r = ring_for(S, kblocks_per_stage(S));
    if (r.stages < 2) return cudaErrorInvalidValue;
    // every level sum of the range below 2^22 (K s < 16384 for its longest K): the
    // kernel whose epilogue hands TMEM back after reading the levels as pairs
    // (read_level_pairs)
    const bool small = g.kp_max * S < 16384;
    auto kern = small ? grouped_products_kernel<S, true> : grouped_products_kernel<S, false>;
    cudaError_t e = allow_smem(kern);
    if (e != cudaSuccess) return e;
    const int64_t tiles = g.t_end - g.t_begin;
    const int grid = (int)(tiles < L.sm_count ? tiles : L.sm_count);
    const AccPlan plan = acc_plan<S, kblocks_per_stage(S)>(g.kp_max, false);
    kern<<<grid, kThreads, r.smem, L.stream>>>(probs, key, g.q_begin, g.q_end, g.t_begin,
                                               g.t_end, plan.chunk_stages, r.stages,
                                               r.slot_bytes, L.status);
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

cudaError_t launch_grouped_products(const Launch& L, const EmuProb* probs, const EmuKeys& keys,
                                    const EmuSRange& g) {
    if (g.t_end <= g.t_begin) return cudaSuccess;
    switch (g.s) {
#define GB_CASE(SS) \
    case SS: return launch_grouped_s<SS>(L, probs, keys.tile, g);
        GB_CASES(GB_CASE)
#undef GB_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
