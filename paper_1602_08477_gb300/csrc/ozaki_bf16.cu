// Emulated FP64 GEMM with BF16 digits: steps e1 - e4 with 8-bit signed digits
// (b1 = 7, b = 8, |d| <= 128, every such integer exact in BF16) multiplied by
// kind::f16 MMAs on the tcgen05 tensor cores.  Same operation and result model
// as the E4M3 path (ozaki_split.cu, ozaki_gemm.cu) with the digit format's own
// constants:
//   a = 2^e ( sum_t d_t 2^-(7 + 8 (t-1)) + ... ),  S_g = sum_{p+q=g} DA_p DB_q^T,
//   T = sum_g S_g 2^(8 (s+1-g)),  C = alpha RN(T 2^(e_i + f_j - 14 - 8 (s-1))) + beta C.
// Seven digits carry 55 bits of each line's scale (E4M3 needs 11 for 54) in 28
// slice pairs, each a BF16 MMA at half the FP8 rate; eight (s <= 8) carry 63.
//
// Exactness: a digit product is an integer of at most 2^14, so an FP32
// accumulator that collects up to s pair products per K index stays exact only
// for K s 2^14 <= 2^24, i.e. 144 K indices at s = 7 (E4M3: 6528).  The products
// kernel therefore reads the level sums out every unit of unit_ksteps(s) K steps
// and adds them exactly (int64, then 128-bit) in the epilogue; the levels of a
// 128 x 32 output tile take s * 32 TMEM columns, so two sets fit in the 512
// columns and the MMAs of one unit run while the epilogue reads the previous one.
//
// Digits are stored pre-tiled as for E4M3, with 16 BF16 digits (32 bytes) per K
// block: for each tile of R lines (128 for A's rows, 32 for B's columns) and each
// K step of 16 elements the s slices follow one another, each an R x 32-byte
// K-major block in the 32-byte swizzle.
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "emu_common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace gb {
namespace {

constexpr int kB = 8;        // bits of every digit after the first (the first: 7)
constexpr int kKStep = 16;   // K elements per 32-byte K block (one kind::f16 MMA)
constexpr int kBN = kBf16BN;

// ---- e1 + e2: exponents and BF16 digit planes ------------------------------------

// BF16 code of the digit d_t that a 10-bit window w = bits 8(S-t) .. 8(S-t)+9 of
// the fixed-point image determines under rounding half up (see digits_bf16):
// Q_t mod 512 = bits 1..9 of w + 1, and Q_(t-1) is odd iff bits 8, 9 of w are 01
// or 10.  A BF16 integer |d| <= 128 is the high half of its FP32 pattern.
__shared__ uint16_t s_window16[1024];

__device__ __forceinline__ void fill_bf16_table() {
    for (int x = threadIdx.x; x < 1024; x += blockDim.x) {
        const int qt = ((x + 1) >> 1) & 511;
        const int qp_odd = (((x >> 8) + 1) >> 1) & 1;
        const int dm = (qt - 256 * qp_odd) & 511;
        const int d = dm >= 256 ? dm - 512 : dm;
        s_window16[x] = (uint16_t)(d >= -128 && d <= 128 ? (__float_as_uint((float)d) >> 16) : 0u);
    }
    __syncthreads();
}

// Fixed-point image of an element for S digits: |F| < 2^(8 S), int64 for S <= 7,
// a 128-bit integer for S = 8.
template <int S>
struct Fixed16Of {
    using type = typename std::conditional<(S <= 7), int64_t, __int128>::type;
};

// The S digits of one finite double (bits) relative to its line exponent e, as
// BF16 codes in half (u & 1) of word u / 2 of each plane's 16-byte chunk out[t]
// (u = 0 .. 7 in increasing order; the caller zeroes out).
//
// With x = X 2^E2 (X the signed integer significand), digit t is
// d_t = Q_t - 256 Q_(t-1), Q_t = RNE(x 2^(7 + 8 (t-1) - e)): the recurrence
// d_t = rint(256 r), r <- 256 r - d_t, since subtracting the integer multiple
// 256 Q_(t-1) commutes with rounding to nearest even.  F = X 2^k with
// k = E2 - e + 8 S puts the unit of Q_t at bit 1 + 8 (S - t), so
// W = floor(F / 2^(8 (S-t))) and Q_t = floor((W + 1) / 2) under rounding half up;
// d_t mod 512 follows from the 10 low bits of W alone.
// Half up differs from ties-to-even only at an exact tie with an even quotient,
// which can only sit at the digit whose rounding point is F's lowest set bit;
// F - 1 gives the even quotient there and leaves every other digit unchanged
// (no lower rounding point is crossed and the higher windows see no borrow).
template <int S>
__device__ __forceinline__ void digits_bf16(uint64_t bits, int e, int u, uint32_t (&out)[S][4]) {
    using Fixed = typename Fixed16Of<S>::type;
    const int ef = (int)((bits >> 52) & 0x7FF);
    int64_t M = (int64_t)(bits & 0xFFFFFFFFFFFFFull);
    int E2;
    if (ef == 0) {
        E2 = -1074;
    } else {
        M |= (int64_t)1 << 52;
        E2 = ef - 1075;
    }
    if (M == 0) return;  // +-0: every digit 0
    const int64_t X = (bits >> 63) ? -M : M;
    const int k = E2 - e + kB * S;
    const int tzF = (__ffsll((long long)M) - 1) + k;
    Fixed F;
    if (k >= 0) F = (Fixed)X << k;  // exact: |F| < 2^(8 S)
    else F = (Fixed)(X >> (-k < 63 ? -k : 63));
    // an exact tie at a digit's rounding point with an even quotient rounds down
    const bool tie_down = tzF >= 0 && tzF <= kB * (S - 1) && tzF % kB == 0 &&
                          (((uint32_t)(F >> (tzF + 1))) & 1u) == 0u;
    F -= tie_down ? 1 : 0;
#pragma unroll
    for (int t = 1; t <= S; ++t) {
        const uint32_t w = (uint32_t)(F >> (kB * (S - t))) & 1023u;
        const uint32_t code = s_window16[w];
        // u is a compile-time constant in the unrolled callers
        out[t - 1][u >> 1] = (u & 1) ? __byte_perm(out[t - 1][u >> 1], code, 0x5410) : code;
    }
}

// Byte offset of the 16-byte chunk holding digits l0 .. l0+7 (l0 % 8 == 0) of
// digit plane t of line x, in the tiled layout with R-line tiles and nks K steps.
__device__ __forceinline__ int64_t tiled_offset16(int64_t x, int64_t l0, int t, int64_t nks,
                                                  int R, int s) {
    const int64_t tile = x / R;
    const int r = (int)(x - tile * R);
    const int chunk = (int)((l0 >> 3) & 1) ^ ((r >> 2) & 1);
    return ((tile * nks + (l0 >> 4)) * s + t) * (int64_t)(R * 32) + r * 32 + (chunk << 4);
}

// Row i of A by a CTA of 128 threads: pass 1 max |a| and finiteness, pass 2 the
// digits of 8 consecutive elements per thread (one 16-byte chunk per plane).
// Rows m <= i < (128-row tile padding) get zero digits.
template <int S>
__device__ __forceinline__ void bf16_split_row(int64_t i, int64_t m, int64_t k,
                                               const double* __restrict__ A, int64_t lda,
                                               uint8_t* __restrict__ digits, int64_t kp,
                                               int32_t* __restrict__ exps, unsigned* status,
                                               uint64_t* red, int* bad_sh) {
    const int tid = threadIdx.x;
    const int64_t nks = kp / kKStep;
    if (i >= m) {
        for (int64_t l0 = (int64_t)tid * 8; l0 < kp; l0 += (int64_t)blockDim.x * 8)
#pragma unroll
            for (int t = 0; t < S; ++t)
                *reinterpret_cast<uint4*>(digits + tiled_offset16(i, l0, t, nks, kEmuBM, S)) =
                    make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const uint64_t* row = reinterpret_cast<const uint64_t*>(A + i * lda);
    uint64_t mx = 0;
    int bad = 0;
    for (int64_t l0 = (int64_t)tid * 8; l0 < k; l0 += (int64_t)blockDim.x * 8) {
        uint64_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = l0 + u < k ? row[l0 + u] : 0ull;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint64_t a = v[u] & 0x7FFFFFFFFFFFFFFFull;
            bad |= a >= 0x7FF0000000000000ull;
            mx = (a < 0x7FF0000000000000ull && a > mx) ? a : mx;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    bad = __syncthreads_or(bad);
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        uint64_t v = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = red[w] > v ? red[w] : v;
        red[0] = v;
        *bad_sh = bad;
    }
    __syncthreads();
    const int e = frexp_exp_bits(red[0]);
    const bool is_bad = *bad_sh != 0;
    if (tid == 0) {
        exps[i] = is_bad ? GB_BAD_LINE_DEV : e;
        if (is_bad && status) atomicOr(status, kStatusNonfinite);
    }
    for (int64_t l0 = (int64_t)tid * 8; l0 < kp; l0 += (int64_t)blockDim.x * 8) {
        uint32_t w[S][4];
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0;
        if (!is_bad) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (l0 + u < k) digits_bf16<S>(row[l0 + u], e, u, w);
        }
#pragma unroll
        for (int t = 0; t < S; ++t)
            *reinterpret_cast<uint4*>(digits + tiled_offset16(i, l0, t, nks, kEmuBM, S)) =
                make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
    __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(128) bf16_split_rows_kernel(int64_t m, int64_t k,
                                                              const double* __restrict__ A,
                                                              int64_t lda,
                                                              uint8_t* __restrict__ digits,
                                                              int64_t kp,
                                                              int32_t* __restrict__ exps,
                                                              unsigned* status) {
    fill_bf16_table();
    __shared__ uint64_t red[4];
    __shared__ int bad_sh;
    const int64_t mp = (m + kEmuBM - 1) / kEmuBM * kEmuBM;
    for (int64_t i = blockIdx.x; i < mp; i += gridDim.x)
        bf16_split_row<S>(i, m, k, A, lda, digits, kp, exps, status, red, &bad_sh);
}

// Columns of B: CTA (x, y) reduces the `ks` partial maxima of columns 32 x .. +31
// (from launch_colmax_part) to their exponents (the CTAs of the first K tile also
// store them and flag non-finite columns), then transposes the tile of rows
// 64 y .. +63 through shared memory and writes its digits: thread (jj, lsub)
// takes 8 consecutive rows of column jj, one 16-byte chunk per plane.  Columns
// n <= j < (n padded to 32) get zero digits.
template <int S>
__global__ void __launch_bounds__(256) bf16_split_cols_kernel(int64_t n, int64_t k,
                                                              const double* __restrict__ B,
                                                              int64_t ldb,
                                                              uint8_t* __restrict__ digits,
                                                              int64_t kp,
                                                              int32_t* __restrict__ exps,
                                                              const uint64_t* __restrict__ part,
                                                              int ks, unsigned* status) {
    fill_bf16_table();
    __shared__ uint64_t T[64][33];
    __shared__ uint64_t red[8][32];
    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * 32, l0 = (int64_t)blockIdx.y * 64;
    const uint64_t* Bb = reinterpret_cast<const uint64_t*>(B);
    uint64_t v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t l = l0 + ty + 8 * r, j = j0 + tx;
        v[r] = (l < k && j < n) ? Bb[l * ldb + j] : 0ull;
    }
    {
        // two of the (up to 16) partial maxima of column tx per thread, while the
        // tile's loads are in flight
        const int64_t j = j0 + tx;
        uint64_t mx = 0;
        if (j < n) {
            const uint64_t a = ty < ks ? part[(int64_t)ty * n + j] : 0ull;
            const uint64_t b = ty + 8 < ks ? part[(int64_t)(ty + 8) * n + j] : 0ull;
            mx = a > b ? a : b;
        }
        red[ty][tx] = mx;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) T[ty + 8 * r][tx] = v[r];
    __syncthreads();
    const int jj = tid >> 3, lsub = (tid & 7) * 8;
    const int64_t j = j0 + jj, lbase = l0 + lsub;
    const int64_t np = (n + kBN - 1) / kBN * kBN;
    if (lbase < kp && j < np) {
        int e = GB_BAD_LINE_DEV;
        if (j < n) {
            uint64_t mx = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) mx = red[r][jj] > mx ? red[r][jj] : mx;
            const bool bad = (mx >> 63) != 0;
            e = bad ? GB_BAD_LINE_DEV : frexp_exp_bits(mx);
            if (blockIdx.y == 0 && (tid & 7) == 0) {
                exps[j] = e;
                if (bad && status) atomicOr(status, kStatusNonfinite);
            }
        }
        uint32_t w[S][4];
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0;
        if (e != GB_BAD_LINE_DEV) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (lbase + u < k) digits_bf16<S>(T[lsub + u][jj], e, u, w);
        }
        const int64_t nks = kp / kKStep;
#pragma unroll
        for (int t = 0; t < S; ++t)
            *reinterpret_cast<uint4*>(digits + tiled_offset16(j, lbase, t, nks, kBN, S)) =
                make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
}

// ---- e3 + e4: slice-pair products in TMEM, exact recombination ---------------------
//
// Persistent CTAs, one per SM, 576 threads, over the 128 x 32 output tiles:
//   warp 0 lane 0 : producer, two contiguous bulk copies per stage (KB K steps of
//                   all s digit planes of A, then of B) and the tile arguments;
//   warp 1        : allocates the 512 TMEM columns; lane 0 issues the MMAs: per K
//                   step and A slice p one kind::f16 MMA (M = 128, K = 16,
//                   N = 32 (s+1-p)) over the consecutive B slices q = 1 .. s+1-p
//                   into the consecutive levels p-1 .. s-1; a unit's first MMA
//                   (p = 1, all levels) starts the set from zero;
//   warps 2 - 17  : epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                   columns 8 c .. 8 c + 7, c = (w - 2) / 4, of every level.
// Level sets alternate between TMEM columns 0 and 32 s by unit; the MMA issuer
// waits for the epilogue to have read a set (tmem_empty) before its next unit
// starts there.  Every wait is bounded (4 s of wall time, then the timeout bit,
// no output for the CTA's remaining tiles, TMEM still freed).
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s
constexpr int kSmemLimit = 227 * 1024;
constexpr int kArgSlots = 4;
constexpr int kMaxStages = 8;
constexpr int kStageKSteps = 2;  // K steps (of 16) per pipeline stage

// K steps of one exact accumulation unit: a level accumulator collects up to s
// pair products (|d_p d_q| <= 2^14) per K index and is exact while K s 2^14 <= 2^24.
__host__ __device__ constexpr int unit_ksteps(int S) { return (1024 / S) / kKStep; }

struct SmemTail16 {
    uint64_t bars[2 * kMaxStages + 5];  // full, empty per stage; tmem_full[2], tmem_empty[2], drain
    uint64_t args_full[kArgSlots];
    uint64_t args_empty[kArgSlots];
    TileArgs args[kArgSlots];
    uint32_t tmem_holder;
    int abort;
};

// The MMAs of one K step of all slice pairs into the level set at TMEM `acc`.
template <int S>
__device__ __forceinline__ void issue_kstep16(uint64_t adesc, uint64_t bdesc, uint32_t acc,
                                              bool first) {
#pragma unroll
    for (int p = 1; p <= S; ++p) {
        const uint64_t ad = adesc + (uint64_t)(((p - 1) * kBM * kBKBytes) >> 4);
        ptx::mma_bf16(acc + (uint32_t)((p - 1) * kBN), ad, bdesc,
                      ptx::idesc_bf16_f32(kBM, kBN * (S + 1 - p)), (first && p == 1) ? 0u : 1u);
    }
}

// acc[j] += sum_L x_L 2^(8 (L0 + NL - 1 - L)) over the levels L0 .. L0+NL-1 of the
// set at lane_addr, for this thread's columns 8 cg + j: each x_L an exact integer
// (|x| <= 2^24, converted by the FP32 -> int32 instruction), the Horner sum below
// 2^49 for NL <= 4.
template <int L0, int NL>
__device__ __forceinline__ void add_level_run(uint32_t lane_addr, int cg, int64_t (&acc)[8]) {
    uint32_t v[NL][8];
#pragma unroll
    for (int L = 0; L < NL; ++L)
        ptx::tmem_ld_32x32b_x8(lane_addr + (uint32_t)((L0 + L) * kBN + 8 * cg), v[L]);
    ptx::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int64_t h = __float2int_rn(__uint_as_float(v[0][j]));
#pragma unroll
        for (int L = 1; L < NL; ++L) h = h * 256 + __float2int_rn(__uint_as_float(v[L][j]));
        acc[j] += h;
    }
}

// One unit's levels into the thread's running sums, T = HI 2^48 + MID 2^24 + LO.
// S <= 7: MID collects levels 0 .. S-4 (weights 2^(8 (S-4-L))), LO the last three
// (weights 2^(8 (S-1-L))); per unit |MID| < 2^48.01 and |LO| < 2^40.01, and
// K <= 2^22 (at most 29128 units at S = 7) keeps the sums within int64.
// S = 8 (units of 128 K indices, up to 32768): HI takes levels 0, 1, MID 2 .. 4,
// LO 5 .. 7, each below 2^40.01 per unit.
template <int S>
__device__ __forceinline__ void add_unit(uint32_t lane_addr, int cg, int64_t (&HI)[8],
                                         int64_t (&MID)[8], int64_t (&LO)[8]) {
    if constexpr (S == 8) {
        add_level_run<0, 2>(lane_addr, cg, HI);
        add_level_run<2, 3>(lane_addr, cg, MID);
        add_level_run<5, 3>(lane_addr, cg, LO);
    } else {
        constexpr int NH = S > 3 ? S - 3 : 0;
        if constexpr (NH > 0) add_level_run<0, NH>(lane_addr, cg, MID);
        add_level_run<NH, S - NH>(lane_addr, cg, LO);
    }
}

template <int S, int KB, class Walk>
__device__ __forceinline__ void bf16_products_persistent(const Walk& walk, uint8_t* smem,
                                                         int stages, uint32_t slot_bytes,
                                                         unsigned* status) {
    constexpr int kCS = unit_ksteps(S) / KB;  // pipeline stages per exact unit
    static_assert(kCS >= 1, "one stage stays within an exact unit");
    static_assert(2 * S * kBN <= (int)kTmemCols, "two level sets in TMEM");
    constexpr uint32_t set_cols = (uint32_t)S * kBN;
    SmemTail16* tail = reinterpret_cast<SmemTail16*>(smem + (size_t)stages * slot_bytes);
    uint64_t* full = tail->bars;
    uint64_t* empty = tail->bars + stages;
    uint64_t* tmem_full = tail->bars + 2 * stages;       // one per level set
    uint64_t* tmem_empty = tail->bars + 2 * stages + 2;  // one per level set
    uint64_t* drain = tail->bars + 2 * stages + 4;
    volatile int* abort = &tail->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&tmem_full[b], 1);
            ptx::mbar_init(&tmem_empty[b], kEpiWarps);
        }
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
    constexpr uint32_t a_bytes = (uint32_t)S * kBM * kBKBytes;  // one K step of A's slices
    constexpr uint32_t b_bytes = (uint32_t)S * kBN * kBKBytes;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        int st = 0;
        uint32_t ph = 0;
        Walk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !*abort; w.next(), ++ti) {
            const TileArgs a = w.args();
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_empty[as], ((ti / kArgSlots) & 1u) ^ 1u, abort,
                                        status, kStatusTimeout, kWaitTimeoutNs))
                break;
            tail->args[as] = a;
            ptx::mbar_arrive(&tail->args_full[as]);
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
        int st = 0;
        uint32_t ph = 0;
        uint32_t unit = 0;  // units issued by this CTA so far: set unit % 2
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
            int in_unit = 0;
            uint32_t acc = tmem_base;
            for (int j = 0; j < nst; ++j) {
                const bool unit_start = in_unit == 0;
                if (unit_start) {
                    const uint32_t b = unit & 1u;
                    if (unit >= 2) {
                        // the epilogue has read this set's previous unit
                        if (!ptx::mbar_wait_bounded(&tmem_empty[b], ((unit >> 1) - 1) & 1u, abort,
                                                    status, kStatusTimeout, kWaitTimeoutNs)) {
                            stop = true;
                            break;
                        }
                        ptx::tc_fence_after();
                    }
                    acc = tmem_base + b * set_cols;
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
                        issue_kstep16<S>(adesc + (uint64_t)((kk * a_bytes) >> 4),
                                         bdesc + (uint64_t)((kk * b_bytes) >> 4), acc,
                                         unit_start && kk == 0);
                }
                ptx::mma_commit(&empty[st]);
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
                if (++in_unit == kCS || j + 1 == nst) {
                    ptx::mma_commit(&tmem_full[unit & 1u]);
                    ++unit;
                    in_unit = 0;
                }
            }
        }
    } else if (warp >= 2) {
        // ---- epilogue ----
        const int quarter = warp & 3;
        const int cgroup = (warp - 2) >> 2;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
        uint32_t unit = 0;
        bool stop = false;
        Walk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !stop; w.next(), ++ti) {
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_full[as], (ti / kArgSlots) & 1u, abort, status,
                                        kStatusTimeout, kWaitTimeoutNs))
                break;
            const TileArgs& a = tail->args[as];
            const int nunits = ((a.nkb + KB - 1) / KB + kCS - 1) / kCS;
            // a warp whose rows or columns all lie in the tile's padding only hands
            // the level sets back
            const bool live = a.row0 + quarter * 32 < a.m && a.col0 + 8 * cgroup < a.n;
            const int64_t row = a.row0 + quarter * 32 + lane;
            const bool row_ok = live && row < a.m;
            if (row_ok) {
                ptx::prefetch_l1(a.eA + row);
                if (lane == 0) ptx::prefetch_l1(a.fB + a.col0 + 8 * cgroup);
            }
            int64_t HI[8], MID[8], LO[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) HI[j] = MID[j] = LO[j] = 0;
            for (int c = 0; c < nunits; ++c, ++unit) {
                const uint32_t b = unit & 1u;
                const bool ok = ptx::mbar_wait_bounded(&tmem_full[b], (unit >> 1) & 1u, abort,
                                                       status, kStatusTimeout, kWaitTimeoutNs);
                ptx::tc_fence_after();
                if (!ok || *abort) {
                    stop = true;
                    break;
                }
                if (live) add_unit<S>(lane_addr + b * set_cols, cgroup, HI, MID, LO);
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tmem_empty[b]);
            }
            if (stop) break;
            if (row_ok) {
                I128 T[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    T[j] = I128{0, 0};
                    if (S == 8) i128_add_shl(T[j], HI[j], 48);
                    i128_add_shl(T[j], MID[j], 24);
                    i128_add_shl(T[j], LO[j], 0);
                }
                const int64_t n = a.n, col0 = a.col0;
                const double alpha = a.alpha, beta = a.beta;
                double* crow = a.C + row * a.ldc;
                const int32_t ei = a.eA[row];
                const int Ebase = -14 - kB * (S - 1);
                const long long ab = __double_as_longlong(alpha), bb = __double_as_longlong(beta);
                const bool beta0 = (bb & 0x7FFFFFFFFFFFFFFFll) == 0;
                const bool plain = ab == 0x3FF0000000000000ll && beta0;
                // one output at a time: the unit sums HI / MID / LO hold the registers
                store_part<S, 0, 8, 8, 1>(T, ei, Ebase, a.fB, col0, n, cgroup, plain, beta0, alpha,
                                          beta, crow, 1);
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tail->args_empty[as]);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        if (lane == 0 && *abort) {
            // no MMA may still write the accumulators when they are freed
            volatile int dummy = 0;
            ptx::mma_commit(drain);
            ptx::mbar_wait_bounded(drain, 0, &dummy, nullptr, 0, kWaitTimeoutNs);
        }
        __syncwarp();
        ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    bf16_products_kernel(const uint8_t* __restrict__ ad, const uint8_t* __restrict__ bd,
                         int64_t m, int64_t n, int nks, double alpha, double beta,
                         double* __restrict__ C, int64_t ldc, const int32_t* __restrict__ eA,
                         const int32_t* __restrict__ fB, int tiles_m, int tiles_n, int stages,
                         uint32_t slot_bytes, unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    const RasterWalk<kBN> w{ad, bd, m, n, ldc, nks, tiles_m, tiles_n, S, alpha, beta, C, eA, fB, 0};
    bf16_products_persistent<S, kStageKSteps>(w, smem, stages, slot_bytes, status);
}

template <int S>
cudaError_t launch_bf16_products_s(const Launch& L, int64_t m, int64_t n, int64_t kp,
                                   double alpha, double beta, double* C, int64_t ldc,
                                   const uint8_t* ad, const uint8_t* bd, const int32_t* ea,
                                   const int32_t* fb) {
    // slots on 1024-byte boundaries (the 32-byte swizzle wants 256-byte aligned tiles)
    const uint32_t slot = ((uint32_t)kStageKSteps * S * (kBM + kBN) * kBKBytes + 1023u) & ~1023u;
    const int fixed = 1024 + (int)sizeof(SmemTail16) + 64;
    int stages = (kSmemLimit - fixed) / (int)slot;
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t smem = (size_t)stages * slot + fixed;
    const int tiles_m = (int)((m + kBM - 1) / kBM), tiles_n = (int)((n + kBN - 1) / kBN);
    const int64_t tiles = (int64_t)tiles_m * tiles_n;
    const int grid = (int)(tiles < L.sm_count ? tiles : L.sm_count);
    cudaError_t e = cudaFuncSetAttribute(bf16_products_kernel<S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    bf16_products_kernel<S><<<grid, kThreads, smem, L.stream>>>(
        ad, bd, m, n, (int)(kp / kKStep), alpha, beta, C, ldc, ea, fb, tiles_m, tiles_n, stages,
        slot, L.status);
    return cudaGetLastError();
}

}  // namespace

#define GB_SWITCH_S8(s, CALL)                                                          \
    switch (s) {                                                                       \
        case 1: CALL(1); break;  case 2: CALL(2); break;  case 3: CALL(3); break;      \
        case 4: CALL(4); break;  case 5: CALL(5); break;  case 6: CALL(6); break;      \
        case 7: CALL(7); break;  case 8: CALL(8); break;                               \
        default: return cudaErrorInvalidValue;                                         \
    }

cudaError_t launch_bf16_split_rows(const Launch& L, int s, int64_t m, int64_t k, const double* A,
                                   int64_t lda, uint8_t* digits, int64_t kp, int32_t* exps) {
    if (m == 0) return cudaSuccess;
    int64_t blocks = (m + kEmuBM - 1) / kEmuBM * kEmuBM;
    const int64_t cap = (int64_t)L.sm_count * 16;
    if (blocks > cap) blocks = cap;
#define GB_LAUNCH(SS)                                                                        \
    bf16_split_rows_kernel<SS><<<(unsigned)blocks, 128, 0, L.stream>>>(m, k, A, lda, digits, \
                                                                       kp, exps, L.status)
    GB_SWITCH_S8(s, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_bf16_split_cols(const Launch& L, int s, int64_t n, int64_t k, const double* B,
                                   int64_t ldb, uint8_t* digits, int64_t kp, int32_t* exps,
                                   uint64_t* part) {
    if (n == 0) return cudaSuccess;
    int ks = 1;
    cudaError_t err = launch_colmax_part(L, n, k, B, ldb, part, &ks);
    if (err != cudaSuccess) return err;
    const int64_t np = (n + kBN - 1) / kBN * kBN;
    const dim3 grid((unsigned)((np + 31) / 32), (unsigned)((kp + 63) / 64));
#define GB_LAUNCH(SS)                                                                      \
    bf16_split_cols_kernel<SS><<<grid, 256, 0, L.stream>>>(n, k, B, ldb, digits, kp, exps, \
                                                           part, ks, L.status)
    GB_SWITCH_S8(s, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_bf16_products(const Launch& L, int s, int64_t m, int64_t n, double alpha,
                                 double beta, double* C, int64_t ldc, const uint8_t* a_digits,
                                 const uint8_t* b_digits, int64_t kp, const int32_t* a_exp,
                                 const int32_t* b_exp) {
    if (m == 0 || n == 0) return cudaSuccess;
#define GB_LAUNCH(SS)                                                                      \
    return launch_bf16_products_s<SS>(L, m, n, kp, alpha, beta, C, ldc, a_digits, b_digits, \
                                      a_exp, b_exp)
    GB_SWITCH_S8(s, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace gb
