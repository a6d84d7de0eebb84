// Pieces of the emulated GEMM's kernels that do not depend on the digit format
// (E4M3 digits: ozaki_split.cu, ozaki_gemm.cu; BF16 digits: ozaki_bf16.cu): the
// line exponents of the split, the exact 128-bit recombination sum and its single
// rounding to FP64, the arguments of an output tile, the rasterised tile order of
// one GEMM and the stores to C.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"

#ifndef GB_BAD_LINE_DEV
#define GB_BAD_LINE_DEV 0x40000000
#endif

namespace gb {
namespace {

constexpr int kBM = kEmuBM;        // output tile rows: TMEM lanes, A digit tile rows
constexpr int kBKBytes = 32;       // bytes of K per row of a digit tile (one MMA's K)

// frexp exponent of a finite non-negative double given by its bits (0 -> 0).
__device__ __forceinline__ int frexp_exp_bits(uint64_t absbits) {
    if (absbits == 0) return 0;
    const int ef = (int)(absbits >> 52);
    if (ef != 0) return ef - 1022;
    const int p = 63 - __clzll((long long)absbits);  // subnormal: value = mant * 2^-1074
    return p - 1073;
}

struct I128 {
    int64_t hi;
    uint64_t lo;
};

// RN(T * 2^E) as an FP64 (T a signed 128-bit integer, E any int): the double
// nearest to the exact value, ties to even, with gradual underflow (subnormal
// results carry the unit 2^-1074) and overflow to +-Inf.  One rounding, done on
// the integer, so no FP64 multiplication (and no power of two outside the double
// range) is used.  Normal results (the usual case) take a branch-free path: |T|
// is shifted so that its leading one sits at bit 127, the significand is then
// bits 75..127, the round bit bit 74 and the sticky bits 0..73.  Subnormal
// results round |T| at bit q = -1074 - E instead (the general path).
__device__ __forceinline__ double i128_to_double_subnormal(uint64_t hi, uint64_t lo, int p, int E,
                                                        bool neg) {
    const int q = -1074 - E;  // > p - 52: the last place of the subnormal grid
    uint64_t M;               // |T| / 2^q rounded: the subnormal's bit pattern
    if (q <= 0) {
        M = lo << (-q);  // exact: q <= 0 here means p <= 52 and |T| < 2^53
    } else if (q > p + 1) {
        M = 0;           // below half of the last place
    } else if (q == p + 1) {
        // |T| in [2^p, 2^(p+1)): at least half of the last place; exactly half
        // (|T| = 2^p) ties to the even 0
        const bool is_pow2 = p >= 64 ? (lo == 0 && hi == (1ull << (p - 64)))
                                     : (hi == 0 && lo == (1ull << p));
        M = is_pow2 ? 0 : 1;
    } else {
        const int sh = q;  // 1 .. p <= 127
        uint64_t rem_hi, rem_lo, half_hi, half_lo;
        if (sh < 64) {
            M = (lo >> sh) | (hi << (64 - sh));
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
        if (gt || (eq && (M & 1))) M += 1;
    }
    // M <= 2^52: the subnormal's bit pattern (2^52 is the smallest normal's)
    return __longlong_as_double((long long)(M | (neg ? 0x8000000000000000ull : 0ull)));
}

// |T| as (hi, lo), its sign and the position p of its leading one (p = -1 for
// T = 0).
__device__ __forceinline__ void i128_magnitude(I128 x, uint64_t& hi, uint64_t& lo, bool& neg,
                                               int& p) {
    neg = x.hi < 0;
    hi = (uint64_t)x.hi;
    lo = x.lo;
    // two's complement negation of the 128-bit value when negative
    lo = neg ? ~lo + 1 : lo;
    hi = neg ? ~hi + (lo == 0 ? 1 : 0) : hi;
    p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
}

// The normal-range rounding of |T| 2^E (T != 0, p + E + 1023 >= 1), branch-free
// so that the outputs of a thread round as independent instruction streams.
__device__ __forceinline__ double i128_round_normal(uint64_t hi, uint64_t lo, int p, int E,
                                                    bool neg) {
    const int eb = p + E + 1023;  // biased exponent before a rounding carry
    // leading one to bit 127: by 64 first when the high word is empty
    const int c = (127 - p) & 127;            // 0 .. 127
    const uint64_t h1 = c >= 64 ? lo : hi;
    const uint64_t l1 = c >= 64 ? 0 : lo;
    const int c1 = c & 63;
    const uint64_t nh = c1 ? (h1 << c1) | (l1 >> (64 - c1)) : h1;
    const uint64_t nl = l1 << c1;
    uint64_t M = nh >> 11;                                  // 53 bits, leading one at 52
    const bool rb = (nh >> 10) & 1;                         // half of the last place
    const bool sticky = ((nh & 0x3FFull) | nl) != 0;        // anything below it
    M += (rb && (sticky || (M & 1))) ? 1 : 0;               // nearest, ties to even
    const bool carry = (M >> 53) != 0;                      // rounded up to 2^53
    M = carry ? M >> 1 : M;
    const int e = eb + (carry ? 1 : 0);
    const uint64_t bits = e >= 2047 ? 0x7FF0000000000000ull
                                    : (((uint64_t)e << 52) | (M & 0xFFFFFFFFFFFFFull));
    // sign by bit manipulation: GB300's FP64 pipe is slow even for negation
    return __longlong_as_double((long long)(bits | (neg ? 0x8000000000000000ull : 0ull)));
}

__device__ __forceinline__ double i128_to_double_scaled(I128 x, int E) {
    uint64_t hi, lo;
    bool neg;
    int p;
    i128_magnitude(x, hi, lo, neg, p);
    if ((hi | lo) == 0) return 0.0;
    if (p + E + 1023 < 1) return i128_to_double_subnormal(hi, lo, p, E, neg);
    return i128_round_normal(hi, lo, p, E, neg);
}

// x += v * 2^sh exactly (0 <= sh <= 127 - 63).
__device__ __forceinline__ void i128_add_shl(I128& x, int64_t v, int sh) {
    uint64_t lo, hi;
    if (sh == 0) {
        lo = (uint64_t)v;
        hi = v < 0 ? ~0ull : 0ull;
    } else if (sh < 64) {
        lo = (uint64_t)v << sh;
        hi = (uint64_t)(v >> (64 - sh));
    } else {
        lo = 0;
        hi = (uint64_t)v << (sh - 64);
    }
    const uint64_t nlo = x.lo + lo;
    x.hi += (int64_t)(hi + (nlo < x.lo ? 1 : 0));
    x.lo = nlo;
}

// Arguments of one output tile (row0, col0) of one problem.
struct TileArgs {
    const uint8_t* a_src;  // A digit tiles of this tile row, K block 0 (s * 4 KiB per block)
    const uint8_t* b_src;  // B digit tiles of this tile column, K block 0 (s * 1 KiB per block)
    int s, nkb;
    bool reverse;  // stream the K blocks last to first
    bool trans;    // the tile's rows are columns of C (C^T = B^T A^T): store transposed
    int64_t m, n, ldc, row0, col0;
    double alpha, beta;
    double* C;
    const int32_t* eA;  // row exponents (indexed by row)
    const int32_t* fB;  // column exponents (indexed by column)
};

// Columns of an epilogue warp: column group g (0 .. 3) of a BN-column level owns
// columns 8g .. 8g+7 and, for BN = 48, also 32 + 4g .. 32 + 4g + 3 (so every TMEM
// load starts on a multiple of its own width).  Column j (< BN / 4) of the group:
__host__ __device__ constexpr int epi_col(int g, int j) {
    return j < 8 ? 8 * g + j : 32 + 4 * g + (j - 8);
}

// Columns J0 .. J0+W-1 of this thread (see epi_col) of one output row, in groups
// of G: the group's column exponents loaded (L1 hits), its outputs RN(T 2^E)
// formed, alpha / beta applied, then its stores; `crow` is the row (stride
// `cstride` between columns).  G = 4 rounds four outputs as independent
// instruction streams; G = 1 where the registers for that are not free.  The
// sums of these columns are T[TJ .. TJ+W-1].
template <int S, int J0, int W, int N, int G = 4, int TJ = J0>
__device__ __forceinline__ void store_part(const I128 (&T)[N], int32_t ei, int Ebase,
                                           const int32_t* fB, int64_t col0, int64_t n, int cg,
                                           bool plain, bool beta0, double alpha, double beta,
                                           double* crow, int64_t cstride) {
    static_assert(W % G == 0, "whole groups of columns");
    const bool bad_row = ei == GB_BAD_LINE_DEV;
#pragma unroll
    for (int g0 = 0; g0 < W; g0 += G) {
        int32_t fj[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int64_t col = col0 + epi_col(cg, J0 + g0 + j);
            fj[j] = col < n ? fB[col] : 0;
        }
        // the group's outputs through the branch-free normal-range rounding
        // (independent instruction streams; T = 0 by a select), subnormal results
        // again in a second pass that is rarely taken
        double out[G];
        uint32_t special = 0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const bool bad = bad_row || fj[j] == GB_BAD_LINE_DEV;
            uint64_t hi, lo;
            bool neg;
            int p;
            i128_magnitude(T[TJ + g0 + j], hi, lo, neg, p);
            const int E = ei + fj[j] + Ebase;
            const bool zero = (hi | lo) == 0;
            const bool in_c = col0 + epi_col(cg, J0 + g0 + j) < n;
            special |= (in_c && !bad && !zero && p + E + 1023 < 1) ? (1u << j) : 0u;
            out[j] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : zero ? 0.0 : i128_round_normal(hi, lo, p, E, neg);
        }
        if (special) {
#pragma unroll
            for (int j = 0; j < G; ++j)
                if ((special >> j) & 1u)
                    out[j] = i128_to_double_scaled(T[TJ + g0 + j], ei + fj[j] + Ebase);
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const bool bad = bad_row || fj[j] == GB_BAD_LINE_DEV;
            const int64_t col = col0 + epi_col(cg, J0 + g0 + j);
            if (!plain && !bad && col < n) {
                double o = __dmul_rn(alpha, out[j]);
                if (!beta0) o = __dadd_rn(o, __dmul_rn(beta, crow[col * cstride]));
                out[j] = o;
            }
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int64_t col = col0 + epi_col(cg, J0 + g0 + j);
            if (col < n) crow[col * cstride] = out[j];
        }
    }
}

__device__ __forceinline__ uint8_t* aligned_smem(uint8_t* raw) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
}

// One GEMM: persistent CTAs over its tiles t = blockIdx.x, + gridDim.x, ... in the
// rasterised order (groups of 8 tile rows sweep the tile columns, so concurrent
// CTAs share A and B strips in L2).  Every other wave of tiles streams K from
// the end: the next wave keeps the same A strips, and the K blocks the previous
// wave read last are the ones still in L2.  The order of the K blocks does not
// change a bit of the result: the level sums are exact integers.
template <int BN>
struct RasterWalk {
    const uint8_t* ad;
    const uint8_t* bd;
    int64_t m, n, ldc;
    int nkb, tiles_m, tiles_n, s;
    double alpha, beta;
    double* C;
    const int32_t* eA;
    const int32_t* fB;
    int64_t t;
    __device__ void start() { t = blockIdx.x; }
    __device__ bool valid() const { return t < (int64_t)tiles_m * tiles_n; }
    __device__ void next() { t += gridDim.x; }
    __device__ TileArgs args() const {
        const int bid = (int)t;
        const int group_size = 8 * tiles_n;
        const bool reverse = ((t / gridDim.x) & 1) != 0;
        const int first_m = (bid / group_size) * 8;
        const int gm = min(tiles_m - first_m, 8);
        const int tm = first_m + (bid % group_size) % gm;
        const int tn = (bid % group_size) / gm;
        TileArgs a;
        a.a_src = ad + (size_t)tm * nkb * s * kBM * kBKBytes;
        a.b_src = bd + (size_t)tn * nkb * s * BN * kBKBytes;
        a.s = s;
        a.nkb = nkb;
        a.reverse = reverse;
        a.trans = false;
        a.m = m;
        a.n = n;
        a.ldc = ldc;
        a.row0 = (int64_t)tm * kBM;
        a.col0 = (int64_t)tn * BN;
        a.alpha = alpha;
        a.beta = beta;
        a.C = C;
        a.eA = eA;
        a.fB = fB;
        return a;
    }
};

}  // namespace
}  // namespace gb
