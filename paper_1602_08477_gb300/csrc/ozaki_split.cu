// Emulated FP64 GEMM, steps e1 + e2: exponent extraction and E4M3 digit slicing.
//
// For a line (row of A, column of B) with max |value| = mu, e = frexp exponent of
// mu (mu < 2^e).  Each value a = 2^e (sum_t d_t 2^-(4 + 5(t-1)) + remainder) with
// signed digits d_t in [-16, 16] taken by round-to-nearest-even:
//   d_1 = rint(a 2^(4-e)),  r = a 2^(4-e) - d_1,  d_t = rint(32 r),  r = 32 r - d_t.
//
// GB300 executes FP64 at a small fraction of its integer rate, so every step here
// is integer arithmetic on the IEEE-754 bit pattern: a = M 2^E2 with an integer
// significand M, and "r scaled by 2^-sh" is kept as the exact integer R with an
// explicit shift sh.  Rounding R / 2^sh to nearest-even with integer shifts gives
// the same digits as the FP64 recurrence, which is exact at every step.
//
// Output layout: one E4M3 byte per digit, pre-tiled for the tensor-core
// products (tiles of R lines x 32 bytes, R = 128 for A and 32 for B, in the
// 32-byte swizzle; see tiled_offset), zero for l >= k and for padding lines;
//   exps[line] = e, or GB_BAD_LINE when the line holds a NaN or Inf (its digits
//   are all zero and the products mark its outputs NaN).
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "emu_common.cuh"
#include "internal.h"

namespace gb {
namespace {

constexpr int kB1 = 4;   // bits of the first digit
constexpr int kB = 5;    // bits of every further digit

// E4M3 encoding (sign bit 7, exponent bias 7, 3 mantissa bits) of an integer
// d with |d| <= 16: magnitudes 0..7 from a byte table (prmt), 8..16 are
// exponent 10 or 11 with mantissa a - 8 or (a - 16) / 2, i.e. code 0x48 + a.
__device__ __forceinline__ uint32_t e4m3_of_int(int d) {
    const uint32_t a = (uint32_t)(d < 0 ? -d : d);
    // codes of 0..7: 00 38 40 44 | 48 4A 4C 4E
    const uint32_t lo = __byte_perm(0x44403800u, 0x4E4C4A48u, a & 7u) & 0xFFu;
    const uint32_t code = a >= 8 ? 0x48u + a : lo;
    return (d < 0 ? 0x80u : 0u) | code;
}

// E4M3 byte of the digit d_t that a 7-bit window w = bits 5(S-t) .. 5(S-t)+6 of the
// fixed-point image determines under rounding half up (see digits_of):
// Q_t mod 64 = bits 1..6 of w + 1, and Q_(t-1) is odd iff bits 5, 6 of w are 01 or
// 10.  Each split kernel fills the table first (fill_e4m3_table); the lookup runs
// on the load/store pipe, which these integer-ALU-bound kernels leave idle.
__shared__ uint8_t s_window[128];

__device__ __forceinline__ void fill_e4m3_table() {
    const int x = threadIdx.x;
    if (x < 128) {
        const int qt = ((x + 1) >> 1) & 63;
        const int qp_odd = (((x >> 5) + 1) >> 1) & 1;
        const int dm = (qt - 32 * qp_odd) & 63;
        const int d = dm >= 32 ? dm - 64 : dm;
        s_window[x] = (uint8_t)(d >= -16 && d <= 16 ? e4m3_of_int(d) : 0u);
    }
    __syncthreads();
}

// Fixed-point image of an element for S digits: int64 holds it for S <= 11,
// a 128-bit integer above (|F| < 2^(5 S)).
template <int S>
struct FixedOf {
    using type = typename std::conditional<(S <= 11), int64_t, __int128>::type;
};

// The S digits of one finite double x relative to line exponent e, packed as
// E4M3 bytes into out[t] (byte `lane` of the 8-byte word of digit plane t, as
// its two 32-bit halves out[t][0] (bytes 0-3) and out[t][1] (bytes 4-7)).
//
// With x = X 2^E2 (X the signed integer significand) and sh_t = e - 4 - E2 -
// 5 (t - 1), the recurrence above satisfies  r_t 2^(...) = X - Q_t 2^(sh_t)  with
// Q_t = RNE(X / 2^(sh_t)) (round to nearest, ties to even): subtracting the
// integer multiple 32 Q_(t-1) commutes with RNE.  Hence every digit is
// d_t = Q_t - 32 Q_(t-1), computed independently of the others.
//
// F = X 2^k (k chosen per element) puts the unit of digit t at the fixed bit
// 1 + 5 (S - t), so each Q_t comes from a constant shift: W = floor(F / 2^(5(S-t)))
// = 2 Q0 + h, Q_t = (W + 1 - tie) / 2, where the tie (exactly half, Q0 even) is:
// the lowest set bit of F is bit 5 (S - t) (read off the trailing-zero count of
// X, which also covers the bits a right shift drops for k < 0) and bit 1 of W is
// clear.  Only d_t mod 64 is needed (it indexes the E4M3 table), i.e. Q_t mod 64
// and Q_(t-1) mod 2, and with rounding half up (W + 1) / 2 these depend on the
// seven bits 5(S-t) .. 5(S-t)+6 of F alone: one window lookup per digit.  A tie
// can only sit at the one digit t* with 5(S - t*) = tzF, and round-half-up differs
// from ties-to-even there only when Q0 is even; using F - 1 instead of F then
// gives the even rounding at t* and changes no other digit (F - 1 stays above
// every lower rounding point by less than a half unit, and the higher windows
// see no borrow), so the whole element is one subtraction plus S lookups.
// Byte `pos` (0..3) of x replaced by the low byte of y (one byte permute).
__device__ __forceinline__ uint32_t insert_byte(uint32_t x, uint32_t y, int pos) {
    return __byte_perm(x, y, pos == 0 ? 0x3214u : pos == 1 ? 0x3240u : pos == 2 ? 0x3410u : 0x4210u);
}

template <int S>
__device__ __forceinline__ void digits_of(uint64_t bits, int e, int lane, uint32_t (&out)[S][2]) {
    using Fixed = typename FixedOf<S>::type;
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
    const int k = 1 - (e - kB1 - E2) + kB * (S - 1);
    const int tzF = (__ffsll((long long)M) - 1) + k;
    Fixed F;
    if (k >= 0) F = (Fixed)X << k;  // exact: |F| < 2^(5 S)
    else F = (Fixed)(X >> (-k < 63 ? -k : 63));
    // an exact tie at a digit's rounding point with an even quotient rounds down
    const bool tie_down = tzF >= 0 && tzF <= kB * (S - 1) && tzF % kB == 0 &&
                          (((uint32_t)(F >> (tzF + 1))) & 1u) == 0u;
    F -= tie_down ? 1 : 0;
#pragma unroll
    for (int t = 1; t <= S; ++t) {
        const int sh = kB * (S - t);
        const uint32_t w = (uint32_t)(F >> sh) & 127u;
        // lane is a compile-time constant in the unrolled callers: one byte
        // permute into the right half of the digit plane's 8-byte word
        out[t - 1][lane >> 2] = insert_byte(out[t - 1][lane >> 2], s_window[w], lane & 3);
    }
}

// Byte offset of digit t of line x at K index l0 (l0 % 8 == 0; the 8 bytes
// l0 .. l0+7 are contiguous) in the tiled layout with R-line tiles.
__device__ __forceinline__ int64_t tiled_offset(int64_t x, int64_t l0, int t, int s, int64_t nkb,
                                                int R) {
    const int64_t tile = x / R;
    const int r = (int)(x - tile * R);
    const int64_t kb = l0 >> 5;
    const int c = (int)(l0 & 31);
    const int chunk = (c >> 4) ^ ((r >> 2) & 1);
    return ((tile * nkb + kb) * s + t) * (int64_t)(R * 32) + r * 32 + (chunk << 4) + (c & 15);
}

// Row i of A: pass 1 max |a| and finiteness, pass 2 digits (all threads call it).
// Rows m <= i < (tile padding) get zero digits.
template <int S>
__device__ __forceinline__ void split_one_row(int64_t i, int64_t m, int64_t k,
                                              const double* __restrict__ A, int64_t lda, int s,
                                              uint8_t* __restrict__ digits, int64_t kp,
                                              int32_t* __restrict__ exps, unsigned* status,
                                              uint64_t* red, int* bad_sh) {
    const int tid = threadIdx.x;
    const int64_t nkb = kp >> 5;
    if (i >= m) {
        for (int64_t l0 = (int64_t)tid * 8; l0 < kp; l0 += (int64_t)blockDim.x * 8)
            for (int t = 0; t < s; ++t)
                *reinterpret_cast<uint64_t*>(digits + tiled_offset(i, l0, t, s, nkb, kEmuBM)) = 0;
        return;
    }
    const uint64_t* row = reinterpret_cast<const uint64_t*>(A + i * lda);
    uint64_t mx = 0;
    int bad = 0;
    // the same 8 consecutive elements per thread as the digit pass (L1 reuse),
    // eight independent loads in flight per thread
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
    // pass 2: 8 consecutive elements per thread -> one 8-byte word per plane
    for (int64_t l0 = (int64_t)tid * 8; l0 < kp; l0 += (int64_t)blockDim.x * 8) {
        uint32_t w[S][2];
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][0] = w[t][1] = 0;
        if (!is_bad) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t l = l0 + u;
                if (l < k) digits_of<S>(row[l], e, u, w);
            }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
            if (t >= s) break;
            *reinterpret_cast<uint2*>(digits + tiled_offset(i, l0, t, s, nkb, kEmuBM)) =
                make_uint2(w[t][0], w[t][1]);
        }
    }
    __syncthreads();
}

// Column block jb (32 columns) of B: max |b| over all rows, per column, by R
// warps (R row phases; blockDim.x = 32 R).
template <int R>
__device__ __forceinline__ void colmax_block(int64_t jb, int64_t n, int64_t k,
                                             const double* __restrict__ B, int64_t ldb,
                                             int32_t* __restrict__ exps, unsigned* status,
                                             uint64_t (*mx_sh)[32], int (*bad_sh)[32]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j = jb * 32 + tx;
    uint64_t mx = 0;
    int bad = 0;
    if (j < n) {
        const uint64_t* col = reinterpret_cast<const uint64_t*>(B) + j;
#pragma unroll 4
        for (int64_t l = ty; l < k; l += R) {
            const uint64_t a = col[l * ldb] & 0x7FFFFFFFFFFFFFFFull;
            if (a >= 0x7FF0000000000000ull) bad = 1;
            else if (a > mx) mx = a;
        }
    }
    mx_sh[ty][tx] = mx;
    bad_sh[ty][tx] = bad;
    __syncthreads();
    if (ty == 0 && j < n) {
        for (int r = 1; r < R; ++r) {
            mx = mx_sh[r][tx] > mx ? mx_sh[r][tx] : mx;
            bad |= bad_sh[r][tx];
        }
        exps[j] = bad ? GB_BAD_LINE_DEV : frexp_exp_bits(mx);
        if (bad && status) atomicOr(status, kStatusNonfinite);
    }
    __syncthreads();
}

// Transposing digit pass for B over the tile of 64 rows (l) x 32 columns (j)
// at (lb, jb), into B digit tiles of R lines; columns n <= j < (n padded to whole
// tiles) get zero digits, columns beyond are not written.  `pre()` runs between
// the tile's loads and the barrier after them (its own loads overlap theirs);
// `ecol(jj, j)` gives the exponent of column j = 32 jb + jj after the barrier.
template <int S, class Pre, class ECol>
__device__ __forceinline__ void split_cols_tile(int64_t jb, int64_t lb, int64_t n, int64_t k,
                                                const double* __restrict__ B, int64_t ldb, int s,
                                                uint8_t* __restrict__ digits, int64_t kp,
                                                uint64_t (*T)[33], int R, Pre pre, ECol ecol) {
    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int64_t j0 = jb * 32, l0 = lb * 64;
    const uint64_t* Bb = reinterpret_cast<const uint64_t*>(B);
    uint64_t v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t l = l0 + ty + 8 * r, j = j0 + tx;
        v[r] = (l < k && j < n) ? Bb[l * ldb + j] : 0ull;
    }
    pre();
#pragma unroll
    for (int r = 0; r < 8; ++r) T[ty + 8 * r][tx] = v[r];
    __syncthreads();
    const int jj = tid >> 3, lsub = (tid & 7) * 8;
    const int64_t j = j0 + jj, lbase = l0 + lsub;
    const int64_t np = (n + R - 1) / R * R;
    if (lbase < kp && j < np) {
        const int e = ecol(jj, j);
        uint32_t w[S][2];
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][0] = w[t][1] = 0;
        if (e != GB_BAD_LINE_DEV) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (lbase + u < k) digits_of<S>(T[lsub + u][jj], e, u, w);
            }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
            if (t >= s) break;
            *reinterpret_cast<uint2*>(digits + tiled_offset(j, lbase, t, s, kp >> 5, R)) =
                make_uint2(w[t][0], w[t][1]);
        }
    }
    __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(128) split_rows_kernel(int64_t m, int64_t k,
                                                         const double* __restrict__ A,
                                                         int64_t lda,
                                                         uint8_t* __restrict__ digits,
                                                         int64_t kp, int32_t* __restrict__ exps,
                                                         unsigned* status) {
    fill_e4m3_table();
    __shared__ uint64_t red[4];
    __shared__ int bad_sh;
    const int64_t mp = (m + kEmuBM - 1) / kEmuBM * kEmuBM;
    for (int64_t i = blockIdx.x; i < mp; i += gridDim.x)
        split_one_row<S>(i, m, k, A, lda, S, digits, kp, exps, status, red, &bad_sh);
}

// One GEMM, first half of e1 for B: the column maxima over a K range.  CTA (x, y)
// takes columns 32 x .. 32 x + 31 and rows y rows_per .. (y + 1) rows_per - 1 by 8
// row phases; part[y n + j] = the largest absolute bit pattern in the range, or
// bit 63 alone when it holds a NaN or Inf (larger than every finite pattern, so the
// maximum over the ranges keeps it).  Many short strips keep every SM loading: one
// CTA per column strip left a narrow B bound by the latency of a strip of all rows.
__global__ void __launch_bounds__(256) colmax_part_kernel(int64_t n, int64_t k,
                                                          const double* __restrict__ B,
                                                          int64_t ldb, int64_t rows_per,
                                                          uint64_t* __restrict__ part) {
    __shared__ uint64_t mx_sh[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + tx;
    const int64_t l0 = (int64_t)blockIdx.y * rows_per;
    const int64_t l1 = l0 + rows_per < k ? l0 + rows_per : k;
    uint64_t mx = 0;
    if (j < n) {
        const uint64_t* col = reinterpret_cast<const uint64_t*>(B) + j;
#pragma unroll 8
        for (int64_t l = l0 + ty; l < l1; l += 8) {
            const uint64_t a = col[l * ldb] & 0x7FFFFFFFFFFFFFFFull;
            const uint64_t t = a >= 0x7FF0000000000000ull ? (1ull << 63) : a;
            mx = t > mx ? t : mx;
        }
    }
    mx_sh[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && j < n) {
#pragma unroll
        for (int r = 1; r < 8; ++r) mx = mx_sh[r][tx] > mx ? mx_sh[r][tx] : mx;
        part[(int64_t)blockIdx.y * n + j] = mx;
    }
}

// One GEMM, second half of e1 and e2 for B: each CTA reduces the `ks` partial
// maxima of its 32 columns to their exponents (the CTAs of the first K tile also
// store them in exps and flag non-finite columns), then writes the digit tiles of
// its 64 rows x 32 columns.
template <int S>
__global__ void __launch_bounds__(256) split_cols_kernel(int64_t n, int64_t k,
                                                         const double* __restrict__ B,
                                                         int64_t ldb,
                                                         uint8_t* __restrict__ digits,
                                                         int64_t kp, int32_t* __restrict__ exps,
                                                         const uint64_t* __restrict__ part, int ks,
                                                         unsigned* status) {
    fill_e4m3_table();
    __shared__ uint64_t T[64][33];
    __shared__ uint64_t red[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    static_assert(kColmaxParts <= 16, "two partial maxima per thread of 8 row phases");
    // every thread loads two of the (up to 16) partial maxima of column tx while
    // the tile loads fly; the barrier after the tile's loads publishes red
    auto partial_maxima = [&]() {
        const int64_t j = (int64_t)blockIdx.x * 32 + tx;
        uint64_t mx = 0;
        if (j < n) {
            const uint64_t a = ty < ks ? part[(int64_t)ty * n + j] : 0ull;
            const uint64_t b = ty + 8 < ks ? part[(int64_t)(ty + 8) * n + j] : 0ull;
            mx = a > b ? a : b;
        }
        red[ty][tx] = mx;
    };
    // column exponent from the 8 row-phase maxima; the first K tile's CTAs store it
    auto column_exponent = [&](int jj, int64_t j) {
        if (j >= n) return (int)GB_BAD_LINE_DEV;
        uint64_t mx = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) mx = red[r][jj] > mx ? red[r][jj] : mx;
        const bool bad = (mx >> 63) != 0;
        const int e = bad ? GB_BAD_LINE_DEV : frexp_exp_bits(mx);
        if (blockIdx.y == 0 && (threadIdx.x & 7) == 0) {
            exps[j] = e;
            if (bad && status) atomicOr(status, kStatusNonfinite);
        }
        return e;
    };
    split_cols_tile<S>(blockIdx.x, blockIdx.y, n, k, B, ldb, S, digits, kp, T, emu_bn(S),
                       partial_maxima, column_exponent);
}

#define GB_SWITCH_S(s, CALL)                                                           \
    switch (s) {                                                                       \
        case 1: CALL(1); break;  case 2: CALL(2); break;  case 3: CALL(3); break;      \
        case 4: CALL(4); break;  case 5: CALL(5); break;  case 6: CALL(6); break;      \
        case 7: CALL(7); break;  case 8: CALL(8); break;  case 9: CALL(9); break;      \
        case 10: CALL(10); break; case 11: CALL(11); break; case 12: CALL(12); break;  \
        case 13: CALL(13); break; case 14: CALL(14); break; case 15: CALL(15); break;  \
        case 16: CALL(16); break; default: break;                                      \
    }

// ---- grouped: one launch per step over the problems of a table ---------------------
// Last table entry q in [lo, hi] with key[q] <= x (keys ascending).
__device__ __forceinline__ int find_prob(const int64_t* __restrict__ key, int lo, int hi,
                                         int64_t x) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One 128-row tile of A (rows row0 .. row0+127 of a problem, rows >= m are the
// tile padding) by a CTA of 256 threads.  Both passes use the same map: slot p of
// 512 (two per thread) takes row p / 4 and, in every K block of 32, elements
// 8 (p % 4) .. +7.  Pass 1: max |a| and finiteness of each slot's elements, then
// of the row over its 4 neighbouring lanes (all rows' loads in flight at once).
// Pass 2: the digits, so a warp writes 256 contiguous bytes per digit plane (8
// rows x 32 bytes of the tiled layout) and every lane has work even for short rows.
template <int S>
__device__ __forceinline__ void split_row_tile(int64_t row0, int64_t m, int64_t k,
                                               const double* __restrict__ A, int64_t lda,
                                               uint8_t* __restrict__ digits, int64_t kp,
                                               int32_t* __restrict__ exps, unsigned* status,
                                               int* e_sh, int R) {
    const int64_t nkb = kp >> 5;
    const int64_t mp = (m + R - 1) / R * R;  // rows with digits (R-line tiles)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int p = threadIdx.x + 256 * half;
        const int r = p >> 2;
        const int64_t i = row0 + r;
        uint64_t mx = 0;
        unsigned bad = 0;
        if (i < m) {
            const uint64_t* row = reinterpret_cast<const uint64_t*>(A + i * lda);
            for (int64_t l0 = (p & 3) * 8; l0 < k; l0 += 32) {
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
        }
        // the row's 4 slots are lanes 4q .. 4q+3 of this warp
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            const uint64_t w = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = w > mx ? w : mx;
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if ((p & 3) == 0) {
            if (i >= m) {
                e_sh[r] = GB_BAD_LINE_DEV;  // padding: zero digits
            } else {
                const int e = bad ? GB_BAD_LINE_DEV : frexp_exp_bits(mx);
                exps[i] = e;
                e_sh[r] = e;
                if (bad && status) atomicOr(status, kStatusNonfinite);
            }
        }
    }
    __syncthreads();
    for (int64_t kb = 0; kb < nkb; ++kb) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int p = threadIdx.x + 256 * half;
            const int r = p >> 2;
            const int64_t i = row0 + r, l0 = kb * 32 + (p & 3) * 8;
            if (i >= mp) continue;  // beyond the last R-line tile of this problem
            const int e = e_sh[r];
            uint32_t w[S][2];
#pragma unroll
            for (int t = 0; t < S; ++t) w[t][0] = w[t][1] = 0;
            if (e != GB_BAD_LINE_DEV) {
                const uint64_t* src = reinterpret_cast<const uint64_t*>(A + i * lda) + l0;
                uint64_t v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = l0 + u < k ? src[u] : 0ull;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (l0 + u < k) digits_of<S>(v[u], e, u, w);
            }
#pragma unroll
            for (int t = 0; t < S; ++t)
                *reinterpret_cast<uint2*>(digits + tiled_offset(i, l0, t, S, nkb, R)) =
                    make_uint2(w[t][0], w[t][1]);
        }
    }
    __syncthreads();
}

// Grouped kernels: one launch per step over the problems of one slice count S.
template <int S>
__global__ void __launch_bounds__(256) grouped_split_rows_kernel(const EmuProb* __restrict__ P,
                                                                 const int64_t* __restrict__ key,
                                                                 int q_begin, int q_end,
                                                                 int64_t row_begin,
                                                                 int64_t row_end,
                                                                 unsigned* status) {
    fill_e4m3_table();
    __shared__ int e_sh[kEmuBM];
    // rows are padded to 128 per problem, so a 128-row block is one problem's tile
    for (int64_t r0 = row_begin + (int64_t)blockIdx.x * kEmuBM; r0 < row_end;
         r0 += (int64_t)gridDim.x * kEmuBM) {
        const EmuProb& q = P[find_prob(key, q_begin, q_end - 1, r0)];
        split_row_tile<S>(r0 - q.first_row, q.m, q.k, q.A, q.lda, q.a_digits, q.kp, q.a_exp,
                          status, e_sh, q.ra);
    }
}

// Column maxima and digits of B in one pass per 32-column strip: a CTA takes one
// strip of a problem's padded columns (strips past the real columns get zero
// digits), finds the strip's column maxima over all K rows, then splits its
// 64-row tiles, which it re-reads while they are still in L2.
template <int S>
__global__ void __launch_bounds__(256) grouped_split_strips_kernel(const EmuProb* __restrict__ P,
                                                                   const int64_t* __restrict__ key,
                                                                   int q_begin, int q_end,
                                                                   int64_t cb_begin,
                                                                   int64_t cb_end,
                                                                   unsigned* status) {
    fill_e4m3_table();
    __shared__ uint64_t T[64][33];
    __shared__ uint64_t mx_sh[8][32];
    __shared__ int bad_sh[8][32];
    for (int64_t b = cb_begin + blockIdx.x; b < cb_end; b += gridDim.x) {
        const EmuProb& q = P[find_prob(key, q_begin, q_end - 1, b)];
        const int64_t jb = b - q.first_colblk;
        // the exponents of the strip's real columns, visible to the whole CTA after
        // colmax_block's closing barrier
        colmax_block<8>(jb, q.n, q.k, q.B, q.ldb, q.b_exp, status, mx_sh, bad_sh);
        const int32_t* b_exp = q.b_exp;
        const int64_t qn = q.n;
        const int64_t nlb = (q.kp + 63) / 64;
        for (int64_t lb = 0; lb < nlb; ++lb)
            split_cols_tile<S>(jb, lb, q.n, q.k, q.B, q.ldb, S, q.b_digits, q.kp, T, q.rb,
                               [] {}, [=](int, int64_t j) {
                                   return j < qn ? (int)b_exp[j] : (int)GB_BAD_LINE_DEV;
                               });
    }
}

}  // namespace

cudaError_t launch_split_rows(const Launch& L, int s, int64_t m, int64_t k, const double* A,
                              int64_t lda, uint8_t* digits, int64_t kp, int32_t* exps) {
    if (m == 0) return cudaSuccess;
    int64_t blocks = (m + kEmuBM - 1) / kEmuBM * kEmuBM;
    const int64_t cap = (int64_t)L.sm_count * 16;
    if (blocks > cap) blocks = cap;
#define GB_LAUNCH_ROWS(SS)                                                                   \
    split_rows_kernel<SS><<<(unsigned)blocks, 128, 0, L.stream>>>(m, k, A, lda, digits, kp, \
                                                                  exps, L.status)
    GB_SWITCH_S(s, GB_LAUNCH_ROWS)
#undef GB_LAUNCH_ROWS
    return cudaGetLastError();
}

cudaError_t launch_grouped_split(const Launch& L, const EmuProb* probs, const EmuKeys& keys,
                                 const EmuSRange& r, const SplitFork* fk) {
    if (r.q_end <= r.q_begin) return cudaSuccess;
    const int64_t cap = (int64_t)L.sm_count * 16;
    auto g = [&](int64_t x) { return (unsigned)(x < cap ? (x > 0 ? x : 1) : cap); };
    const unsigned g_rows = g((r.row_end - r.row_begin) / kEmuBM);
    // A's rows and B's columns are independent inputs of the products: with a
    // fork the split of A runs on the side stream, beside the launches for B
    cudaError_t err = cudaSuccess;
    cudaStream_t rows_stream = L.stream;
    if (fk) {
        err = cudaEventRecord(fk->fork, L.stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(fk->side, fk->fork, 0);
        if (err != cudaSuccess) return err;
        rows_stream = fk->side;
    }
#define GB_LAUNCH_GROWS(SS)                                                                   \
    grouped_split_rows_kernel<SS><<<g_rows, 256, 0, rows_stream>>>(                           \
        probs, keys.row, r.q_begin, r.q_end, r.row_begin, r.row_end, L.status)
    GB_SWITCH_S(r.s, GB_LAUNCH_GROWS)
#undef GB_LAUNCH_GROWS
    err = cudaGetLastError();
    if (err == cudaSuccess && fk) err = cudaEventRecord(fk->join, fk->side);
    if (err != cudaSuccess) return err;
#define GB_LAUNCH_GSTRIPS(SS)                                                                 \
    grouped_split_strips_kernel<SS><<<g(r.cb_end - r.cb_begin), 256, 0, L.stream>>>(          \
        probs, keys.colblk, r.q_begin, r.q_end, r.cb_begin, r.cb_end, L.status)
    GB_SWITCH_S(r.s, GB_LAUNCH_GSTRIPS)
#undef GB_LAUNCH_GSTRIPS
    err = cudaGetLastError();
    if (err == cudaSuccess && fk) err = cudaStreamWaitEvent(L.stream, fk->join, 0);
    return err;
}

cudaError_t launch_colmax_part(const Launch& L, int64_t n, int64_t k, const double* B,
                               int64_t ldb, uint64_t* part, int* ks_out) {
    // K ranges of the column maxima: about sixteen CTAs per SM over the column
    // strips (enough loads in flight to stream B), at least 64 rows each, at most
    // kColmaxParts
    const int64_t ncb = (n + 31) / 32;
    int64_t ks = (16 * (int64_t)L.sm_count + ncb - 1) / ncb;
    const int64_t kcap = (k + 63) / 64;
    if (ks > kcap) ks = kcap;
    if (ks > kColmaxParts) ks = kColmaxParts;
    if (ks < 1) ks = 1;
    *ks_out = (int)ks;
    const int64_t rows_per = (k + ks - 1) / ks;
    colmax_part_kernel<<<dim3((unsigned)ncb, (unsigned)ks), 256, 0, L.stream>>>(n, k, B, ldb,
                                                                              rows_per, part);
    return cudaGetLastError();
}

cudaError_t launch_split_cols(const Launch& L, int s, int64_t n, int64_t k, const double* B,
                              int64_t ldb, uint8_t* digits, int64_t kp, int32_t* exps,
                              uint64_t* part) {
    if (n == 0) return cudaSuccess;
    int ks = 1;
    cudaError_t err = launch_colmax_part(L, n, k, B, ldb, part, &ks);
    if (err != cudaSuccess) return err;
    const int64_t np = (n + emu_bn(s) - 1) / emu_bn(s) * emu_bn(s);  // B digit tile padding
    const dim3 grid((unsigned)((np + 31) / 32), (unsigned)((kp + 63) / 64));
#define GB_LAUNCH_COLS(SS)                                                                   \
    split_cols_kernel<SS><<<grid, 256, 0, L.stream>>>(n, k, B, ldb, digits, kp, exps, part, \
                                                      ks, L.status)
    GB_SWITCH_S(s, GB_LAUNCH_COLS)
#undef GB_LAUNCH_COLS
    return cudaGetLastError();
}

}  // namespace gb
