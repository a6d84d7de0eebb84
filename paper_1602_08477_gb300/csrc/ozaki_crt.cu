// Emulated FP64 GEMM by residue arithmetic: the operands are scaled to integers
// once and multiplied modulo N small pairwise-coprime moduli on the tcgen05
// tensor cores; the Chinese remainder theorem gives the exact integer product
// back, which is rounded once to FP64.
//
//   c1  e_i = frexp exponent of max_l |A[i,l]| (f_j for the columns of B);
//   c2  A'[i,l] = RNE(A[i,l] 2^(b - e_i)), B'[l,j] = RNE(B[l,j] 2^(b - f_j)), with
//       b the largest bit count such that K 2^(2b) <= M / 4 (M = m_1 ... m_N), so
//       every |(A'B')[i,j]| <= M / 4;
//   c3  symmetric residues R_t = A' mod m_t in [-(m_t - 1) / 2, (m_t - 1) / 2]
//       (every modulus an odd prime <= 509: |R| <= 254, exact in BF16);
//   c4  P_t = R^A_t R^B_t on the tensor cores: one kind::f16 MMA per 16 K per
//       output tile; each FP32 accumulator sums at most 256 K (256 * 254^2 <
//       2^24: every partial sum an exact integer) before the epilogue adds it
//       into an int32 and reduces it to the symmetric residue c_t;
//   c5  C' = sum_t c_t w_t - q M (w_t = (M / m_t) ((M / m_t)^-1 mod m_t), q the
//       nearest integer to sum_t c_t w_t / M), which is A'B' exactly;
//   c6  C = alpha RN(C' 2^(e_i + f_j - 2b)) + beta C.
//
// Compared with the digit-slice form (ozaki_gemm.cu), the tensor cores do N
// products of the whole K instead of s (s + 1) / 2 pair products: 13 BF16
// GEMMs (the work of 26 FP8 GEMMs) against 55 FP8 pair products at s = 10.
// Residues are stored pre-tiled, tile by tile: for each tile of R lines (128 rows
// of A, 256 columns of B), each modulus and each K step of 16 elements, an R x
// 32-byte K-major block in the 32-byte swizzle, the K steps of a (tile, modulus)
// one after another, so a pipeline stage is one contiguous bulk copy per operand,
// and the residues of a band of tiles are one contiguous range (a band of rows or
// a block of columns is computed like a GEMM of its own).
#include <cuda_runtime.h>
#include <cstdint>

#include "emu_common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace gb {
namespace {

// the moduli, largest first: odd primes below 513, pairwise coprime
constexpr int kModuli[kCrtMaxModuli] = {509, 503, 499, 491, 487, 479, 467,
                                        463, 461, 457, 449, 443, 439, 433};
constexpr int kTileLines = 128;  // lines of an A residue tile (rows of A) = output tile rows
constexpr int kTileLinesB = 256; // lines of a B residue tile (columns of B) = output tile columns
constexpr int kStep = 16;        // K elements of one kind::f16 MMA (32 bytes of BF16)
constexpr uint32_t kBlockBytes = kTileLines * 32;    // one A tile's K step
constexpr uint32_t kBlockBytesB = kTileLinesB * 32;  // one B tile's K step

// ---- c2 + c3: integers and residues -------------------------------------------------

// |RNE(x 2^(b - e))| of the finite double with bit pattern `bits` (e the frexp
// exponent of its line's maximum, so the result is at most 2^b <= 2^62), and the
// sign of x.
__device__ __forceinline__ uint64_t scaled_magnitude(uint64_t bits, int e, int b, bool& neg) {
    neg = (bits >> 63) != 0;
    const int ef = (int)((bits >> 52) & 0x7FF);
    uint64_t M = bits & 0xFFFFFFFFFFFFFull;
    int E2;
    if (ef == 0) {
        E2 = -1074;
    } else {
        M |= 1ull << 52;
        E2 = ef - 1075;
    }
    if (M == 0) return 0;
    const int k = E2 + b - e;
    if (k >= 0) return M << k;  // exact: M 2^k < 2^b
    const int sh = -k;
    if (sh >= 64) return 0;     // below half of the unit
    const uint64_t q = M >> sh;
    const uint64_t rem = M & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);  // nearest, ties to even
}

// x mod P for x < 2^32 (Barrett: the quotient estimate is low by at most one).
template <int P>
__device__ __forceinline__ uint32_t mod_u32(uint32_t x) {
    constexpr uint32_t magic = (uint32_t)((1ull << 32) / (uint64_t)P);
    const uint32_t q = __umulhi(x, magic);
    const uint32_t r = x - q * (uint32_t)P;
    return r >= (uint32_t)P ? r - (uint32_t)P : r;
}

// BF16 code of the symmetric residue of +-u modulo kModuli[T], u < 2^62 given as
// three 21-bit limbs (u = u2 2^42 + u1 2^21 + u0): the limbs weighted by 2^21 and
// 2^42 mod P stay below 2^31, one Barrett reduction.
template <int T>
__device__ __forceinline__ uint32_t residue_code(uint32_t u0, uint32_t u1, uint32_t u2, bool neg) {
    constexpr int P = kModuli[T];
    constexpr uint32_t c21 = (uint32_t)((1ull << 21) % (uint64_t)P);
    constexpr uint32_t c42 = (uint32_t)(((uint64_t)c21 * c21) % (uint64_t)P);
    const uint32_t r = mod_u32<P>(u2 * c42 + u1 * c21 + u0);
    int s = 2 * (int)r <= P ? (int)r : (int)r - P;
    s = neg ? -s : s;
    return __float_as_uint((float)s) >> 16;  // |s| <= 254: exact in BF16
}

// The N residue codes of one element, into half (u & 1) of word u / 2 of each
// modulus' 16-byte chunk (u = 0 .. 7 in increasing order; the caller zeroes out).
template <int N, int T = 0>
__device__ __forceinline__ void residues_of(uint64_t mag, bool neg, int u, uint32_t (&out)[N][4]) {
    if constexpr (T < N) {
        const uint32_t u0 = (uint32_t)mag & 0x1FFFFFu;
        const uint32_t u1 = (uint32_t)(mag >> 21) & 0x1FFFFFu;
        const uint32_t u2 = (uint32_t)(mag >> 42);
        const uint32_t code = residue_code<T>(u0, u1, u2, neg);
        out[T][u >> 1] = (u & 1) ? __byte_perm(out[T][u >> 1], code, 0x5410) : code;
        residues_of<N, T + 1>(mag, neg, u, out);
    }
}

// Byte offset of the 16-byte chunk holding K indices l0 .. l0+7 (l0 % 8 == 0) of
// line x for modulus t (N moduli, tiles of R lines, nks K steps).
template <int R>
__device__ __forceinline__ int64_t crt_offset(int64_t x, int64_t l0, int t, int N, int64_t nks) {
    const int64_t tile = x / R;
    const int r = (int)(x - tile * R);
    const int chunk = (int)((l0 >> 3) & 1) ^ ((r >> 2) & 1);
    return ((tile * N + t) * nks + (l0 >> 4)) * (int64_t)(R * 32) + r * 32 + (chunk << 4);
}

// Row i of A by a CTA of 128 threads: pass 1 max |a| and finiteness, pass 2 the
// residues of 8 consecutive elements per thread (one 16-byte chunk per modulus).
// Rows m <= i < (128-row padding) get zero residues.
template <int N>
__device__ __forceinline__ void crt_split_row(int64_t i, int64_t m, int64_t k,
                                              const double* __restrict__ A, int64_t lda,
                                              uint8_t* __restrict__ res, int64_t kp,
                                              int b, int32_t* __restrict__ exps, unsigned* status,
                                              uint64_t* red, int* bad_sh) {
    const int tid = threadIdx.x;
    const int64_t nks = kp / kStep;
    if (i >= m) {
        for (int64_t l0 = (int64_t)tid * 8; l0 < kp; l0 += (int64_t)blockDim.x * 8)
#pragma unroll
            for (int t = 0; t < N; ++t)
                *reinterpret_cast<uint4*>(res + crt_offset<kTileLines>(i, l0, t, N, nks)) =
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
        uint32_t w[N][4];
#pragma unroll
        for (int t = 0; t < N; ++t) w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0;
        if (!is_bad) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (l0 + u < k) {
                    bool neg;
                    const uint64_t mag = scaled_magnitude(row[l0 + u], e, b, neg);
                    residues_of<N>(mag, neg, u, w);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < N; ++t)
            *reinterpret_cast<uint4*>(res + crt_offset<kTileLines>(i, l0, t, N, nks)) =
                make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(128) crt_split_rows_kernel(int64_t m, int64_t k,
                                                             const double* __restrict__ A,
                                                             int64_t lda, uint8_t* __restrict__ res,
                                                             int64_t kp, int b,
                                                             int32_t* __restrict__ exps,
                                                             unsigned* status) {
    __shared__ uint64_t red[4];
    __shared__ int bad_sh;
    const int64_t mp = (m + kTileLines - 1) / kTileLines * kTileLines;
    for (int64_t i = blockIdx.x; i < mp; i += gridDim.x)
        crt_split_row<N>(i, m, k, A, lda, res, kp, b, exps, status, red, &bad_sh);
}

// Columns of B: CTA (x, y) reduces the `ks` partial maxima of columns 32 x .. +31
// (launch_colmax_part) to their exponents (the CTAs of the first K tile store
// them and flag non-finite columns), then transposes the tile of rows
// 64 y .. +63 through shared memory: thread (jj, lsub) takes 8 consecutive rows
// of column jj, one 16-byte chunk per modulus.  Columns n <= j < (n padded to 256)
// get zero residues.
template <int N>
__global__ void __launch_bounds__(256) crt_split_cols_kernel(int64_t n, int64_t k,
                                                             const double* __restrict__ B,
                                                             int64_t ldb, uint8_t* __restrict__ res,
                                                             int64_t kp, int b,
                                                             int32_t* __restrict__ exps,
                                                             const uint64_t* __restrict__ part,
                                                             int ks, unsigned* status) {
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
            const uint64_t c = ty + 8 < ks ? part[(int64_t)(ty + 8) * n + j] : 0ull;
            mx = a > c ? a : c;
        }
        red[ty][tx] = mx;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) T[ty + 8 * r][tx] = v[r];
    __syncthreads();
    const int jj = tid >> 3, lsub = (tid & 7) * 8;
    const int64_t j = j0 + jj, lbase = l0 + lsub;
    const int64_t np = (n + kTileLinesB - 1) / kTileLinesB * kTileLinesB;
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
        uint32_t w[N][4];
#pragma unroll
        for (int t = 0; t < N; ++t) w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0;
        if (e != GB_BAD_LINE_DEV) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (lbase + u < k) {
                    bool neg;
                    const uint64_t mag = scaled_magnitude(T[lsub + u][jj], e, b, neg);
                    residues_of<N>(mag, neg, u, w);
                }
            }
        }
        const int64_t nks = kp / kStep;
#pragma unroll
        for (int t = 0; t < N; ++t)
            *reinterpret_cast<uint4*>(res + crt_offset<kTileLinesB>(j, lbase, t, N, nks)) =
                make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
}

// ---- c4: residue products on the tensor cores ----------------------------------------
//
// Persistent CTAs, one per SM, 576 threads, over the work items (modulus t, 128 x
// 256 output tile), the tiles of modulus 0 first.  Each modulus is a GEMM of its
// own (no operand is shared between moduli), so the tile is as wide as one MMA
// allows: per K step 12 KiB of operands for 128 x 256 x 16 products.
//   warp 0 lane 0 : producer, two contiguous bulk copies per stage (kKB K steps of
//                   A's and of B's residue tiles) and the item arguments;
//   warp 1        : allocates the 512 TMEM columns; lane 0 issues one kind::f16 MMA
//                   (M = 128, N = 256, K = 16) per K step into one of two
//                   256-column accumulators, the other one every exact unit of
//                   256 K;
//   warps 2 - 17  : epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 and the
//                   64 columns of group (w - 2) / 4, adds each unit's FP32 sums
//                   (exact integers) into int32s, reduces them modulo m_t at the
//                   end and stores the residues as int16.
// Every wait is bounded (4 s of wall time, then the timeout bit, no output for the
// CTA's remaining items, TMEM still freed).
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
constexpr int kBufs = 2;                      // 256-column accumulators
constexpr uint64_t kWaitTimeoutNs = 4000000000ull;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kArgSlots = 4;
constexpr int kKB = 4;                        // K steps per pipeline stage
constexpr int kUnitStages = 4;                // stages per exact unit: 256 K
constexpr int kMaxStages = 4;
constexpr int kEpiCols = kTileLinesB / 4;     // columns of one epilogue warp
constexpr int64_t kUnitK = (int64_t)kKB * kStep * kUnitStages;  // K of one exact unit

struct ItemArgs {
    const uint8_t* a_src;  // A residue tiles of this item's tile row, K step 0
    const uint8_t* b_src;  // B residue tiles of its tile column, K step 0
    int16_t* cres;         // its 128 x 256 block of C residues (row stride ldr)
    int modulus;
};

struct SmemTailCrt {
    uint64_t bars[2 * kMaxStages + 2 * kBufs + 1];  // full, empty; tmem_full, tmem_empty; drain
    uint64_t args_full[kArgSlots];
    uint64_t args_empty[kArgSlots];
    ItemArgs args[kArgSlots];
    uint32_t tmem_holder;
    int abort;
};

// kModuli[t] for a run-time t.
template <int T = 0>
__device__ __forceinline__ int modulus_of(int t) {
    if constexpr (T + 1 < kCrtMaxModuli) {
        constexpr int P = kModuli[T];
        return t == T ? P : modulus_of<T + 1>(t);
    } else {
        constexpr int P = kModuli[T];
        return P;
    }
}

// The items t = blockIdx.x, + gridDim.x, ...: modulus-major; within a modulus
// rasterised (groups of 16 tile rows sweep the tile columns).
struct CrtWalk {
    const uint8_t* ares;
    const uint8_t* bres;
    int16_t* cres;
    int64_t ldr, nks;
    int tiles_m, tiles_n, nmod;
    int64_t t;
    __device__ void start() { t = blockIdx.x; }
    __device__ bool valid() const { return t < (int64_t)nmod * tiles_m * tiles_n; }
    __device__ void next() { t += gridDim.x; }
    __device__ ItemArgs args() const {
        const int64_t per = (int64_t)tiles_m * tiles_n;
        const int mod = (int)(t / per);
        const int bid = (int)(t - (int64_t)mod * per);
        // 16 tile rows per group: a wave of 152 tiles then spans ~16 x 10 tiles,
        // near the shape that minimises the re-reads of 128-row A strips and
        // 256-column B strips from DRAM
        const int group_size = 16 * tiles_n;
        const int first_m = (bid / group_size) * 16;
        const int gm = min(tiles_m - first_m, 16);
        const int tm = first_m + (bid % group_size) % gm;
        const int tn = (bid % group_size) / gm;
        ItemArgs a;
        a.a_src = ares + (((int64_t)tm * nmod + mod) * nks) * kBlockBytes;
        a.b_src = bres + (((int64_t)tn * nmod + mod) * nks) * kBlockBytesB;
        a.cres = cres + (int64_t)mod * ((int64_t)tiles_m * kTileLines) * ldr +
                 (int64_t)tm * kTileLines * ldr + (int64_t)tn * kTileLinesB;
        a.modulus = modulus_of(mod);
        return a;
    }
};

// The symmetric residue of x modulo p (odd), as int16.
__device__ __forceinline__ int32_t sym_mod_i32(int32_t x, int p) {
    int32_t r = x % p;  // sign of x, |r| < p
    r = 2 * r > p ? r - p : r;
    r = 2 * r < -p ? r + p : r;
    return r;
}

__global__ void __launch_bounds__(kThreads, 1)
    crt_products_kernel(CrtWalk walk, int stages, uint32_t slot_bytes, unsigned* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    SmemTailCrt* tail = reinterpret_cast<SmemTailCrt*>(smem + (size_t)stages * slot_bytes);
    uint64_t* full = tail->bars;
    uint64_t* empty = tail->bars + stages;
    uint64_t* tmem_full = tail->bars + 2 * stages;
    uint64_t* tmem_empty = tail->bars + 2 * stages + kBufs;
    uint64_t* drain = tail->bars + 2 * stages + 2 * kBufs;
    volatile int* abort = &tail->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nks = (int)walk.nks;
    const int nst = (nks + kKB - 1) / kKB;

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < kBufs; ++b) {
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

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        int st = 0;
        uint32_t ph = 0;
        CrtWalk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !*abort; w.next(), ++ti) {
            const ItemArgs a = w.args();
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_empty[as], ((ti / kArgSlots) & 1u) ^ 1u, abort,
                                        status, kStatusTimeout, kWaitTimeoutNs))
                break;
            tail->args[as] = a;
            ptx::mbar_arrive(&tail->args_full[as]);
            for (int j = 0; j < nst; ++j) {
                if (!ptx::mbar_wait_bounded(&empty[st], ph ^ 1u, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs))
                    break;
                const int ks0 = j * kKB;
                const int kc = nks - ks0 < kKB ? nks - ks0 : kKB;
                uint8_t* sa = smem + (size_t)st * slot_bytes;
                ptx::mbar_arrive_expect_tx(&full[st],
                                           (uint32_t)kc * (kBlockBytes + kBlockBytesB));
                ptx::bulk_load(sa, a.a_src + (size_t)ks0 * kBlockBytes, (uint32_t)kc * kBlockBytes,
                               &full[st]);
                ptx::bulk_load(sa + kKB * kBlockBytes, a.b_src + (size_t)ks0 * kBlockBytesB,
                               (uint32_t)kc * kBlockBytesB, &full[st]);
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = ptx::idesc_bf16_f32(kTileLines, kTileLinesB);
        const uint64_t adesc0 = ptx::umma_desc_sw32(ptx::smem_u32(smem));
        const uint32_t slot16 = slot_bytes >> 4;  // descriptor address step of one slot
        int st = 0;
        uint32_t ph = 0;
        uint32_t unit = 0;  // units issued by this CTA so far: accumulator unit % kBufs
        bool stop = false;
        CrtWalk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !*abort && !stop; w.next(), ++ti) {
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_full[as], (ti / kArgSlots) & 1u, abort, status,
                                        kStatusTimeout, kWaitTimeoutNs))
                break;
            ptx::mbar_arrive(&tail->args_empty[as]);
            if (stages == kUnitStages) {
                // K is a whole number of units (the layout pads it), so every unit is
                // kUnitStages full stages starting at slot 0: slots, descriptors and
                // MMAs at compile-time offsets.  The issuing thread's own instructions
                // per MMA are what bound this kernel's tensor pipe, so this loop keeps
                // them to the barrier waits, the MMAs and the commits.
                for (int u = 0; u < nst / kUnitStages; ++u) {
                    const uint32_t b = unit % kBufs;
                    if (unit >= (uint32_t)kBufs) {
                        // the epilogue has read this accumulator's previous unit
                        if (!ptx::mbar_wait_bounded(&tmem_empty[b], ((unit / kBufs) - 1) & 1u,
                                                    abort, status, kStatusTimeout,
                                                    kWaitTimeoutNs)) {
                            stop = true;
                            break;
                        }
                        ptx::tc_fence_after();
                    }
                    const uint32_t acc = tmem_base + b * (uint32_t)kTileLinesB;
#pragma unroll
                    for (int s2 = 0; s2 < kUnitStages; ++s2) {
                        if (!ptx::mbar_wait_bounded(&full[s2], ph, abort, status, kStatusTimeout,
                                                    kWaitTimeoutNs)) {
                            stop = true;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint64_t adesc = adesc0 + (uint64_t)(s2 * slot16);
                        const uint64_t bdesc = adesc + (uint64_t)((kKB * kBlockBytes) >> 4);
#pragma unroll
                        for (int kk = 0; kk < kKB; ++kk)
                            ptx::mma_bf16(acc, adesc + (uint64_t)((kk * kBlockBytes) >> 4),
                                          bdesc + (uint64_t)((kk * kBlockBytesB) >> 4), idesc,
                                          (s2 == 0 && kk == 0) ? 0u : 1u);
                        ptx::mma_commit(&empty[s2]);
                    }
                    if (stop) break;
                    ph ^= 1u;
                    ptx::mma_commit(&tmem_full[b]);
                    ++unit;
                }
                continue;
            }
            // fewer ring slots than stages per unit: slot by slot
            int in_unit = 0;
            uint32_t acc = tmem_base;
            for (int j = 0; j < nst; ++j) {
                const bool unit_start = in_unit == 0;
                if (unit_start) {
                    const uint32_t b = unit % kBufs;
                    if (unit >= (uint32_t)kBufs) {
                        // the epilogue has read this accumulator's previous unit
                        if (!ptx::mbar_wait_bounded(&tmem_empty[b], ((unit / kBufs) - 1) & 1u,
                                                    abort, status, kStatusTimeout,
                                                    kWaitTimeoutNs)) {
                            stop = true;
                            break;
                        }
                        ptx::tc_fence_after();
                    }
                    acc = tmem_base + b * (uint32_t)kTileLinesB;
                }
                if (!ptx::mbar_wait_bounded(&full[st], ph, abort, status, kStatusTimeout,
                                            kWaitTimeoutNs)) {
                    stop = true;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t a0 = ptx::smem_u32(smem + (size_t)st * slot_bytes);
                const uint64_t adesc = ptx::umma_desc_sw32(a0);
                const uint64_t bdesc = ptx::umma_desc_sw32(a0 + kKB * kBlockBytes);
                const int kc = nks - j * kKB < kKB ? nks - j * kKB : kKB;
#pragma unroll
                for (int kk = 0; kk < kKB; ++kk) {
                    if (kk < kc)
                        ptx::mma_bf16(acc, adesc + (uint64_t)((kk * kBlockBytes) >> 4),
                                      bdesc + (uint64_t)((kk * kBlockBytesB) >> 4), idesc,
                                      (unit_start && kk == 0) ? 0u : 1u);
                }
                ptx::mma_commit(&empty[st]);
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
                if (++in_unit == kUnitStages || j + 1 == nst) {
                    ptx::mma_commit(&tmem_full[unit % kBufs]);
                    ++unit;
                    in_unit = 0;
                }
            }
        }
    } else if (warp >= 2) {
        // ---- epilogue ----
        const int quarter = warp & 3;
        const int cgroup = (warp - 2) >> 2;
        const uint32_t lane_addr =
            tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(kEpiCols * cgroup);
        const int nunits = (nst + kUnitStages - 1) / kUnitStages;
        uint32_t unit = 0;
        bool stop = false;
        CrtWalk w = walk;
        int ti = 0;
        for (w.start(); w.valid() && !stop; w.next(), ++ti) {
            const int as = ti % kArgSlots;
            if (!ptx::mbar_wait_bounded(&tail->args_full[as], (ti / kArgSlots) & 1u, abort, status,
                                        kStatusTimeout, kWaitTimeoutNs))
                break;
            int16_t* cres = tail->args[as].cres;
            const int p = tail->args[as].modulus;
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tail->args_empty[as]);
            int32_t acc[kEpiCols];
#pragma unroll
            for (int j = 0; j < kEpiCols; ++j) acc[j] = 0;
            for (int c = 0; c < nunits; ++c, ++unit) {
                const uint32_t b = unit % kBufs;
                const bool ok = ptx::mbar_wait_bounded(&tmem_full[b], (unit / kBufs) & 1u, abort,
                                                       status, kStatusTimeout, kWaitTimeoutNs);
                ptx::tc_fence_after();
                if (!ok || *abort) {
                    stop = true;
                    break;
                }
                // 16 columns per load (the 64 totals hold most of the registers);
                // each unit's sums are integers of at most 2^24 in magnitude
#pragma unroll
                for (int h = 0; h < kEpiCols; h += 16) {
                    uint32_t v[16];
                    ptx::tmem_ld_32x32b_x16(lane_addr + b * (uint32_t)kTileLinesB + h, v);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[h + j] += __float2int_rn(__uint_as_float(v[j]));
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tmem_empty[b]);
                // the int32 totals are reduced every 64 units, before they could
                // reach 2^31
                if ((c & 63) == 63) {
#pragma unroll
                    for (int j = 0; j < kEpiCols; ++j) acc[j] = sym_mod_i32(acc[j], p);
                }
            }
            if (stop) break;
            // this thread's row of the tile, columns 64 cgroup .. + 63: 128 bytes
            int16_t* dst = cres + (int64_t)(quarter * 32 + lane) * walk.ldr + kEpiCols * cgroup;
#pragma unroll
            for (int q4 = 0; q4 < kEpiCols / 8; ++q4) {
                uint32_t wv[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int j = 8 * q4 + 2 * h;
                    const uint32_t lo = (uint32_t)(uint16_t)(int16_t)sym_mod_i32(acc[j], p);
                    const uint32_t hi = (uint32_t)(uint16_t)(int16_t)sym_mod_i32(acc[j + 1], p);
                    wv[h] = lo | (hi << 16);
                }
                *reinterpret_cast<uint4*>(dst + 8 * q4) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
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

// ---- c5 + c6: reconstruction and the single rounding -------------------------------

// The reconstruction's constants in 26-bit limbs (every product of a residue
// and a limb then fits a 32 x 32 -> 64-bit multiply and the limb sums stay far
// below 2^63): w_t = sum_i wl[t][i] 2^(26 i), M = sum_i Ml[i] 2^(26 i).
constexpr int kLimbs = 5;  // 130 bits > the 125 of M
struct CrtConsts {
    int32_t wl[kCrtMaxModuli][kLimbs];
    int32_t Ml[kLimbs];
    float frac[kCrtMaxModuli];  // w_t / M
};

// The reconstruction of one output from its N residues r: q = nearest integer
// to sum_t r_t w_t / M (FP32 is ample: the sum lies within 1/4 of an integer
// because |C'| <= M / 4), then C' = sum_t r_t w_t - q M limb by limb (each limb
// sum |L_i| < 2^39) and the limbs joined in 128 bits (|C'| < 2^123).
template <int N>
__device__ __forceinline__ I128 reconstruct(const int32_t (&r)[N], const CrtConsts& K) {
    float qf = 0.0f;
#pragma unroll
    for (int t = 0; t < N; ++t) qf = __fmaf_rn((float)r[t], K.frac[t], qf);
    const int32_t q = __float2int_rn(qf);
    int64_t L[kLimbs];
#pragma unroll
    for (int i = 0; i < kLimbs; ++i) L[i] = -(int64_t)q * (int64_t)K.Ml[i];
#pragma unroll
    for (int t = 0; t < N; ++t)
#pragma unroll
        for (int i = 0; i < kLimbs; ++i) L[i] += (int64_t)r[t] * (int64_t)K.wl[t][i];
    __int128 acc = L[kLimbs - 1];
#pragma unroll
    for (int i = kLimbs - 2; i >= 0; --i) acc = acc * ((__int128)1 << 26) + L[i];
    return I128{(int64_t)(acc >> 64), (uint64_t)acc};
}

// Two consecutive outputs per thread (the residues of a pair are one 32-bit word
// per modulus), threads along a row of C, rows across grid.y: reconstruction,
// RN(C' 2^E) and alpha / beta.
template <int N>
__global__ void __launch_bounds__(256) crt_combine_kernel(int64_t m, int64_t n,
                                                          const int16_t* __restrict__ cres,
                                                          int64_t ldr, int64_t plane,
                                                          const int32_t* __restrict__ eA,
                                                          const int32_t* __restrict__ fB,
                                                          int b, double alpha, double beta,
                                                          double* __restrict__ C, int64_t ldc,
                                                          CrtConsts K) {
    const long long ab = __double_as_longlong(alpha), bb = __double_as_longlong(beta);
    const bool beta0 = (bb & 0x7FFFFFFFFFFFFFFFll) == 0;
    const bool plain = ab == 0x3FF0000000000000ll && beta0;
    const int64_t j0 = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (j0 >= n) return;
    const bool two = j0 + 1 < n;
    const int32_t f0 = fB[j0], f1 = two ? fB[j0 + 1] : 0;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
        // ldr is a multiple of 256 and j0 even: one aligned 32-bit load per modulus
        const uint32_t* src = reinterpret_cast<const uint32_t*>(cres + i * ldr + j0);
        int32_t r0[N], r1[N];
#pragma unroll
        for (int t = 0; t < N; ++t) {
            const uint32_t w = src[(int64_t)t * (plane >> 1)];
            r0[t] = (int32_t)(int16_t)(w & 0xFFFFu);
            r1[t] = (int32_t)(int16_t)(w >> 16);
        }
        const int32_t ei = eA[i];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int32_t fj = h ? f1 : f0;
            double out;
            if (ei == GB_BAD_LINE_DEV || fj == GB_BAD_LINE_DEV) {
                out = __longlong_as_double(0x7FF8000000000000ll);
            } else {
                out = i128_to_double_scaled(reconstruct<N>(h ? r1 : r0, K), ei + fj - 2 * b);
                if (!plain) {
                    double o = __dmul_rn(alpha, out);
                    if (!beta0) o = __dadd_rn(o, __dmul_rn(beta, C[i * ldc + j0 + h]));
                    out = o;
                }
            }
            C[i * ldc + j0 + h] = out;
        }
    }
}

#define GB_SWITCH_N(nm, CALL)                                                           \
    switch (nm) {                                                                       \
        case 1: CALL(1); break;  case 2: CALL(2); break;  case 3: CALL(3); break;       \
        case 4: CALL(4); break;  case 5: CALL(5); break;  case 6: CALL(6); break;       \
        case 7: CALL(7); break;  case 8: CALL(8); break;  case 9: CALL(9); break;       \
        case 10: CALL(10); break; case 11: CALL(11); break; case 12: CALL(12); break;   \
        case 13: CALL(13); break; case 14: CALL(14); break;                             \
        default: return cudaErrorInvalidValue;                                          \
    }

// Host copies of the moduli (the device code takes them from kModuli at compile time).
unsigned __int128 modulus_product(int N) {
    unsigned __int128 M = 1;
    for (int t = 0; t < N; ++t) M *= (unsigned __int128)kModuli[t];
    return M;
}

int bit_length(unsigned __int128 x) {
    int l = 0;
    while (x) {
        ++l;
        x >>= 1;
    }
    return l;
}

// x^-1 mod p (p prime, x not a multiple of p), by the extended Euclidean algorithm.
int64_t inverse_mod(int64_t x, int64_t p) {
    int64_t a = ((x % p) + p) % p, b = p, u = 1, v = 0;
    while (b) {
        const int64_t q = a / b;
        int64_t t = a - q * b;
        a = b;
        b = t;
        t = u - q * v;
        u = v;
        v = t;
    }
    return ((u % p) + p) % p;
}

CrtConsts crt_consts(int N) {
    CrtConsts K{};
    const unsigned __int128 M = modulus_product(N);
    const unsigned __int128 mask = ((unsigned __int128)1 << 26) - 1;
    for (int t = 0; t < N; ++t) {
        const unsigned __int128 Mt = M / (unsigned __int128)kModuli[t];
        const int64_t inv = inverse_mod((int64_t)(Mt % (unsigned __int128)kModuli[t]), kModuli[t]);
        const unsigned __int128 w = Mt * (unsigned __int128)inv;  // < M
        for (int i = 0; i < kLimbs; ++i) K.wl[t][i] = (int32_t)((w >> (26 * i)) & mask);
        K.frac[t] = (float)((double)w / (double)M);
    }
    for (int i = 0; i < kLimbs; ++i) K.Ml[i] = (int32_t)((M >> (26 * i)) & mask);
    return K;
}

}  // namespace

int crt_scale_bits(int N, int64_t k) {
    if (N < 1 || N > kCrtMaxModuli) return 0;
    const unsigned __int128 M = modulus_product(N);
    const unsigned __int128 kk = (unsigned __int128)(k < 1 ? 1 : k);
    int best = 0;
    for (int b = 1; b <= 62; ++b) {
        // 4 k 2^(2b) <= M, the left side formed only while it fits 128 bits
        if (bit_length(kk) + 2 + 2 * b > 126) break;
        if (((kk << 2) << (2 * b)) <= M) best = b;
    }
    return best;
}

CrtLayout crt_layout(int N, int64_t m, int64_t n, int64_t k) {
    CrtLayout L{};
    L.N = N;
    // K padded to whole exact units (the split kernels write zero residues there):
    // every unit of the products kernel is kUnitStages full stages
    L.kp = ((k + kUnitK - 1) / kUnitK) * kUnitK;
    if (L.kp == 0) L.kp = kUnitK;
    L.mp = (m + kTileLines - 1) / kTileLines * kTileLines;
    L.np = (n + kTileLinesB - 1) / kTileLinesB * kTileLinesB;
    L.b = crt_scale_bits(N, k);
    auto up = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    size_t off = 0;
    L.a_res = off;
    off = up(off + 2 * (size_t)N * (size_t)L.mp * (size_t)L.kp);
    L.b_res = off;
    off = up(off + 2 * (size_t)N * (size_t)L.np * (size_t)L.kp);
    L.c_res = off;
    off = up(off + 2 * (size_t)N * (size_t)L.mp * (size_t)L.np);
    L.a_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)m);
    L.b_exp = off;
    off = up(off + sizeof(int32_t) * (size_t)n);
    L.b_part = off;
    off = up(off + sizeof(uint64_t) * (size_t)kColmaxParts * (size_t)n);
    L.total = off;
    return L;
}

cudaError_t crt_split_a(const Launch& L, int N, int b, int64_t m, int64_t k, const double* A,
                        int64_t lda, uint8_t* ares, int64_t kp, int32_t* ea) {
    if (m == 0) return cudaSuccess;
    int64_t blocks = (m + kTileLines - 1) / kTileLines * kTileLines;
    const int64_t cap = (int64_t)L.sm_count * 16;
    if (blocks > cap) blocks = cap;
#define GB_LAUNCH(NN)                                                                          \
    crt_split_rows_kernel<NN><<<(unsigned)blocks, 128, 0, L.stream>>>(m, k, A, lda, ares, kp, b, \
                                                                      ea, L.status)
    GB_SWITCH_N(N, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaGetLastError();
}

cudaError_t crt_split_b(const Launch& L, int N, int b, int64_t n, int64_t k, const double* B,
                        int64_t ldb, uint8_t* bres, int64_t kp, int32_t* fb, uint64_t* part) {
    if (n == 0) return cudaSuccess;
    int ks = 1;
    cudaError_t e = launch_colmax_part(L, n, k, B, ldb, part, &ks);
    if (e != cudaSuccess) return e;
    const int64_t np = (n + kTileLinesB - 1) / kTileLinesB * kTileLinesB;
    const dim3 grid((unsigned)(np / 32), (unsigned)((kp + 63) / 64));
#define GB_LAUNCH(NN)                                                                        \
    crt_split_cols_kernel<NN><<<grid, 256, 0, L.stream>>>(n, k, B, ldb, bres, kp, b, fb, part, \
                                                          ks, L.status)
    GB_SWITCH_N(N, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaGetLastError();
}

cudaError_t crt_residue_products(const Launch& L, int N, int64_t m, int64_t n, int64_t kp,
                                 const uint8_t* ares, const uint8_t* bres, int16_t* cres) {
    if (m == 0 || n == 0) return cudaSuccess;
    // the residues' K extent is whole exact units (crt_layout pads it so): the
    // kernel's unit loop has no partial stages
    if (kp <= 0 || kp % kUnitK != 0) return cudaErrorInvalidValue;
    const int64_t mp = (m + kTileLines - 1) / kTileLines * kTileLines;
    const int64_t np = (n + kTileLinesB - 1) / kTileLinesB * kTileLinesB;
    {
        const uint32_t slot = kKB * (kBlockBytes + kBlockBytesB);  // 48 KiB, 1024-aligned
        const int fixed = 1024 + (int)sizeof(SmemTailCrt) + 64;
        int stages = (kSmemLimit - fixed) / (int)slot;
        if (stages > kMaxStages) stages = kMaxStages;
        if (stages < 2) return cudaErrorInvalidValue;
        const size_t smem = (size_t)stages * slot + fixed;
        const int tiles_m = (int)(mp / kTileLines), tiles_n = (int)(np / kTileLinesB);
        const int64_t items = (int64_t)N * tiles_m * tiles_n;
        const int grid = (int)(items < L.sm_count ? items : L.sm_count);
        cudaError_t e = cudaFuncSetAttribute(crt_products_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemLimit);
        if (e != cudaSuccess) return e;
        const CrtWalk w{ares, bres, cres, np, kp / kStep, tiles_m, tiles_n, N, 0};
        crt_products_kernel<<<grid, kThreads, smem, L.stream>>>(w, stages, slot, L.status);
        return cudaGetLastError();
    }
}

cudaError_t crt_combine(const Launch& L, int N, int b, int64_t m, int64_t n, double alpha,
                        double beta, double* C, int64_t ldc, const int16_t* cres,
                        const int32_t* ea, const int32_t* fb) {
    if (m == 0 || n == 0) return cudaSuccess;
    const int64_t mp = (m + kTileLines - 1) / kTileLines * kTileLines;
    const int64_t np = (n + kTileLinesB - 1) / kTileLinesB * kTileLinesB;
    const CrtConsts K = crt_consts(N);
    // column pairs across the threads of a CTA (coalesced), rows across grid.y
    const int64_t bx = (n + 511) / 512;
    int64_t by = ((int64_t)L.sm_count * 8 + bx - 1) / bx;
    if (by > m) by = m;
    if (by > 65535) by = 65535;
    const dim3 grid((unsigned)bx, (unsigned)by);
    const int64_t plane = mp * np;
#define GB_LAUNCH(NN)                                                                           \
    crt_combine_kernel<NN><<<grid, 256, 0, L.stream>>>(m, n, cres, np, plane, ea, fb, b, alpha, \
                                                       beta, C, ldc, K)
    GB_SWITCH_N(N, GB_LAUNCH)
#undef GB_LAUNCH
    return cudaGetLastError();
}

cudaError_t crt_products(const Launch& L, int N, int b, int64_t m, int64_t n, int64_t kp,
                         double alpha, double beta, double* C, int64_t ldc, const uint8_t* ares,
                         const uint8_t* bres, int16_t* cres, const int32_t* ea,
                         const int32_t* fb) {
    cudaError_t e = crt_residue_products(L, N, m, n, kp, ares, bres, cres);
    if (e == cudaSuccess) e = crt_combine(L, N, b, m, n, alpha, beta, C, ldc, cres, ea, fb);
    return e;
}

cudaError_t launch_crt_gemm(const Launch& L, const Gemm& g, uint8_t* ws, const CrtLayout& lay) {
    const int N = lay.N;
    if (g.m == 0 || g.n == 0) return cudaSuccess;
    if (N < 1 || N > kCrtMaxModuli || lay.b < 1) return cudaErrorInvalidValue;
    int32_t* ea = reinterpret_cast<int32_t*>(ws + lay.a_exp);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + lay.b_exp);
    cudaError_t e = crt_split_a(L, N, lay.b, g.m, g.k, g.A, g.lda, ws + lay.a_res, lay.kp, ea);
    if (e == cudaSuccess)
        e = crt_split_b(L, N, lay.b, g.n, g.k, g.B, g.ldb, ws + lay.b_res, lay.kp, fb,
                        reinterpret_cast<uint64_t*>(ws + lay.b_part));
    if (e == cudaSuccess)
        e = crt_products(L, N, lay.b, g.m, g.n, lay.kp, g.alpha, g.beta, g.C, g.ldc,
                         ws + lay.a_res, ws + lay.b_res,
                         reinterpret_cast<int16_t*>(ws + lay.c_res), ea, fb);
    return e;
}

}  // namespace gb
