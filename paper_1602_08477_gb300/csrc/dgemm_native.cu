// Native FP64 GEMM kernels for sm_103a: C <- alpha*A*B + beta*C (Section 4.2).
//
// Three work divisions of the grid / block / thread / element hierarchy
// (Section 3.2, Table 2 CUDA row: blocks = N/(B*V), threads = B, elements = V):
//   naive  - one thread per element of C, operands straight from global memory
//            (the nested-loop kernel of Section 4.2.1 mapped to CUDA);
//   tiled  - square T x T shared-memory tiles, one element per thread (the
//            block-parallel tiling kernel of Section 4.2.1);
//   dfma   - hierarchical tiling with V x V elements per thread in registers
//            (Section 4.2.2, Fig. "tiling_kernel"), FP64 FMA pipe;
//   dmma   - the same hierarchy with a warp as the thread level and the warp's
//            register tile as the element level, on FP64 mma.sync (DMMA).
// On GB300 the FP64 FMA pipe sustains the nominal 2 FMA / clock / SM, ahead of
// FP64 mma.sync; the library's default is therefore the tiled (small sizes) and
// dfma (large sizes) path.
// Row-major operands with leading dimensions; beta == 0 never reads C.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace gb {
namespace {

template <bool kBeta0>
__device__ __forceinline__ void store_out(double* C, int64_t idx, double alpha, double acc,
                                          double beta) {
    if (kBeta0) {
        C[idx] = alpha * acc;
    } else {
        C[idx] = alpha * acc + beta * C[idx];
    }
}

// ---- C <- beta * C ---------------------------------------------------------------
__global__ void scale_kernel(int64_t m, int64_t n, double beta, double* __restrict__ C,
                             int64_t ldc) {
    const int64_t total = m * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, j = t - i * n;
        double* c = &C[i * ldc + j];
        *c = (beta == 0.0) ? 0.0 : beta * (*c);
    }
}

// ---- naive: one element per thread ---------------------------------------------------
template <bool kBeta0>
__global__ void naive_kernel(int64_t m, int64_t n, int64_t k, double alpha,
                             const double* __restrict__ A, int64_t lda,
                             const double* __restrict__ B, int64_t ldb, double beta,
                             double* __restrict__ C, int64_t ldc) {
    const int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m || j >= n) return;
    const double* a = A + i * lda;
    const double* b = B + j;
    double s = 0.0;
    for (int64_t l = 0; l < k; ++l) s = fma(a[l], b[l * ldb], s);
    store_out<kBeta0>(C, i * ldc + j, alpha, s, beta);
}

// ---- tiled: T x T shared-memory tiles, one element per thread ------------------------
template <int T, bool kBeta0>
__global__ void tiled_kernel(int64_t m, int64_t n, int64_t k, double alpha,
                             const double* __restrict__ A, int64_t lda,
                             const double* __restrict__ B, int64_t ldb, double beta,
                             double* __restrict__ C, int64_t ldc) {
    __shared__ double As[T][T];
    __shared__ double Bs[T][T];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i = blockIdx.y * (int64_t)T + ty;
    const int64_t j = blockIdx.x * (int64_t)T + tx;
    double s = 0.0;
    for (int64_t l0 = 0; l0 < k; l0 += T) {
        As[ty][tx] = (i < m && l0 + tx < k) ? A[i * lda + l0 + tx] : 0.0;
        Bs[ty][tx] = (l0 + ty < k && j < n) ? B[(l0 + ty) * ldb + j] : 0.0;
        __syncthreads();
#pragma unroll
        for (int e = 0; e < T; ++e) s = fma(As[ty][e], Bs[e][tx], s);
        __syncthreads();
    }
    if (i < m && j < n) store_out<kBeta0>(C, i * ldc + j, alpha, s, beta);
}

// ---- dfma: TY x TX = 256 threads, VY x VX elements per thread -------------------------
// Tile (TY VY) x (TX VX); thread (ty, tx) = (tid / TX, tid % TX) owns rows ty + TY r
// and columns tx + TX c (r < VY, c < VX), so shared-memory reads are broadcasts /
// consecutive and a warp's global stores are runs of TX contiguous doubles.  K
// advances in steps of BK through a register-prefetched, double-buffered
// shared-memory stage.  Every element accumulates fma(A[i,l], B[l,j], acc) for
// l = 0, 1, ..., k-1 in order, so all tile shapes and thread layouts give
// bit-identical results.
// FP64 is the bottleneck on GB300: a warp FMA holds the SM's FP64 pipe for 16 clocks
// whether 1 or 32 of its lanes are active.  So no warp issues an FMA for padding: a
// warp (rows 32w / TX + [0, 32 / TX)) skips the row parts r that hold no row below m,
// every warp the column parts c with TX c >= n - col0 (warp-uniform branches into
// code specialised for the active parts), and the last K step runs only the k % BK
// remaining indices.  Ragged problems then waste FMAs only at the granularity of a
// warp's (32 / TX) x TX block, not on whole padded tiles.  TX = 16 serves the
// single-GEMM kernel, TX = 8 (4 x 8 blocks) the grouped kernel's small problems.
template <int VY, int VX, int TX = 16>
struct DfmaShape {
    static_assert(TX == 8 || TX == 16, "8 or 16 threads along the columns");
    static constexpr int TY = 256 / TX;
    static constexpr int BM = TY * VY, BN = TX * VX;
    static constexpr int BK = (VY * VX >= 64) ? 8 : 16;   // <= 48 KB static smem
    static constexpr int A_STAGE = BK * (BM + 1), B_STAGE = BK * BN;
    static constexpr int SMEM_DOUBLES = 2 * (A_STAGE + B_STAGE);
};

// One K index l of the active parts r < RA, c < CA.
template <int VY, int VX, int TX, int RA, int CA>
__device__ __forceinline__ void dfma_step(const double* __restrict__ as,
                                          const double* __restrict__ bs, int l, int ty, int tx,
                                          double (&acc)[VY][VX]) {
    using S = DfmaShape<VY, VX, TX>;
    double av[RA], bv[CA];
#pragma unroll
    for (int r = 0; r < RA; ++r) av[r] = as[l * (S::BM + 1) + ty + S::TY * r];
#pragma unroll
    for (int c = 0; c < CA; ++c) bv[c] = bs[l * S::BN + tx + TX * c];
#pragma unroll
    for (int r = 0; r < RA; ++r)
#pragma unroll
        for (int c = 0; c < CA; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
}

// The nl (<= BK) K indices of one shared-memory stage for the active parts.
template <int VY, int VX, int TX, int RA, int CA>
__device__ __forceinline__ void dfma_stage(const double* __restrict__ as,
                                           const double* __restrict__ bs, int nl, int ty,
                                           int tx, double (&acc)[VY][VX]) {
    constexpr int BK = DfmaShape<VY, VX, TX>::BK;
    if (nl == BK) {
#pragma unroll
        for (int l = 0; l < BK; ++l) dfma_step<VY, VX, TX, RA, CA>(as, bs, l, ty, tx, acc);
    } else {
#pragma unroll 1
        for (int l = 0; l < nl; ++l) dfma_step<VY, VX, TX, RA, CA>(as, bs, l, ty, tx, acc);
    }
}

template <int VY, int VX, int TX, int RA, int CA>
__device__ __forceinline__ void dfma_stage_ca(int ca, const double* __restrict__ as,
                                              const double* __restrict__ bs, int nl, int ty,
                                              int tx, double (&acc)[VY][VX]) {
    if constexpr (CA > 1) {
        if (ca < CA) return dfma_stage_ca<VY, VX, TX, RA, CA - 1>(ca, as, bs, nl, ty, tx, acc);
    }
    dfma_stage<VY, VX, TX, RA, CA>(as, bs, nl, ty, tx, acc);
}

template <int VY, int VX, int TX, int RA>
__device__ __forceinline__ void dfma_stage_ra(int ra, int ca, const double* __restrict__ as,
                                              const double* __restrict__ bs, int nl, int ty,
                                              int tx, double (&acc)[VY][VX]) {
    if constexpr (RA > 1) {
        if (ra < RA) return dfma_stage_ra<VY, VX, TX, RA - 1>(ra, ca, as, bs, nl, ty, tx, acc);
    }
    dfma_stage_ca<VY, VX, TX, RA, VX>(ca, as, bs, nl, ty, tx, acc);
}

// Dispatch on the warp's active row parts ra and the tile's active column parts ca
// (both >= 1).  Register tiles of more than 16 elements (large square problems,
// where padding is negligible) keep the full tile and only trim the K tail.
template <int VY, int VX, int TX>
__device__ __forceinline__ void dfma_stage_active(int ra, int ca, const double* __restrict__ as,
                                                  const double* __restrict__ bs, int nl,
                                                  int ty, int tx, double (&acc)[VY][VX]) {
    if constexpr (VY * VX <= 16)
        dfma_stage_ra<VY, VX, TX, VY>(ra, ca, as, bs, nl, ty, tx, acc);
    else
        dfma_stage<VY, VX, TX, VY, VX>(as, bs, nl, ty, tx, acc);
}

// kMayBeEmpty: the tile may belong to a problem with k == 0 (grouped problems with
// alpha == 0 or k == 0 run here as C <- beta C); single launches never do.
template <int VY, int VX, int TX = 16, bool kMayBeEmpty = false>
__device__ __forceinline__ void dfma_tile(int64_t m, int64_t n, int64_t k, double alpha,
                                          const double* __restrict__ A, int64_t lda,
                                          const double* __restrict__ B, int64_t ldb,
                                          double beta, double* __restrict__ C, int64_t ldc,
                                          int64_t row0, int64_t col0, double* smem) {
    using S = DfmaShape<VY, VX, TX>;
    constexpr int BM = S::BM, BN = S::BN, BK = S::BK, TY = S::TY;
    constexpr int A_PER_T = BM * BK / 256;  // elements of the A tile each thread loads
    constexpr int B_PER_T = BK * BN / 256;
    double* As = smem;                       // [2][BK][BM + 1]: transposed, As[l][row]
    double* Bs = smem + 2 * S::A_STAGE;      // [2][BK][BN]
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    double acc[VY][VX];
#pragma unroll
    for (int r = 0; r < VY; ++r)
#pragma unroll
        for (int c = 0; c < VX; ++c) acc[r][c] = 0.0;

    double ra[A_PER_T], rb[B_PER_T];
    auto load_regs = [&](int64_t l0) {
#pragma unroll
        for (int u = 0; u < A_PER_T; ++u) {
            const int e = tid + 256 * u;          // e in [0, BM*BK)
            const int r = e / BK, l = e % BK;     // consecutive threads along l
            const int64_t gi = row0 + r, gl = l0 + l;
            ra[u] = (gi < m && gl < k) ? A[gi * lda + gl] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < B_PER_T; ++u) {
            const int e = tid + 256 * u;
            const int l = e / BN, c = e % BN;     // consecutive threads along columns
            const int64_t gl = l0 + l, gj = col0 + c;
            rb[u] = (gl < k && gj < n) ? B[gl * ldb + gj] : 0.0;
        }
    };
    auto store_smem = [&](int buf) {
        double* as = As + buf * S::A_STAGE;
        double* bs = Bs + buf * S::B_STAGE;
#pragma unroll
        for (int u = 0; u < A_PER_T; ++u) {
            const int e = tid + 256 * u;
            as[(e % BK) * (BM + 1) + e / BK] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < B_PER_T; ++u) {
            const int e = tid + 256 * u;
            bs[(e / BN) * BN + e % BN] = rb[u];
        }
    };

    // active parts: row part r of warp w holds rows 32w / TX + [0, 32 / TX) + TY r
    const int64_t mr = m - row0, nr = n - col0;
    const int64_t wrows = mr - (int64_t)((tid >> 5) * (32 / TX));
    const int act_r = wrows <= 0 ? 0 : (wrows >= (int64_t)TY * VY ? VY
                                                                   : (int)((wrows + TY - 1) / TY));
    const int act_c = nr <= 0 ? 0 : (nr >= (int64_t)TX * VX ? VX : (int)((nr + TX - 1) / TX));
    const int64_t nk = (k + BK - 1) / BK;
    if (nk > 0) {
        load_regs(0);
        store_smem(0);
    }
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load_regs((kt + 1) * BK);
        const double* as = As + buf * S::A_STAGE;
        const double* bs = Bs + buf * S::B_STAGE;
        const int nl = kt + 1 < nk ? BK : (int)(k - kt * BK);
        if (act_r == VY && act_c == VX && nl == BK)
            dfma_stage<VY, VX, TX, VY, VX>(as, bs, BK, ty, tx, acc);
        else if (act_r > 0 && act_c > 0)
            dfma_stage_active<VY, VX, TX>(act_r, act_c, as, bs, nl, ty, tx, acc);
        if (kt + 1 < nk) store_smem(buf ^ 1);
        __syncthreads();
    }
    const bool beta0 = beta == 0.0;
    // k == 0 (a grouped problem with alpha == 0 or k == 0): C <- beta C exactly as
    // the scaling kernel writes it (beta C, or 0 when beta == 0), not alpha 0 + beta C,
    // whose zeros would differ in sign
    const bool scale_only = kMayBeEmpty && k == 0;
#pragma unroll
    for (int r = 0; r < VY; ++r) {
        const int64_t gi = row0 + ty + TY * r;
        if (gi >= m) continue;
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int64_t gj = col0 + tx + TX * c;
            if (gj < n) {
                double* cp = &C[gi * ldc + gj];
                if (scale_only)
                    *cp = beta0 ? 0.0 : beta * (*cp);
                else
                    *cp = beta0 ? alpha * acc[r][c] : alpha * acc[r][c] + beta * (*cp);
            }
        }
    }
    __syncthreads();  // the shared-memory stages may be reused by the caller's next tile
}

template <int V>
__global__ void __launch_bounds__(256) dfma_kernel(int64_t m, int64_t n, int64_t k,
                                                   double alpha, const double* __restrict__ A,
                                                   int64_t lda, const double* __restrict__ B,
                                                   int64_t ldb, double beta,
                                                   double* __restrict__ C, int64_t ldc) {
    __shared__ __align__(16) double smem[DfmaShape<V, V>::SMEM_DOUBLES];
    dfma_tile<V, V>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                    blockIdx.y * (int64_t)DfmaShape<V, V>::BM,
                    blockIdx.x * (int64_t)DfmaShape<V, V>::BN, smem);
}

// ---- dmma: FP64 mma.sync.m16n8k4 warp tiles ----------------------------------------
// Fragment layout of mma.m16n8k4 .f64 (PTX ISA, "Matrix fragments for mma.m16n8k4"):
// with g = lane / 4 and t = lane % 4,
//   A (16x4, row): a0 = A[g][t], a1 = A[g+8][t]
//   B (4x8, col):  b0 = B[t][g]
//   C (16x8):      c0, c1 = C[g][2t], C[g][2t+1];  c2, c3 = C[g+8][2t], C[g+8][2t+1]
__device__ __forceinline__ void dmma_16x8x4(double (&c)[4], double a0, double a1, double b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a0), "d"(a1), "d"(b0));
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int src_bytes = valid ? 8 : 0;  // 0: zero-fill, global not read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Shared-memory footprint (doubles) of one DMMA tile variant.
template <int WARPS_M, int WARPS_N, int WT_M, int WT_N>
struct DmmaShape {
    static constexpr int NT = 32 * WARPS_M * WARPS_N;
    static constexpr int BM = WARPS_M * WT_M, BN = WARPS_N * WT_N, BK = 8;
    // Row pitches chosen so each half-warp's fragment reads hit distinct banks.
    static constexpr int LDA_S = BK + 4;
    static constexpr int LDB_S = BN + 4;
    static constexpr int STAGES = (BM >= 128) ? 2 : 3;  // <= 48 KB static smem
    static constexpr int A_STAGE = BM * LDA_S, B_STAGE = BK * LDB_S;
    static constexpr int SMEM_DOUBLES = STAGES * (A_STAGE + B_STAGE);
};

// One BM x BN tile of C at (row0, col0) on the FP64 tensor pipe; `smem` holds
// DmmaShape::SMEM_DOUBLES doubles (16-byte aligned).  All threads of the block call it.
template <int WARPS_M, int WARPS_N, int WT_M, int WT_N>
__device__ __forceinline__ void dmma_tile(int64_t m, int64_t n, int64_t k, double alpha,
                                          const double* __restrict__ A, int64_t lda,
                                          const double* __restrict__ B, int64_t ldb,
                                          double beta, double* __restrict__ C, int64_t ldc,
                                          int64_t row0, int64_t col0, double* smem) {
    using S = DmmaShape<WARPS_M, WARPS_N, WT_M, WT_N>;
    constexpr int NT = S::NT, BM = S::BM, BN = S::BN, BK = S::BK;
    constexpr int MT = WT_M / 16, NTILE = WT_N / 8;
    constexpr int LDA_S = S::LDA_S, LDB_S = S::LDB_S, STAGES = S::STAGES;
    double* As = smem;
    double* Bs = smem + STAGES * S::A_STAGE;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp / WARPS_N, wn = warp % WARPS_N;
    const int g = lane >> 2, t = lane & 3;
    const int64_t nk = (k + BK - 1) / BK;

    auto issue = [&](int stage, int64_t kt) {
        const int64_t l0 = kt * BK;
        double* as = As + stage * S::A_STAGE;
        double* bs = Bs + stage * S::B_STAGE;
        for (int e = tid; e < BM * BK; e += NT) {
            const int r = e / BK, l = e % BK;
            const int64_t gi = row0 + r, gl = l0 + l;
            const bool ok = gi < m && gl < k;
            cp_async8(&as[r * LDA_S + l], ok ? &A[gi * lda + gl] : A, ok);
        }
        for (int e = tid; e < BK * BN; e += NT) {
            const int l = e / BN, c = e % BN;
            const int64_t gl = l0 + l, gj = col0 + c;
            const bool ok = gl < k && gj < n;
            cp_async8(&bs[l * LDB_S + c], ok ? &B[gl * ldb + gj] : B, ok);
        }
    };

    double acc[MT][NTILE][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NTILE; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0;

    // prologue: STAGES-1 tiles in flight
#pragma unroll
    for (int st = 0; st < STAGES - 1; ++st) {
        if (st < nk) issue(st, st);
        cp_async_commit();
    }
    for (int64_t kt = 0; kt < nk; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int64_t nxt = kt + STAGES - 1;
        if (nxt < nk) issue((int)(nxt % STAGES), nxt);
        cp_async_commit();
        const double* as = As + (kt % STAGES) * S::A_STAGE;
        const double* bs = Bs + (kt % STAGES) * S::B_STAGE;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double af[MT][2], bf[NTILE];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const int r = wm * WT_M + i * 16 + g;
                af[i][0] = as[r * LDA_S + kk + t];
                af[i][1] = as[(r + 8) * LDA_S + kk + t];
            }
#pragma unroll
            for (int j = 0; j < NTILE; ++j) bf[j] = bs[(kk + t) * LDB_S + wn * WT_N + j * 8 + g];
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int j = 0; j < NTILE; ++j) dmma_16x8x4(acc[i][j], af[i][0], af[i][1], bf[j]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();  // the shared-memory stages may be reused by the caller's next tile

    const bool beta0 = beta == 0.0;
#pragma unroll
    for (int i = 0; i < MT; ++i) {
#pragma unroll
        for (int j = 0; j < NTILE; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t gi = row0 + wm * WT_M + i * 16 + g + 8 * h;
                if (gi >= m) continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int64_t gj = col0 + wn * WT_N + j * 8 + 2 * t + q;
                    if (gj >= n) continue;
                    double* c = &C[gi * ldc + gj];
                    const double v = acc[i][j][2 * h + q];
                    *c = beta0 ? alpha * v : alpha * v + beta * (*c);
                }
            }
        }
    }
}

template <int WARPS_M, int WARPS_N, int WT_M, int WT_N>
__global__ void __launch_bounds__(32 * WARPS_M * WARPS_N)
    dmma_kernel(int64_t m, int64_t n, int64_t k, double alpha, const double* __restrict__ A,
                int64_t lda, const double* __restrict__ B, int64_t ldb, double beta,
                double* __restrict__ C, int64_t ldc) {
    using S = DmmaShape<WARPS_M, WARPS_N, WT_M, WT_N>;
    __shared__ __align__(16) double smem[S::SMEM_DOUBLES];
    dmma_tile<WARPS_M, WARPS_N, WT_M, WT_N>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                            blockIdx.y * (int64_t)S::BM,
                                            blockIdx.x * (int64_t)S::BN, smem);
}

// ---- grouped: persistent CTAs over the tiles of many problems ----------------------
// Each CTA repeatedly takes the next tile index from a global counter (so tiles
// of expensive problems, placed first in the table, start first), finds its
// problem by binary search over the tile prefix, and runs that problem's tile
// variant on the FP64 FMA pipe.  One shared buffer serves every variant.
// Tiles use 32 x 8 threads (TX = 8): a warp covers 4 rows x 8 columns per part, so
// the ragged edges of small problems cost FMAs only up to that granularity.
constexpr int kGroupedTX = 8;
constexpr int kGroupedSmemDoubles = DfmaShape<2, 8, kGroupedTX>::SMEM_DOUBLES;
static_assert(DfmaShape<1, 4, kGroupedTX>::SMEM_DOUBLES <= kGroupedSmemDoubles, "smem");
static_assert(DfmaShape<2, 4, kGroupedTX>::SMEM_DOUBLES <= kGroupedSmemDoubles, "smem");
static_assert(DfmaShape<1, 8, kGroupedTX>::SMEM_DOUBLES <= kGroupedSmemDoubles, "smem");

__global__ void __launch_bounds__(256) grouped_native_kernel(const GroupProb* __restrict__ probs,
                                                             int nprob, int64_t total_tiles,
                                                             unsigned long long* counter) {
    __shared__ __align__(16) double smem[kGroupedSmemDoubles];
    __shared__ long long next_tile;
    for (;;) {
        if (threadIdx.x == 0) next_tile = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long t = next_tile;
        __syncthreads();
        if (t >= total_tiles) break;
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].first_tile <= t) lo = mid; else hi = mid - 1;
        }
        const GroupProb& P = probs[lo];
        const int64_t local = t - P.first_tile;
        const int64_t tm = local / P.tiles_n, tn = local % P.tiles_n;
        switch (P.tile) {
            case kTile64x64:
                dfma_tile<2, 8, kGroupedTX, true>(P.m, P.n, P.k, P.alpha, P.A, P.lda, P.B, P.ldb,
                                            P.beta, P.C, P.ldc, tm * 64, tn * 64, smem);
                break;
            case kTile32x32:
                dfma_tile<1, 4, kGroupedTX, true>(P.m, P.n, P.k, P.alpha, P.A, P.lda, P.B, P.ldb,
                                            P.beta, P.C, P.ldc, tm * 32, tn * 32, smem);
                break;
            case kTile64x32:
                dfma_tile<2, 4, kGroupedTX, true>(P.m, P.n, P.k, P.alpha, P.A, P.lda, P.B, P.ldb,
                                            P.beta, P.C, P.ldc, tm * 64, tn * 32, smem);
                break;
            default:
                dfma_tile<1, 8, kGroupedTX, true>(P.m, P.n, P.k, P.alpha, P.A, P.lda, P.B, P.ldb,
                                            P.beta, P.C, P.ldc, tm * 32, tn * 64, smem);
                break;
        }
    }
}

template <typename K>
cudaError_t finish(K) {
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scale(const Launch& L, const Gemm& g) {
    if (g.m == 0 || g.n == 0) return cudaSuccess;
    const int64_t total = g.m * g.n;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)L.sm_count * 8;
    if (blocks > cap) blocks = cap;
    scale_kernel<<<(unsigned)blocks, 256, 0, L.stream>>>(g.m, g.n, g.beta, g.C, g.ldc);
    return cudaGetLastError();
}

#define GB_ARGS g.m, g.n, g.k, g.alpha, g.A, g.lda, g.B, g.ldb, g.beta, g.C, g.ldc

cudaError_t launch_naive(const Launch& L, const Gemm& g, int by, int bx) {
    const dim3 block(bx, by);
    const dim3 grid((unsigned)((g.n + bx - 1) / bx), (unsigned)((g.m + by - 1) / by));
    if (g.beta == 0.0)
        naive_kernel<true><<<grid, block, 0, L.stream>>>(GB_ARGS);
    else
        naive_kernel<false><<<grid, block, 0, L.stream>>>(GB_ARGS);
    return cudaGetLastError();
}

template <int T>
static cudaError_t launch_tiled_t(const Launch& L, const Gemm& g) {
    const dim3 block(T, T);
    const dim3 grid((unsigned)((g.n + T - 1) / T), (unsigned)((g.m + T - 1) / T));
    if (g.beta == 0.0)
        tiled_kernel<T, true><<<grid, block, 0, L.stream>>>(GB_ARGS);
    else
        tiled_kernel<T, false><<<grid, block, 0, L.stream>>>(GB_ARGS);
    return cudaGetLastError();
}

cudaError_t launch_tiled(const Launch& L, const Gemm& g, int T) {
    switch (T) {
        case 8: return launch_tiled_t<8>(L, g);
        case 16: return launch_tiled_t<16>(L, g);
        case 32: return launch_tiled_t<32>(L, g);
        default: return cudaErrorInvalidValue;
    }
}

template <int V>
static cudaError_t launch_dfma_t(const Launch& L, const Gemm& g) {
    const int B = 16 * V;
    const dim3 grid((unsigned)((g.n + B - 1) / B), (unsigned)((g.m + B - 1) / B));
    dfma_kernel<V><<<grid, 256, 0, L.stream>>>(GB_ARGS);
    return cudaGetLastError();
}

cudaError_t launch_dfma(const Launch& L, const Gemm& g, int V) {
    switch (V) {
        case 2: return launch_dfma_t<2>(L, g);
        case 4: return launch_dfma_t<4>(L, g);
        case 8: return launch_dfma_t<8>(L, g);
        default: return cudaErrorInvalidValue;
    }
}

template <int WM, int WN, int TM, int TN>
static cudaError_t launch_dmma_t(const Launch& L, const Gemm& g) {
    const int BM = WM * TM, BN = WN * TN;
    const dim3 grid((unsigned)((g.n + BN - 1) / BN), (unsigned)((g.m + BM - 1) / BM));
    dmma_kernel<WM, WN, TM, TN><<<grid, 32 * WM * WN, 0, L.stream>>>(GB_ARGS);
    return cudaGetLastError();
}

bool dmma_variant_exists(int wm, int wn, int tm, int tn) {
    return (wm == 2 && wn == 2 && tm == 32 && tn == 32) ||
           (wm == 2 && wn == 2 && tm == 16 && tn == 16) ||
           (wm == 4 && wn == 2 && tm == 32 && tn == 32);
}

cudaError_t launch_dmma(const Launch& L, const Gemm& g, int wm, int wn, int tm, int tn) {
    if (wm == 2 && wn == 2 && tm == 32 && tn == 32) return launch_dmma_t<2, 2, 32, 32>(L, g);
    if (wm == 2 && wn == 2 && tm == 16 && tn == 16) return launch_dmma_t<2, 2, 16, 16>(L, g);
    if (wm == 4 && wn == 2 && tm == 32 && tn == 32) return launch_dmma_t<4, 2, 32, 32>(L, g);
    return cudaErrorInvalidValue;
}

const void* native_kernel_handle(const char* name) {
    struct Entry {
        const char* name;
        const void* fn;
    };
    static const Entry table[] = {
        {"dgemm_naive", reinterpret_cast<const void*>(&naive_kernel<false>)},
        {"dgemm_tiled16", reinterpret_cast<const void*>(&tiled_kernel<16, false>)},
        {"dgemm_dfma4", reinterpret_cast<const void*>(&dfma_kernel<4>)},
    };
    for (const Entry& e : table)
        if (name && !std::strcmp(name, e.name)) return e.fn;
    return nullptr;
}

int grouped_native_occupancy() {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, grouped_native_kernel, 256, 0) !=
            cudaSuccess ||
        blocks < 1)
        blocks = 1;
    return blocks;
}

cudaError_t launch_grouped_native(const Launch& L, const GroupProb* probs, int nprob,
                                  int64_t total_tiles, unsigned long long* counter, int grid) {
    if (nprob == 0 || total_tiles == 0) return cudaSuccess;
    grouped_native_kernel<<<grid, 256, 0, L.stream>>>(probs, nprob, total_tiles, counter);
    return cudaGetLastError();
}

}  // namespace gb
