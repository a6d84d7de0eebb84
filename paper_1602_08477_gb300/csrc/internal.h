// Internal launcher interface between the C ABI (api.cpp) and the kernels.
// Not installed; the public interface is include/gb_gemm.h.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace gb {

// Bits of the per-queue device status word.
enum : unsigned {
    kStatusTimeout = 1u,    // a bounded device-side wait gave up
    kStatusNonfinite = 2u,  // the emulated path saw NaN/Inf input
};

struct Launch {
    cudaStream_t stream;
    unsigned* status;  // device status word (may be null)
    int sm_count;
};

struct Gemm {
    int64_t m, n, k;
    double alpha, beta;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
};

// ---- native FP64 kernels (dgemm_native.cu) ----
// C <- beta * C (alpha == 0 or k == 0).
cudaError_t launch_scale(const Launch& L, const Gemm& g);
// One thread per element; block by x bx threads (rows x cols).
cudaError_t launch_naive(const Launch& L, const Gemm& g, int by, int bx);
// Square shared-memory tiles of T x T (T in {8, 16, 32}), one element per thread.
cudaError_t launch_tiled(const Launch& L, const Gemm& g, int T);
// Register-tiled FP64 FMA: 16 x 16 threads with V x V elements (V in {2, 4, 8}).
cudaError_t launch_dfma(const Launch& L, const Gemm& g, int V);
// Warp-tiled DMMA: warps_m x warps_n warps, each wt_m x wt_n elements
// (supported: (2,2,32,32), (2,2,16,16), (4,2,32,32)).
cudaError_t launch_dmma(const Launch& L, const Gemm& g, int warps_m, int warps_n, int wt_m,
                        int wt_n);
bool dmma_variant_exists(int warps_m, int warps_n, int wt_m, int wt_n);

// ---- grouped native FP64 (dgemm_native.cu) ----
// Tile variants of the grouped kernel (256 threads on the FP64 FMA pipe): BM x BN.
enum : int { kTile64x64 = 1, kTile32x32 = 2, kTile64x32 = 3, kTile32x64 = 4 };
inline int tile_bm(int v) { return (v == kTile64x64 || v == kTile64x32) ? 64 : 32; }
inline int tile_bn(int v) { return (v == kTile64x64 || v == kTile32x64) ? 64 : 32; }

// One problem of a grouped launch, as the device reads it.
struct GroupProb {
    int64_t m, n, k, lda, ldb, ldc;
    const double* A;
    const double* B;
    double* C;
    double alpha, beta;
    int32_t tile, tiles_n;
    int64_t first_tile;  // exclusive prefix of tile counts over the table
};

// Persistent kernel over `total_tiles` tiles of `nprob` problems; CTAs take
// tiles from *counter (zeroed by the caller) in table order.  `grid` CTAs.
cudaError_t launch_grouped_native(const Launch& L, const GroupProb* probs, int nprob,
                                  int64_t total_tiles, unsigned long long* counter, int grid);
// Host handle of a native DGEMM kernel by name ("dgemm_naive", "dgemm_tiled16",
// "dgemm_dfma4"; parameters m, n, k, alpha, A, lda, B, ldb, beta, C, ldc), or null.
const void* native_kernel_handle(const char* name);
// Resident 256-thread CTAs per SM of the grouped native kernel.
int grouped_native_occupancy();

// ---- emulated FP64 (ozaki_split.cu, ozaki_gemm.cu) ----
// Workspace of the emulated path.  Digits are stored pre-tiled: for each tile of
// R rows (R = 128 for A's rows, emu_bn(s) for B's columns) and each 32-byte K block,
// the s slices follow one another, each an R x 32-byte K-major block in the
// 32-byte swizzle (16-byte chunk c of row r stored at chunk c ^ ((r / 4) & 1)),
// i.e. exactly the shared-memory image the tensor core reads:
//   byte of digit t of line x at column l:
//     ((x / R) * nkb + l / 32) * s + t) * (R * 32) + (x % R) * 32
//     + (((l % 32) / 16) ^ (((x % R) / 4) & 1)) * 16 + l % 16,   nkb = kp / 32.
// Lines are padded to multiples of R (zero digits); columns to kp (zero digits).
// After the exponents: b_part, scratch for the partial column maxima of B
// (kColmaxParts x n uint64, see launch_split_cols).
struct EmuLayout {
    int64_t kp;
    size_t a_digits, b_digits, a_exp, b_exp, b_part, total;
    int bn;  // lines of a B digit tile = output tile columns, emu_bn(s)
};
constexpr int kColmaxParts = 16;  // K ranges of the column maxima of one launch, at most
EmuLayout emu_layout(int s, int64_t m, int64_t n, int64_t k, bool colmax_scratch = true);

// A grouped emulated problem is computed as C^T = B^T A^T (B's columns on the
// 128-row side of the output tiles, A's rows on the emu_bn(s)-column side) when
// that pads fewer tile slots: pad(n, 128) pad(m, bn) < pad(m, 128) pad(n, bn).
bool emu_group_trans(int s, int64_t m, int64_t n);
// Workspace layout of one grouped emulated problem: emu_layout(s, m, n, k), or for
// a transposed problem (trans) emu_layout(s, n, m, k) with the roles swapped (its a_*
// regions hold B's column digits and exponents, its b_* regions A's rows'); no
// b_part scratch (the grouped column maxima need none).
EmuLayout emu_group_layout(int s, int64_t m, int64_t n, int64_t k, bool trans);

// One emulated problem of a grouped launch, as the device reads it.
struct EmuProb {
    int64_t m, n, k, lda, ldb, ldc, kp;
    const double* A;
    const double* B;
    double* C;
    double alpha, beta;
    uint8_t* a_digits;  // digit tiles of A's rows (ra lines per tile)
    uint8_t* b_digits;  // digit tiles of B's columns (rb lines per tile)
    int32_t* a_exp;
    int32_t* b_exp;
    int32_t s, tiles_n;
    int32_t trans;   // computed as C^T = B^T A^T: B's columns on the 128-row side
    int32_t ra, rb;  // tile lines of A's and B's digits: 128 and emu_bn(s), swapped if trans
    int32_t pad_;
    int64_t first_row;     // exclusive prefixes over the table of: rows of A padded to 128,
    int64_t first_colblk;  // 32-column strips of B's columns padded to whole tiles,
    int64_t first_tile;    // 128 x emu_bn(s) output tiles
};

// Points the digit and exponent fields of `e` (m, n, s, trans set) into the
// problem's workspace at `base`, laid out as emu_group_layout.
void emu_group_assign(EmuProb& e, uint8_t* base, const EmuLayout& w);

// The same four prefixes as compact arrays (one int64 per table entry), the
// keys of the device-side binary searches: a search touches a few cache lines
// instead of one EmuProb per probe.
struct EmuKeys {
    const int64_t* row;
    const int64_t* colblk;
    const int64_t* tile;
};
constexpr int kEmuKeys = 3;  // prefix arrays in EmuKeys

// The emulated problems of one slice count s occupy consecutive table entries;
// their rows, column strips and output tiles are the ranges
// [*_begin, *_end) of the table's prefixes.
struct EmuSRange {
    int s;
    int q_begin, q_end;  // table entries
    int64_t row_begin, row_end;
    int64_t cb_begin, cb_end;
    int64_t t_begin, t_end;
    int64_t kp_max;  // longest padded K of the range's problems
};

// A second stream and two events for running the split of A beside that of B:
// the A rows go to `side` after `fork` is recorded on the launch stream, which
// waits for `join` (recorded on `side` after them) before the products.
struct SplitFork {
    cudaStream_t side;
    cudaEvent_t fork, join;
};

// Grouped e1 + e2 over the problems of one slice-count range (three launches;
// with `fk`, the split of A on fk->side beside the two launches for B).
cudaError_t launch_grouped_split(const Launch& L, const EmuProb* probs, const EmuKeys& keys,
                                 const EmuSRange& r, const SplitFork* fk = nullptr);
// Grouped e3 + e4: persistent CTAs over the 128 x emu_bn(s) output tiles of the
// problems of one slice-count range.
cudaError_t launch_grouped_products(const Launch& L, const EmuProb* probs, const EmuKeys& keys,
                                    const EmuSRange& r);
constexpr int kEmuBM = 128;  // output tile rows of the products kernel (A digit tile rows)
// Output tile columns of the products kernel (= lines of a B digit tile) for s
// slices: the s level accumulators of a tile take s * BN of the 512 TMEM columns,
// and a wider tile reuses each staged A slice for more outputs, so BN = 48 while
// 48 s <= 512 (s <= 10) and 32 above.
__host__ __device__ constexpr int emu_bn(int s) { return s <= 10 ? 48 : 32; }

// ---- emulated FP64 by residue arithmetic (ozaki_crt.cu) ----
// Integers of b bits per line, multiplied modulo N primes (BF16 residues,
// kind::f16 MMAs into FP32 sums of at most 256 K), recovered by the Chinese
// remainder theorem and rounded once.
constexpr int kCrtMaxModuli = 14;      // the product of the moduli stays below 2^125
constexpr int kCrtDefaultModuli = 13;
struct CrtLayout {
    int N;       // moduli
    int b;       // bits of the scaled integers (0: k too long for N moduli)
    int64_t kp, mp, np;  // K padded to 16, m and n padded to 128
    size_t a_res, b_res, c_res, a_exp, b_exp, b_part, total;
};
// The largest b in [1, 62] with 4 k 2^(2b) <= M (M the product of the first N
// moduli), 0 when none.
int crt_scale_bits(int N, int64_t k);
CrtLayout crt_layout(int N, int64_t m, int64_t n, int64_t k);
// Split of A and B, residue products, reconstruction (m, n > 0, k > 0, alpha != 0).
cudaError_t launch_crt_gemm(const Launch& L, const Gemm& g, uint8_t* ws, const CrtLayout& lay);
// The steps one at a time, for a band of rows of A (whole 128-row tiles of the
// full layout: its residues start band_row0 N kp 2 bytes into the A residues) or a
// block of columns of B (whole 256-column tiles: band_col0 N kp 2 bytes in):
// residues and exponents of A's rows / B's columns; the products of the tiles of
// A (m rows) and B (n columns) given, their residues in cres (2 N pad(m, 128)
// pad(n, 256) bytes) and the reconstruction into C.
constexpr int kCrtTileRows = 128;  // row edges of bands of A
constexpr int kCrtTileCols = 256;  // column edges of blocks of B
cudaError_t crt_split_a(const Launch& L, int N, int b, int64_t m, int64_t k, const double* A,
                        int64_t lda, uint8_t* ares, int64_t kp, int32_t* ea);
cudaError_t crt_split_b(const Launch& L, int N, int b, int64_t n, int64_t k, const double* B,
                        int64_t ldb, uint8_t* bres, int64_t kp, int32_t* fb, uint64_t* part);
cudaError_t crt_products(const Launch& L, int N, int b, int64_t m, int64_t n, int64_t kp,
                         double alpha, double beta, double* C, int64_t ldc, const uint8_t* ares,
                         const uint8_t* bres, int16_t* cres, const int32_t* ea,
                         const int32_t* fb);
// crt_products in its two launches: the residue products, the reconstruction.
cudaError_t crt_residue_products(const Launch& L, int N, int64_t m, int64_t n, int64_t kp,
                                 const uint8_t* ares, const uint8_t* bres, int16_t* cres);
cudaError_t crt_combine(const Launch& L, int N, int b, int64_t m, int64_t n, double alpha,
                        double beta, double* C, int64_t ldc, const int16_t* cres,
                        const int32_t* ea, const int32_t* fb);

// ---- emulated FP64 with BF16 digits (ozaki_bf16.cu) ----
// 8-bit signed digits (|d| <= 128) in BF16, kind::f16 MMAs.  Output tiles of
// 128 x kBf16BN; digits stored pre-tiled as for E4M3 with 16 digits (32 bytes)
// per K block, so K is padded to a multiple of 16:
//   byte of digit t of line x at K index l (nks = kp / 16, c = 2 (l % 16)):
//     ((x / R) * nks + l / 16) * s + t) * (R * 32) + (x % R) * 32
//     + ((c / 16) ^ (((x % R) / 4) & 1)) * 16 + c % 16,   R = 128 (A) or 32 (B).
constexpr int kBf16BN = 32;
constexpr int kBf16MaxSlices = 8;          // two sets of 8 levels x 32 columns fill TMEM
constexpr int64_t kBf16MaxK = (int64_t)1 << 22;  // the epilogue's int64 sums stay exact
EmuLayout emu_layout_bf16(int s, int64_t m, int64_t n, int64_t k);
cudaError_t launch_bf16_split_rows(const Launch& L, int s, int64_t m, int64_t k, const double* A,
                                   int64_t lda, uint8_t* digits, int64_t kp, int32_t* exps);
cudaError_t launch_bf16_split_cols(const Launch& L, int s, int64_t n, int64_t k, const double* B,
                                   int64_t ldb, uint8_t* digits, int64_t kp, int32_t* exps,
                                   uint64_t* part);
cudaError_t launch_bf16_products(const Launch& L, int s, int64_t m, int64_t n, double alpha,
                                 double beta, double* C, int64_t ldc, const uint8_t* a_digits,
                                 const uint8_t* b_digits, int64_t kp, const int32_t* a_exp,
                                 const int32_t* b_exp);


// First half of e1 for the columns of B: partial column maxima over *ks_out (at
// most kColmaxParts) K ranges into `part` (ks_out x n uint64): the largest
// absolute bit pattern of each range, bit 63 alone for a range with NaN or Inf.
cudaError_t launch_colmax_part(const Launch& L, int64_t n, int64_t k, const double* B,
                               int64_t ldb, uint64_t* part, int* ks_out);

cudaError_t launch_split_rows(const Launch& L, int s, int64_t m, int64_t k, const double* A,
                              int64_t lda, uint8_t* digits, int64_t kp, int32_t* exps);
// e1 + e2 for the columns of B: partial column maxima over up to kColmaxParts K
// ranges into `part` (kColmaxParts x n uint64 of scratch), then exponents and digits.
cudaError_t launch_split_cols(const Launch& L, int s, int64_t n, int64_t k, const double* B,
                              int64_t ldb, uint8_t* digits, int64_t kp, int32_t* exps,
                              uint64_t* part);
cudaError_t launch_emu_products(const Launch& L, int s, int64_t m, int64_t n, int64_t k,
                                double alpha, double beta, double* C, int64_t ldc,
                                const uint8_t* a_digits, const uint8_t* b_digits, int64_t kp,
                                const int32_t* a_exp, const int32_t* b_exp);

// Last error text helper used by launchers (thread-local in api.cu).
void set_error(const char* fmt, ...);

// Host-side validation of a GEMM's sizes, leading dimensions and pointers;
// returns a gb_status value (0 = OK) and sets the error text.
int validate_gemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, const double* C, int64_t ldc);

}  // namespace gb
