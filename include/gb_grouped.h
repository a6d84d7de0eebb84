/*
 * gb_grouped.h -- many independent FP64 GEMMs in one launch (C ABI).
 *
 * Each problem is the DGEMM of Section 4.2, C_i <- alpha_i A_i B_i + beta_i C_i,
 * with the conventions and accuracy contract of gb_gemm.h.  The grid level of
 * the work division (Section 3.2) becomes persistent: a fixed grid of CTAs
 * (SM count x resident CTAs per SM) takes tiles of all problems from a device
 * counter, expensive tiles first; emulated problems run each split-precision
 * step in one launch per distinct slice count (three launches per slice count:
 * the split of A's rows, the column maxima and split of B's columns, the
 * products).  A plan records the launches in a CUDA graph once and replays it,
 * the two splits as parallel branches.
 *
 * Ownership: descriptors are read during the call only; A, B, C and the
 * workspace are the caller's device buffers and must stay valid while a plan
 * that uses them exists.  Problems of one call must not write overlapping C.
 */
#ifndef GB_GROUPED_H
#define GB_GROUPED_H

#include "gb_gemm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Tile variants.  Native problems: the grouped kernel's tiles (rows x columns
 * of C per CTA, 256 threads with 4 x 4, 2 x 2, 4 x 2 or 2 x 4 elements each on
 * the FP64 FMA pipe).  Emulated problems: the orientation of the 128 x
 * emu_bn(s) product tiles -- A's rows on the 128-line side, or B's columns
 * there (the problem runs as C^T = B^T A^T); the result is the same bit for
 * bit, only the padding and the tile count differ. */
typedef enum {
    GB_TILE_AUTO = 0,   /* from the tuning table (gb_tune_set), else a size rule */
    GB_TILE_64x64 = 1,
    GB_TILE_32x32 = 2,
    GB_TILE_64x32 = 3,
    GB_TILE_32x64 = 4,
    GB_TILE_EMU_ROWS = 5, /* emulated: A's rows on the 128-line side */
    GB_TILE_EMU_COLS = 6  /* emulated: B's columns on the 128-line side */
} gb_tile;

/* One GEMM of a group: layout and conventions of gb_dgemm. */
typedef struct {
    int64_t m, n, k;
    double alpha, beta;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
    int32_t precision; /* gb_precision */
    int32_t slices;    /* emulated: 1..16, 0 = the tuning table's slice count for
                          this shape (gb_tune_lookup_slices), else 11 */
    int32_t tile;      /* native: GB_TILE_AUTO .. GB_TILE_32x64; emulated: GB_TILE_AUTO,
                          GB_TILE_EMU_ROWS or GB_TILE_EMU_COLS */
    int32_t reserved;  /* must be 0 */
} gb_gemm_desc;

typedef struct gb_grouped_plan gb_grouped_plan;

/* Device workspace bytes a group needs (problem tables, tile counter and the
 * emulated problems' digit planes). */
gb_status gb_grouped_workspace_size(const gb_gemm_desc* descs, int64_t count, size_t* out);

/* Validate the group, build its tables in `workspace` (256-byte aligned, at
 * least gb_grouped_workspace_size bytes) and, with use_graph != 0, capture its
 * launches (counter reset, persistent native kernel, emulated split and
 * product launches) in a CUDA graph.  Blocks until the tables are on the device. */
gb_status gb_grouped_plan_create(gb_queue* q, const gb_gemm_desc* descs, int64_t count,
                                 void* workspace, size_t workspace_bytes, int use_graph,
                                 gb_grouped_plan** out);

/* Enqueue one execution of the plan on its queue (one graph launch). */
gb_status gb_grouped_plan_run(gb_grouped_plan* plan);

/* Tiles of the native and emulated parts, kernel launches per run, and the
 * useful FP64 flops 2 m n k summed over the problems. */
gb_status gb_grouped_plan_info(const gb_grouped_plan* plan, int64_t* native_tiles,
                               int64_t* emulated_tiles, int* launches, double* flops);

gb_status gb_grouped_plan_destroy(gb_grouped_plan* plan);

/* Create a plan without a graph, run it once and destroy it. */
gb_status gb_dgemm_grouped(gb_queue* q, const gb_gemm_desc* descs, int64_t count,
                           void* workspace, size_t workspace_bytes);

/* Tuning table of the grouped kernels: for a problem with tile == GB_TILE_AUTO
 * the first entry of its own kind (tile 1..4 for native problems, 5..6 for
 * emulated ones) with m <= m_max, n <= n_max and k <= k_max gives its tile or
 * orientation.  Written by the autotuner; no matching entry = the size rule
 * (native) or the padding rule (emulated: the orientation with fewer padded
 * output slots).  A third kind, tile = GB_TUNE_SLICES + s (s = 1..16), gives an
 * emulated problem with slices = 0 its slice count: the autotuner picks, per size
 * cell, the fastest count whose error on its tuning batches stays a safe margin
 * inside the FP64 bound of gb_gemm.h (a caller whose data spans a wider dynamic
 * range than uniform[-1, 1] passes its own count); no matching entry = 11.
 * GB_ERR_INVALID_ARG for any other tile. */
#define GB_TUNE_SLICES 100
typedef struct {
    int32_t m_max, n_max, k_max;
    int32_t tile;
} gb_tune_entry;

gb_status gb_tune_set(const gb_tune_entry* entries, int64_t count);
gb_status gb_tune_get(gb_tune_entry* entries, int64_t capacity, int64_t* count);

/* The tile a native problem of this shape would get (GB_TILE_AUTO resolved). */
gb_status gb_tune_lookup(int64_t m, int64_t n, int64_t k, int32_t* tile);

/* The orientation (GB_TILE_EMU_ROWS or GB_TILE_EMU_COLS) an emulated problem of
 * this shape and slice count (1..16, 0 = the table's, see gb_tune_lookup_slices)
 * would get with GB_TILE_AUTO.  Host only. */
gb_status gb_tune_lookup_emulated(int slices, int64_t m, int64_t n, int64_t k, int32_t* tile);

/* The slice count an emulated problem of this shape submitted with slices = 0
 * gets: the first matching slice-count entry (GB_TUNE_SLICES + s), else 11.
 * Host only. */
gb_status gb_tune_lookup_slices(int64_t m, int64_t n, int64_t k, int32_t* slices);

#ifdef __cplusplus
}
#endif

#endif /* GB_GROUPED_H */
