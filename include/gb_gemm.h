/*
 * gb_gemm.h -- C ABI of a GB300 (sm_103a) FP64 GEMM library built on the
 * grid / block / thread / element work-division model of Alpaka
 * (arXiv 1602.08477, Section 3.2 "Model of Parallel Abstraction").
 *
 * The one operation is the DGEMM of Section 4.2:   C <- alpha * A * B + beta * C
 * over caller-owned, row-major device buffers with leading dimensions ("pitched"
 * rows, Section 3.4.4):
 *     A is m x k, element (i, l) at A[i * lda + l], lda >= max(1, k)
 *     B is k x n, element (l, j) at B[l * ldb + j], ldb >= max(1, n)
 *     C is m x n, element (i, j) at C[i * ldc + j], ldc >= max(1, n)
 * All pointers are device pointers of the queue's device, 8-byte aligned.
 *
 * Conventions where the paper is silent (BLAS):
 *   beta == 0            : C is not read (NaN/Inf in C do not propagate).
 *   alpha == 0 or k == 0 : C <- beta * C and A, B are not read (may be NULL).
 *   m == 0 or n == 0     : nothing is enqueued; GB_OK.
 *
 * Accuracy contract (both precisions): |C - C*|_ij <= 2 (k + 2) 2^-53
 * (|alpha| (|A||B|)_ij + |beta| |C_ij|), where C* is the exact result; on integer
 * inputs whose partial sums are exact in FP64 the result is exact.  The emulated
 * precision meets it when enough slices are used for the data's dynamic range.
 *
 * Ownership: the caller owns every A, B, C and workspace buffer; the library
 * never frees a caller pointer.  The library owns the opaque handles and frees
 * them in the matching *_destroy / *_release call.  A queue wraps a caller
 * cudaStream_t and never destroys it.
 *
 * Errors: every call returns gb_status and never aborts or throws across the
 * ABI.  Argument errors are found on the host before anything is enqueued.
 * gb_last_error() returns a message for the calling thread's last failure.
 * Errors found on the device (a bounded device-side wait that gave up; a
 * non-finite input to the emulated path) are recorded in the queue's status
 * word and returned by gb_queue_wait().
 *
 * Asynchrony (Section 3.4.5, "Streams"): operations on a queue run in order.
 * On a non-blocking queue every call returns once its work is enqueued; on a
 * blocking queue it returns after the work has finished, with the device
 * status of that work.
 */
#ifndef GB_GEMM_H
#define GB_GEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GB_OK = 0,
    GB_ERR_INVALID_ARG = 1,      /* a size, pointer, leading dimension or option is invalid */
    GB_ERR_INVALID_WORKDIV = 2,  /* the work division does not cover C or no variant has it */
    GB_ERR_UNSUPPORTED = 3,      /* valid request the library does not implement */
    GB_ERR_NO_DEVICE = 4,        /* no CUDA device, or index out of range */
    GB_ERR_CUDA = 5,             /* a CUDA runtime call failed (message in gb_last_error) */
    GB_ERR_OUT_OF_BUDGET = 6,    /* a serving request can never fit the HBM budget */
    GB_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up */
    GB_ERR_NONFINITE = 8,        /* the emulated path saw NaN/Inf input (outputs set to NaN) */
    GB_ERR_BUSY = 9,             /* the handle is in use (e.g. a server still has requests) */
    GB_ERR_WORKSPACE = 10        /* workspace missing, too small or misaligned */
} gb_status;

/* Opaque handles. */
typedef struct gb_device gb_device;
typedef struct gb_queue gb_queue;
typedef struct gb_server gb_server;

/*
 * Work division (Section 3.4.3, "Work Division and Index Retrieval"): the
 * extents of the grid (blocks per grid), block (threads per block) and thread
 * (elements per thread) levels, per dimension.  For the GEMM, dim == 2,
 * dimension 0 runs over the rows of C (m) and dimension 1 over its columns
 * (n); linearisation is row-major.  The CUDA mapping of Table 2 applies per
 * dimension: blocks = N / (B * V), threads = B, elements = V.  For the
 * tensor-pipe kernel one work-division "thread" is one warp and its elements
 * are that warp's register tile.  A work division must cover C:
 * grid_blocks[d] * block_threads[d] * thread_elems[d] >= extent[d].
 */
typedef struct {
    uint32_t dim;
    uint64_t grid_blocks[3];
    uint64_t block_threads[3];
    uint64_t thread_elems[3];
} gb_workdiv;

typedef enum {
    GB_PREC_NATIVE = 0,        /* FP64 arithmetic on the FP64 pipes */
    GB_PREC_EMULATED = 1,      /* FP64 result from E4M3 slices on the tcgen05 tensor cores */
    GB_PREC_EMULATED_BF16 = 2, /* the same from BF16 slices (8-bit digits, kind::f16 MMAs) */
    GB_PREC_EMULATED_CRT = 3   /* the same from integer residues modulo N primes (kind::f16) */
} gb_precision;

typedef enum {
    GB_KERNEL_AUTO = 0,    /* library choice (native: the fastest compiled variant) */
    GB_KERNEL_NAIVE = 1,   /* one thread per element of C, operands read from global memory */
    GB_KERNEL_TILED = 2,   /* square shared-memory tiles, one element per thread */
    GB_KERNEL_DFMA = 3,    /* hierarchical tiles, V x V elements per thread on the FP64 FMA pipe */
    GB_KERNEL_DMMA = 4     /* hierarchical tiles, warp tiles on FP64 mma.sync (DMMA) */
} gb_kernel;

/* Library version as major * 10000 + minor * 100 + patch. */
int gb_version(void);

/* Message for the calling thread's most recent failed call ("" if none).
 * The pointer stays valid until the next library call on this thread. */
const char* gb_last_error(void);

/* ---- Devices (Section 3.4.6, Listing "kernel": DevMan<Acc>::getDevByIdx) ---- */

/* Number of CUDA devices. GB_ERR_NO_DEVICE with *n = 0 when there is none. */
gb_status gb_device_count(int* n);

/* Handle of device `idx` (0-based). No device becomes implicitly current
 * (Section 3.1: no default device or stream). Free with gb_device_release. */
gb_status gb_device_get(int idx, gb_device** out);

/* Streaming multiprocessor count and compute capability of a device. */
gb_status gb_device_info(const gb_device* dev, int* sm_count, int* cc_major, int* cc_minor);

gb_status gb_device_release(gb_device* dev);

/* ---- Queues (Section 3.4.5, "Streams") ----------------------------------------- */

/* Wrap `cuda_stream` (a cudaStream_t of device `dev`, or NULL for the legacy
 * default stream) into a queue.  blocking != 0: every call on the queue waits
 * for its work (a synchronous stream); 0: calls return once enqueued.
 * The queue owns a small device status word; it never destroys the stream. */
gb_status gb_queue_create(gb_device* dev, void* cuda_stream, int blocking, gb_queue** out);

/* Wait for all work enqueued so far; return the first device-side error
 * recorded since the last wait (GB_ERR_TIMEOUT, GB_ERR_NONFINITE) and clear it. */
gb_status gb_queue_wait(gb_queue* q);

/* The wrapped stream (a cudaStream_t). */
void* gb_queue_stream(const gb_queue* q);

gb_status gb_queue_destroy(gb_queue* q);

/* ---- Work division ------------------------------------------------------------- */

/* The work division the library would use for `kernel` on an m x n x k GEMM
 * (the CUDA row of Table 2 with the variant's compiled B and V).  For
 * GB_KERNEL_AUTO the chosen kernel is returned in *chosen (may be NULL). */
gb_status gb_workdiv_suggest(const gb_device* dev, gb_kernel kernel, int64_t m, int64_t n,
                             int64_t k, gb_workdiv* out, gb_kernel* chosen);

/* ---- The GEMM (Section 4.2) --------------------------------------------------- */

/*
 * C <- alpha * A * B + beta * C, enqueued on q (executor "create + enqueue",
 * Section 3.4.6).
 *   wd        work division, or NULL for the library's choice.  Native only;
 *             the emulated precision takes NULL.
 *   kernel    native variant (GB_KERNEL_AUTO for the library's choice).
 *   prec      GB_PREC_NATIVE, GB_PREC_EMULATED, GB_PREC_EMULATED_BF16 or
 *             GB_PREC_EMULATED_CRT.
 *   slices    emulated only: number s of digit slices per operand; E4M3:
 *             1 <= s <= 16 (the first slice carries 4 bits, each further one
 *             5; 0 selects the default of 11); BF16: 1 <= s <= 8 (7 bits, then
 *             8 each; 0 selects 7, which covers 55 bits of each row's and
 *             column's scale like 11 E4M3 slices; 8 covers 63, like 13 E4M3
 *             slices); ignored for native.
 *             BF16 digits: the same steps and rounding as E4M3 digits with
 *             digits |d| <= 128 (b1 = 7, b = 8), the level sums read out of the
 *             FP32 accumulators every 1024 / s K indices (each exact there) and
 *             summed exactly in integers; k <= 2^22 (larger k:
 *             GB_ERR_UNSUPPORTED).  gb_dgemm is its only entry point (the
 *             step-by-step, host-buffer, grouped, serving and no-allocation
 *             calls take E4M3 digits).  Its workspace holds, each part
 *             1024-byte aligned and in this order: A's digits (2 s mp kp bytes,
 *             mp = m rounded up to 128, kp = k rounded up to 16), B's digits
 *             (2 s np kp, np = n rounded up to 32), A's row exponents (m int32),
 *             B's column exponents (n int32), scratch; the digits are BF16 codes
 *             tiled as in the E4M3 layout below, with R = 128 (A) and 32 (B)
 *             lines per tile and 16 digits per 32-byte K block.
 *             Residues (GB_PREC_EMULATED_CRT; `slices` = N, the number of moduli,
 *             1 <= N <= 14, 0 selects 13): each row of A and column of B is scaled
 *             by a power of two to integers of b bits (round to nearest even; b
 *             the largest count with k 2^(2b) <= M / 4, M the product of the
 *             first N of the primes 509, 503, 499, 491, 487, 479, 467, 463, 461,
 *             457, 449, 443, 439, 433; GB_ERR_UNSUPPORTED when k is too long for
 *             b >= 1), the integer product is computed modulo each prime on the
 *             tensor cores (BF16 residues |r| <= 254, FP32 sums of at most 256 K,
 *             each exact) and recovered exactly by the Chinese remainder theorem,
 *             then rounded once: the only approximation is the scaling to b
 *             bits (13 moduli: b = 50 at k = 8192).  Entry points: gb_dgemm and
 *             gb_dgemm_host.  Workspace, each part 1024-byte aligned and in this
 *             order: A's residues (2 N mp kp bytes, mp = m rounded up to 128,
 *             kp = k rounded up to 16), B's residues (2 N np kp, np = n rounded
 *             up to 256), the residues of C (2 N mp np), A's row exponents (m
 *             int32), B's column exponents (n int32), scratch.
 *   workspace device buffer of at least gb_dgemm_workspace_size() bytes,
 *             256-byte aligned (emulated only; native takes NULL, 0).
 * Errors: GB_ERR_INVALID_ARG (sizes, pointers, leading dimensions, slices),
 * GB_ERR_INVALID_WORKDIV, GB_ERR_WORKSPACE, GB_ERR_CUDA; on a blocking queue
 * also the device status of this call (GB_ERR_NONFINITE, GB_ERR_TIMEOUT).
 */
gb_status gb_dgemm(gb_queue* q, const gb_workdiv* wd, gb_kernel kernel, gb_precision prec,
                   int slices, int64_t m, int64_t n, int64_t k, double alpha,
                   const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                   double* C, int64_t ldc, void* workspace, size_t workspace_bytes);

/* Workspace bytes gb_dgemm needs (0 for native; per emulated precision). */
gb_status gb_dgemm_workspace_size(gb_precision prec, int slices, int64_t m, int64_t n,
                                  int64_t k, size_t* out);

/*
 * Layout of the emulated path's workspace (all offsets in bytes from its
 * start, each 1024-byte aligned), for tests and for callers who run the steps
 * one at a time.  Digits are E4M3 bytes stored pre-tiled, in the order the
 * tensor-core products read them: lines (rows of A, columns of B) are grouped in
 * tiles of R lines (R = a_tile_rows = 128 for A, b_tile_rows for B: 48 when
 * slices <= 10, else 32), K in blocks of 32 bytes, and per (tile, K block) the
 * s slices follow one another, each an R x 32-byte K-major block whose 16-byte
 * halves are swapped on lines with ((line % R) / 4) odd (the 32-byte swizzle):
 *   digit t of line x at K index l (nkb = kp / 32, c = l % 32, r = x % R):
 *     base + (((x / R) * nkb + l / 32) * s + t) * R * 32 + r * 32
 *          + ((c / 16) ^ ((r / 4) & 1)) * 16 + c % 16
 *   a_digits  base of A's digits (line x = row i of A), rows padded to R
 *   b_digits  base of B's digits (line x = column j of B), columns padded to R
 *   a_exp     m int32: exponent e_i of max_l |A[i, l]| (frexp convention),
 *             GB_BAD_LINE if row i holds a NaN or Inf
 *   b_exp     n int32: exponent f_j of max_l |B[l, j]|, or GB_BAD_LINE
 * with kp = k rounded up to a multiple of 32; padding lines and K indices
 * l >= k hold zero digits.  After b_exp, `total` also covers 128 n bytes of
 * scratch for the partial column maxima of B (up to 16 K ranges per column).
 */
#define GB_BAD_LINE 0x40000000
typedef struct {
    int64_t kp;
    size_t a_digits, b_digits, a_exp, b_exp, total;
    int32_t a_tile_rows, b_tile_rows;
} gb_emulated_layout;

gb_status gb_emulated_layout_get(int slices, int64_t m, int64_t n, int64_t k,
                                 gb_emulated_layout* out);

/* Emulated step e1+e2 for A: exponents and E4M3 digit planes of the rows of A
 * (m x k, lda) into a workspace laid out as above. */
gb_status gb_emulated_split_a(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                              const double* A, int64_t lda, void* workspace,
                              size_t workspace_bytes);

/* Emulated step e1+e2 for B: exponents and transposed digit planes of the
 * columns of B (k x n, ldb). */
gb_status gb_emulated_split_b(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                              const double* B, int64_t ldb, void* workspace,
                              size_t workspace_bytes);

/* The residue precision (GB_PREC_EMULATED_CRT, `moduli` as its `slices`) one
 * step at a time, on a workspace laid out as gb_dgemm documents for it:
 *   step 0  scaled integers, residues and exponents of A's rows (m x k, lda);
 *   step 1  the same for B's columns (k x n, ldb);
 *   step 2  the residue products on the tensor cores, into the workspace's
 *           residues of C;
 *   step 3  the reconstruction, rounding and alpha / beta into C (m x n, ldc).
 * Steps 0 - 3 in order on one queue compute what gb_dgemm computes (alpha != 0,
 * k > 0); each step reads only the operands it names (the others may be NULL).
 * Errors as gb_dgemm; GB_ERR_INVALID_ARG for a step outside 0 - 3. */
gb_status gb_emulated_crt_step(gb_queue* q, int step, int moduli, int64_t m, int64_t n,
                               int64_t k, double alpha, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double beta, double* C,
                               int64_t ldc, void* workspace, size_t workspace_bytes);

/* Emulated steps e3+e4 from a workspace filled by the two split calls: the
 * slice-pair products on the tensor cores and the recombination into C. */
gb_status gb_emulated_products(gb_queue* q, int slices, int64_t m, int64_t n, int64_t k,
                               double alpha, double beta, double* C, int64_t ldc,
                               void* workspace, size_t workspace_bytes);

/*
 * C <- alpha A B + beta C (Section 4.2) with A, B and C in HOST memory, moved by
 * the explicit host <-> device copies of Section 3.4.4, enqueued by the library
 * and overlapped with the computation.  A (m x k, lda), B (k x n, ldb), C (m x
 * n, ldc) are row-major host arrays, 8-byte aligned; they should be page-locked
 * (cudaHostAlloc / cudaHostRegister, or torch's pin_memory) for the copies to
 * run asynchronously and overlap.  `workspace` is device memory of at least
 * gb_dgemm_host_workspace_size() bytes, 256-byte aligned, owned by the caller:
 * the emulated workspace (emulated precision) followed by dense device copies
 * of A, B and C.
 * Emulated precision: A (and C when beta != 0) is copied in bands of whole
 * 128-row tiles (up to 4, each at least 8 waves of output tiles over the SMs),
 * each band split and multiplied as soon as it arrives; B is copied first, in
 * up to 6 column blocks when there are several bands (the first small, each next
 * as large as the link can deliver while the previous block's products run), so
 * the first band's products start on the first block while the others arrive;
 * the last band runs in two launches so that only a small last block of C is
 * copied back after the products end; each block of C is copied back while the
 * next launches compute (gb_dgemm_host_schedule lists the launches).  Residue
 * precision (GB_PREC_EMULATED_CRT): A's first band of whole 128-row tiles, then B
 * in up to 4 blocks of whole 256-column tiles, then A's other bands (up to 4
 * bands, each at least two waves of products); the first band is multiplied with
 * each block of B as it arrives, the other bands with all of B as they arrive,
 * each piece's residues reconstructed into C and copied back while the next
 * piece computes.  BF16 digits: GB_ERR_UNSUPPORTED.  Native precision: A, B (and
 * C) are copied, multiplied by the default native kernel, C copied back.
 * The copies run on two streams the queue creates on the first call (one per
 * direction), ordered after all work already on the queue; the queue's stream
 * passes the end of this call once C is back in host memory.  The caller must
 * not touch A, B, C or the workspace before that (gb_queue_wait).  Asynchronous
 * with respect to the host on a non-blocking queue, synchronous on a blocking one.
 * Errors: as gb_dgemm; GB_ERR_WORKSPACE for a missing, misaligned or small
 * workspace.
 */
gb_status gb_dgemm_host(gb_queue* q, gb_precision prec, int slices, int64_t m, int64_t n,
                        int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double beta, double* C, int64_t ldc, void* workspace,
                        size_t workspace_bytes);

/* Device workspace bytes gb_dgemm_host needs for these sizes. */
gb_status gb_dgemm_host_workspace_size(gb_precision prec, int slices, int64_t m, int64_t n,
                                       int64_t k, size_t* out);

/* The products launches gb_dgemm_host makes for an emulated GEMM with these
 * sizes on a device with sm_count SMs, in enqueue order: launch p computes rows
 * pieces[4p] .. pieces[4p+1] - 1 and columns pieces[4p+2] .. pieces[4p+3] - 1 of C
 * (edges on whole 128-row x bn-column output tiles; together the launches cover
 * C once).  The launches of the first row band use the column blocks of B in the
 * order they are copied in.  Host-only (no device is touched).  *count receives
 * the number of launches (at most 10; 0 for an empty product); GB_ERR_INVALID_ARG
 * when it exceeds max_pieces (nothing written), for negative sizes, sm_count < 1
 * or slices outside [0, 16]. */
gb_status gb_dgemm_host_schedule(int slices, int64_t m, int64_t n, int64_t k, double beta,
                                 int sm_count, int64_t* pieces, int max_pieces, int* count);

/* Diagnostic of the failure path (the paper has no failure model; this library
 * bounds every device-side wait): enqueues a kernel that waits on a barrier
 * nothing will ever complete, gives up after timeout_us microseconds (1 .. 2e6),
 * records the timeout in the queue's status word and exits normally.  The next
 * gb_queue_wait returns GB_ERR_TIMEOUT and the queue stays usable. */
gb_status gb_selftest_wait_timeout(gb_queue* q, uint32_t timeout_us);

/*
 * The emulated GEMM without any allocation or workspace argument.  The paper
 * has no counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the product -- programs whose memory pool owns
 * the whole device (a cudaMalloc would fail), plug-ins that are handed only
 * their input and output buffers, and latency-bound loops that must not pay
 * for cudaMalloc / cudaFree, which may synchronize the whole device.
 *
 * Same operation, arguments and result as gb_dgemm(prec = GB_PREC_EMULATED,
 * slices) with C <- alpha A B + beta C, enqueued on `cuda_stream` (a
 * cudaStream_t of the current device, or NULL); slices = 0 takes 11.  Its
 * scratch (digit planes and exponents) is one 64 MiB array in the library's
 * device memory; a GEMM whose gb_dgemm_workspace_size() exceeds 64 MiB is
 * rejected with GB_ERR_UNSUPPORTED.  No cudaMalloc, cudaFree or other
 * allocating call is made by this function.
 * Set-up: the first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress).  With CUDA's lazy module
 * loading (the default) that first call is also when the 64 MiB are reserved
 * on the device, held from then until the process exits; so make the first
 * call on each device early -- before any stream capture, and before a memory
 * pool takes the rest of the device.
 * Every call uses the same scratch and leaves its contents behind (nothing in
 * it needs clearing: each call rewrites every byte it reads).  Two calls that
 * can run at the same time on the GPU (different streams, no ordering between
 * them) race on the scratch and corrupt each other's result.
 * Device-side status is not reported: rows of A and columns of B with NaN/Inf
 * give NaN outputs as in gb_dgemm, and if a device-side wait of the products
 * kernel gives up (after 4 s, which only a stalled GPU reaches) the output tiles
 * of that CTA are not written, so C is then undefined and no error says so.
 * Errors: those of gb_dgemm's argument checks, GB_ERR_UNSUPPORTED,
 * GB_ERR_NO_DEVICE, GB_ERR_CUDA.
 */
gb_status gb_dgemm_emulated_noalloc(void* cuda_stream, int slices, int64_t m, int64_t n,
                                    int64_t k, double alpha, const double* A, int64_t lda,
                                    const double* B, int64_t ldb, double beta, double* C,
                                    int64_t ldc);

#ifdef __cplusplus
}
#endif

#endif /* GB_GEMM_H */
