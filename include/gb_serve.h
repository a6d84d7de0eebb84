/*
 * gb_serve.h -- a GEMM request server with HBM-budget admission and
 * continuous batching (C ABI).
 *
 * Every request is one DGEMM of Section 4.2, C <- alpha A B + beta C, with the
 * conventions and accuracy contract of gb_gemm.h, in either precision.  The
 * server keeps operands resident in a device arena of a fixed HBM budget: a
 * request is admitted (first in, first out within its lane) once its operands
 * (and, for the emulated precision, its workspace) fit in the budget; admitted
 * requests are launched on one of several streams, so their work overlaps on
 * the device; a batch's memory returns to the budget when it completes, which
 * admits the next requests.
 *
 * Policies.  GB_SERVE_LANES (the default): a native request of at least 2^31
 * flops (2 m n k; square n >= 1024) is large and runs alone, as an ordinary
 * GEMM launch of many short CTAs, on a low-priority stream; every other request
 * is small and is batched into grouped launches (gb_grouped.h kernels), up to
 * max_batch requests and 2^33 flops of FP64-pipe work (emulated requests count
 * 1/16 of theirs), on high-priority streams, so the CTA slots a large GEMM frees
 * go to waiting small batches first, and no new large request starts while
 * max_batch or more small requests are queued.  With n_streams >= 2, n_streams / 2 streams
 * serve the large lane and the rest the small lane; a single stream serves both
 * lanes, taking whichever head request arrived first.  GB_SERVE_FIFO: one queue,
 * every batch a grouped launch of up to max_batch requests in arrival order
 * (with max_batch = 1: one launch per GEMM).
 *
 * A request's kernels depend only on its own shape, precision and data and on
 * the policy (the lane and the tile variant come from its shape, no reduction
 * spans problems), so its result is the same, bit for bit, alone and in any mix
 * under the same policy.
 *
 * Threading: submit/poll/stats may be called from any host thread; the server
 * runs one worker thread of its own.
 */
#ifndef GB_SERVE_H
#define GB_SERVE_H

#include "gb_gemm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t m, n, k;
    double alpha, beta;
    int32_t precision;  /* gb_precision */
    int32_t slices;     /* emulated: 1..16, 0 = the tuning table's count for the
                           request's shape, fixed at submit (else 11) */
    /* Operands: either host arrays (row-major, leading dimensions = k, n, n),
     * copied in when the request is batched and kept valid by the caller until
     * the request is done; or, with A_host == NULL, generated on the device
     * from `seed`: entries uniform in [-1, 1) from the counter-based splitmix64
     * stream `seed` (A: stream 0, B: stream 1, C: stream 2, element (i, j) of
     * an R x S matrix at counter i S + j + (stream << 40)). */
    const double* A_host;
    const double* B_host;
    const double* C_host;   /* initial C when beta != 0 (NULL: from the seed / zeros) */
    double* C_out;          /* host array receiving C when done (NULL: not copied back);
                               page-locked memory is filled by a copy on the batch's
                               stream, pageable memory by the server's worker thread
                               once the batch has completed */
    uint64_t seed;
} gb_request;

typedef struct {
    int64_t submitted, completed, rejected, pending, in_flight;
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> completion, completed requests */
    double tflops;        /* useful 2 m n k flops of completed requests / busy span */
    double busy_s;        /* first submit -> last completion */
    int64_t max_queue;    /* largest FIFO length seen */
    int64_t batches;      /* grouped launches issued */
    double mean_batch;    /* requests per batch */
    size_t peak_bytes;    /* largest arena use */
    int64_t large_launches;  /* large-lane requests launched (GB_SERVE_LANES) */
} gb_server_stats;

typedef enum { GB_SERVE_LANES = 0, GB_SERVE_FIFO = 1 } gb_serve_policy;

/* hbm_budget_bytes: device arena (allocated once here);  n_streams: batches
 * in flight at once (1..16);  max_batch: requests per grouped launch (1..4096).
 * The GB_SERVE_LANES policy. */
gb_status gb_server_create(gb_device* dev, size_t hbm_budget_bytes, int n_streams,
                           int max_batch, gb_server** out);

/* As gb_server_create with an explicit policy (a gb_serve_policy value;
 * GB_ERR_INVALID_ARG otherwise). */
gb_status gb_server_create_ex(gb_device* dev, size_t hbm_budget_bytes, int n_streams,
                              int max_batch, int policy, gb_server** out);

/* Queue a request; returns at once with its id.  GB_ERR_OUT_OF_BUDGET when it
 * can never fit the budget; argument errors as gb_dgemm. */
gb_status gb_server_submit(gb_server* s, const gb_request* req, uint64_t* request_id);

/* done = 1 once the request finished; *req_status its result (GB_OK, or the
 * device status of its batch); latency_ms from submit to completion. */
gb_status gb_server_poll(gb_server* s, uint64_t request_id, int* done, gb_status* req_status,
                         double* latency_ms);

/* Wait until every submitted request finished or timeout_s passed
 * (GB_ERR_TIMEOUT; requests keep running). */
gb_status gb_server_drain(gb_server* s, double timeout_s);

gb_status gb_server_stats_get(gb_server* s, gb_server_stats* out);

/* Stop: requests not yet batched are cancelled (status GB_ERR_BUSY), batches in
 * flight complete, then every resource is freed. */
gb_status gb_server_destroy(gb_server* s);

/* Fill a rows x cols matrix (leading dimension ld) on the device with the
 * request generator's values for (seed, stream), as a request with
 * A_host == NULL would see them.  Enqueued on cuda_stream. */
gb_status gb_fill_uniform(void* cuda_stream, double* dst, int64_t rows, int64_t cols, int64_t ld,
                          uint64_t seed, int32_t stream_id);

#ifdef __cplusplus
}
#endif

#endif /* GB_SERVE_H */
