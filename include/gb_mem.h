/*
 * gb_mem.h -- pitched buffers and explicit copies (C ABI).
 *
 * Section 3.4.4 ("Memory"): a buffer is a plain pointer plus the device it
 * resides on, its extent per dimension, its pitch and its dimension; buffers of
 * every device (the host included) have the same form, and a copy between any
 * two of them is an explicit operation enqueued in a queue that honours both
 * pitches and takes the copied extent.  With these calls and
 * gb_queue_create_owned the library runs without any other memory or stream
 * provider.
 *
 * Layout: dimension 0 is the outermost (rows of a matrix), the last dimension
 * the innermost (contiguous elements).  Row r of plane p starts at
 *   ptr + (p * extent[dim-2] + r) * pitch_bytes
 * (a 3-D buffer is a stack of 2-D planes with the same pitch; a 1-D buffer is
 * one row).  For a matrix of doubles the leading dimension of gb_dgemm is
 * pitch_bytes / 8.
 *
 * Ownership: gb_buf_alloc allocates and gb_buf_free releases; the library never
 * frees any other pointer.  Errors as in gb_gemm.h (status codes, thread-local
 * message, nothing enqueued on an argument error).
 */
#ifndef GB_MEM_H
#define GB_MEM_H

#include "gb_gemm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    void* ptr;
    int32_t device;        /* device index, or -1 for page-locked host memory */
    uint32_t dim;          /* 1, 2 or 3 */
    uint64_t extent[3];    /* elements per dimension (unused entries 1) */
    uint64_t elem_bytes;   /* bytes per element */
    uint64_t pitch_bytes;  /* bytes between consecutive rows (>= extent[dim-1] * elem_bytes) */
} gb_buf;

/*
 * Allocate a buffer of `dim` dimensions with `extents[0..dim-1]` elements of
 * `elem_bytes` bytes each.  dev != NULL: device memory with the row pitch the
 * CUDA driver prefers for 2-D access (cudaMallocPitch; a multiple of 8 bytes
 * and at least 256-byte aligned rows); dev == NULL: page-locked host memory
 * with rows padded to 16 bytes.  Zero extents give a buffer with ptr == NULL.
 * Errors: GB_ERR_INVALID_ARG (out NULL, dim not 1..3, elem_bytes 0, size
 * overflow), GB_ERR_CUDA (allocation failed), GB_ERR_NO_DEVICE.
 */
gb_status gb_buf_alloc(gb_device* dev, uint32_t dim, const uint64_t* extents, uint64_t elem_bytes,
                       gb_buf* out);

/* Release a buffer from gb_buf_alloc (synchronises with nothing: the caller
 * makes sure no queued work still uses it) and clear *buf.  NULL ptr is a no-op. */
gb_status gb_buf_free(gb_buf* buf);

/* Leading dimension in elements (pitch_bytes / elem_bytes); GB_ERR_UNSUPPORTED
 * when the pitch is not a multiple of the element size. */
gb_status gb_buf_ld(const gb_buf* buf, int64_t* ld);

/*
 * Enqueue on q the copy of the leading `extents` block of src into dst
 * (extents NULL: all of src).  Both buffers must have the same dim and
 * elem_bytes, and the block must fit both.  Host and device buffers in any
 * combination; each row is copied at its own pitch.  Asynchronous on a
 * non-blocking queue, complete on return on a blocking one.
 * Errors: GB_ERR_INVALID_ARG (NULL, mismatched dim or element size, block
 * larger than a buffer), GB_ERR_CUDA.
 */
gb_status gb_buf_copy(gb_queue* q, gb_buf* dst, const gb_buf* src, const uint64_t* extents);

/* A queue with a stream of its own (non-blocking with respect to the legacy
 * default stream), destroyed by gb_queue_destroy.  blocking as in
 * gb_queue_create. */
gb_status gb_queue_create_owned(gb_device* dev, int blocking, gb_queue** out);

#ifdef __cplusplus
}
#endif

#endif /* GB_MEM_H */
