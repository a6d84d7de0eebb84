// Pitched buffers, explicit copies and queues with their own stream
// (include/gb_mem.h).  Rows are the unit of pitch: a buffer of dim D holds
// extent[0] * ... * extent[D-2] rows of extent[D-1] elements, each row at its own
// pitch, so one 2-D strided copy moves any leading block whose planes are whole;
// a 3-D block with fewer rows per plane than its buffers takes one copy per plane.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "gb_mem.h"
#include "handles.h"
#include "internal.h"

using namespace gb;

namespace {

gb_status invalid_mem(const char* msg) {
    set_error("%s", msg);
    return GB_ERR_INVALID_ARG;
}

// rows per plane and planes of a dim-D extent (a 1-D buffer is one row)
void shape_of(uint32_t dim, const uint64_t* ext, uint64_t* rows, uint64_t* planes,
              uint64_t* width) {
    *width = ext[dim - 1];
    *rows = dim >= 2 ? ext[dim - 2] : 1;
    *planes = dim == 3 ? ext[0] : 1;
}

bool mul_ok(uint64_t a, uint64_t b, uint64_t* out) {
    if (a != 0 && b > UINT64_MAX / a) return false;
    *out = a * b;
    return true;
}

}  // namespace

extern "C" {

gb_status gb_buf_alloc(gb_device* dev, uint32_t dim, const uint64_t* extents, uint64_t elem_bytes,
                       gb_buf* out) {
    if (!out || !extents) return invalid_mem("out or extents is NULL");
    std::memset(out, 0, sizeof(*out));
    if (dim < 1 || dim > 3) return invalid_mem("dim must be 1, 2 or 3");
    if (elem_bytes == 0) return invalid_mem("elem_bytes must be > 0");
    gb_buf b{};
    b.device = dev ? dev->idx : -1;
    b.dim = dim;
    b.elem_bytes = elem_bytes;
    for (int d = 0; d < 3; ++d) b.extent[d] = d < (int)dim ? extents[d] : 1;
    uint64_t rows, planes, width, wbytes, nrows;
    shape_of(dim, b.extent, &rows, &planes, &width);
    if (!mul_ok(width, elem_bytes, &wbytes) || !mul_ok(rows, planes, &nrows))
        return invalid_mem("buffer size overflows");
    if (wbytes == 0 || nrows == 0) {  // empty buffer: nothing to allocate
        b.pitch_bytes = (wbytes + 15) & ~15ull;
        *out = b;
        return GB_OK;
    }
    if (dev) {
        DeviceScope scope(dev->idx);
        if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
        size_t pitch = 0;
        cudaError_t e = cudaMallocPitch(&b.ptr, &pitch, (size_t)wbytes, (size_t)nrows);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocPitch");
        b.pitch_bytes = pitch;
    } else {
        b.pitch_bytes = (wbytes + 15) & ~15ull;
        uint64_t total;
        if (!mul_ok(b.pitch_bytes, nrows, &total)) return invalid_mem("buffer size overflows");
        cudaError_t e = cudaHostAlloc(&b.ptr, (size_t)total, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            int c = 0;
            if (cudaGetDeviceCount(&c) != cudaSuccess || c == 0) {
                set_error("page-locked host memory needs a CUDA device");
                return GB_ERR_NO_DEVICE;
            }
            return cuda_fail(e, "cudaHostAlloc");
        }
    }
    *out = b;
    return GB_OK;
}

gb_status gb_buf_free(gb_buf* buf) {
    if (!buf) return invalid_mem("buf is NULL");
    if (buf->ptr) {
        cudaError_t e;
        if (buf->device >= 0) {
            DeviceScope scope(buf->device);
            e = cudaFree(buf->ptr);
        } else {
            e = cudaFreeHost(buf->ptr);
        }
        if (e != cudaSuccess) return cuda_fail(e, "freeing a buffer");
    }
    std::memset(buf, 0, sizeof(*buf));
    return GB_OK;
}

gb_status gb_buf_ld(const gb_buf* buf, int64_t* ld) {
    if (!buf || !ld) return invalid_mem("buf or ld is NULL");
    if (buf->elem_bytes == 0 || buf->pitch_bytes % buf->elem_bytes != 0) {
        set_error("pitch %llu is not a multiple of the element size %llu",
                  (unsigned long long)buf->pitch_bytes, (unsigned long long)buf->elem_bytes);
        return GB_ERR_UNSUPPORTED;
    }
    *ld = (int64_t)(buf->pitch_bytes / buf->elem_bytes);
    return GB_OK;
}

gb_status gb_buf_copy(gb_queue* q, gb_buf* dst, const gb_buf* src, const uint64_t* extents) {
    if (!q || !dst || !src) return invalid_mem("queue, dst or src is NULL");
    if (dst->dim != src->dim || dst->dim < 1 || dst->dim > 3)
        return invalid_mem("dst and src differ in dim (or dim is not 1..3)");
    if (dst->elem_bytes != src->elem_bytes || src->elem_bytes == 0)
        return invalid_mem("dst and src differ in element size");
    const uint32_t dim = src->dim;
    uint64_t ext[3] = {1, 1, 1};
    for (uint32_t d = 0; d < dim; ++d) {
        ext[d] = extents ? extents[d] : src->extent[d];
        if (ext[d] > src->extent[d] || ext[d] > dst->extent[d])
            return invalid_mem("copied extent exceeds a buffer");
    }
    uint64_t rows, planes, width;
    shape_of(dim, ext, &rows, &planes, &width);
    const uint64_t wbytes = width * src->elem_bytes;
    if (wbytes == 0 || rows == 0 || planes == 0) return GB_OK;
    if (!dst->ptr || !src->ptr) return invalid_mem("a non-empty copy names a buffer without memory");
    if (wbytes > dst->pitch_bytes || wbytes > src->pitch_bytes)
        return invalid_mem("a buffer's pitch is below its row width");
    DeviceScope scope(q->dev->idx);
    const uint64_t src_rows = dim >= 2 ? src->extent[dim - 2] : 1;
    const uint64_t dst_rows = dim >= 2 ? dst->extent[dim - 2] : 1;
    cudaError_t e = cudaSuccess;
    if (planes == 1 || (rows == src_rows && rows == dst_rows)) {
        // whole planes (or one plane): every row of the block is one strided run
        e = cudaMemcpy2DAsync(dst->ptr, (size_t)dst->pitch_bytes, src->ptr,
                              (size_t)src->pitch_bytes, (size_t)wbytes, (size_t)(rows * planes),
                              cudaMemcpyDefault, q->stream);
    } else {
        for (uint64_t p = 0; p < planes && e == cudaSuccess; ++p)
            e = cudaMemcpy2DAsync(static_cast<uint8_t*>(dst->ptr) + p * dst_rows * dst->pitch_bytes,
                                  (size_t)dst->pitch_bytes,
                                  static_cast<const uint8_t*>(src->ptr) +
                                      p * src_rows * src->pitch_bytes,
                                  (size_t)src->pitch_bytes, (size_t)wbytes, (size_t)rows,
                                  cudaMemcpyDefault, q->stream);
    }
    return finish_call(q, e, "gb_buf_copy");
}

gb_status gb_queue_create_owned(gb_device* dev, int blocking, gb_queue** out) {
    if (!dev || !out) return invalid_mem("dev or out is NULL");
    *out = nullptr;
    DeviceScope scope(dev->idx);
    if (!scope.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    gb_queue* q = nullptr;
    const gb_status st = gb_queue_create(dev, s, blocking, &q);
    if (st != GB_OK) {
        cudaStreamDestroy(s);
        return st;
    }
    q->owns_stream = true;
    *out = q;
    return GB_OK;
}

}  // extern "C"
