// Definitions of the opaque C-ABI handles shared by the library's host files.
#pragma once

#include <cuda_runtime.h>

#include "gb_gemm.h"
#include "gb_grouped.h"
#include "internal.h"

struct gb_device {
    int idx;
    int sm_count;
    int cc_major, cc_minor;
};

namespace gb {
constexpr int kAuxEvents = 24;  // events of the host-buffer pipeline (see hostpipe.cu)
}

struct gb_queue {
    gb_device* dev;
    cudaStream_t stream;
    int blocking;
    unsigned* status;  // device status word (kStatus* bits)
    bool owns_stream;  // created by gb_queue_create_owned: destroyed with the queue
    // copy streams and events of gb_dgemm_host, created on its first call
    cudaStream_t aux_h2d = nullptr, aux_d2h = nullptr;
    cudaEvent_t aux_ev[gb::kAuxEvents] = {};
};

namespace gb {

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Destroys the copy streams and events of gb_dgemm_host (if created).
void release_aux(gb_queue* q);

// Sets the error text for a failed CUDA call and returns GB_ERR_CUDA.
gb_status cuda_fail(cudaError_t e, const char* what);
// Completes a call on q: the launch error, and on a blocking queue the sync and
// the device status.
gb_status finish_call(gb_queue* q, cudaError_t e, const char* what);

// Bytes of device (and pinned staging) space the tables of `count` grouped
// problems need.
size_t grouped_table_bytes(int64_t count);
// Slice count of an emulated grouped problem (or request) submitted with
// slices = 0: the tuning table's slice-count entry for its shape, else 11.
int default_emulated_slices(int64_t m, int64_t n, int64_t k);

// Enqueues a group on L.stream without any host synchronisation: the tables are
// packed into `staging` (pinned host memory of grouped_table_bytes(count) bytes,
// which must stay untouched until the stream passes this point), copied to
// `tables` (device) and the kernels launched.  Emulated problem i uses the
// workspace emu_ws[i] (laid out as gb_emulated_layout, gb_dgemm_workspace_size
// bytes).  *launches receives the number of kernel launches.
gb_status grouped_enqueue_async(const Launch& L, const gb_gemm_desc* descs, int64_t count,
                                void* tables, size_t table_bytes, void* staging,
                                void* const* emu_ws, int64_t* launches);

}  // namespace gb
