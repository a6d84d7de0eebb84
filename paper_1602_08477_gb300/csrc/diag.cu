// Diagnostic: the bounded device-side wait and its host-visible timeout status.
//
// Every wait of the library's kernels on an mbarrier (pipeline stages, tensor
// memory hand-off) gives up after a wall-clock limit, records kStatusTimeout in
// the queue's status word and lets the kernel finish; gb_queue_wait then returns
// GB_ERR_TIMEOUT.  This kernel waits, with a caller-given limit, on an mbarrier
// that nothing ever arrives on, so that path can be exercised without a fault.
#include <cuda_runtime.h>

#include "gb_gemm.h"
#include "handles.h"
#include "internal.h"
#include "tc_ptx.cuh"

namespace gb {
namespace {

__global__ void wait_nothing_kernel(unsigned* status, uint64_t timeout_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        abort_flag = 0;
        ptx::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        ptx::mbar_wait_bounded(&bar, 0, &abort_flag, status, kStatusTimeout, timeout_ns);
    __syncthreads();
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" gb_status gb_selftest_wait_timeout(gb_queue* q, uint32_t timeout_us) {
    if (!q || timeout_us == 0 || timeout_us > 2000000u) {
        set_error("gb_selftest_wait_timeout: NULL queue or limit outside 1 us .. 2 s");
        return GB_ERR_INVALID_ARG;
    }
    DeviceScope scope(q->dev->idx);
    wait_nothing_kernel<<<1, 32, 0, q->stream>>>(q->status, (uint64_t)timeout_us * 1000ull);
    return finish_call(q, cudaGetLastError(), "gb_selftest_wait_timeout");
}
