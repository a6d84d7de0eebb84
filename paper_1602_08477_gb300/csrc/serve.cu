// GEMM request server (include/gb_serve.h): HBM-budget admission over a device
// arena, FIFO queues, continuous batching into grouped launches on several
// streams, and latency accounting.  All host logic runs on one worker thread.
//
// Lanes (the default policy): a native request of at least kLargeFlops is
// "large" and runs alone as an ordinary GEMM launch (many short CTAs, no
// persistent grid) on a low-priority stream; every other request is "small" and
// is batched, up to a cost cap, into grouped launches on high-priority streams.
// A persistent grouped kernel holds its SMs until its last tile, so a small
// request batched with (or queued behind) a 100 ms GEMM waited for all of it;
// with lanes the block scheduler hands each CTA slot that a large GEMM frees to
// the pending small batch first.  The lane depends only on the request itself,
// so its kernels, and its result, do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gb_grouped.h"
#include "gb_serve.h"
#include "handles.h"
#include "internal.h"

namespace gb {
namespace {

using Clock = std::chrono::steady_clock;

// ---- device-side operand generator (splitmix64, Steele-Lea-Flood 2014) -------------
__global__ void fill_uniform_kernel(double* __restrict__ dst, int64_t rows, int64_t cols,
                                    int64_t ld, uint64_t seed, int32_t stream_id) {
    const int64_t total = rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / cols, j = t - i * cols;
        const uint64_t c = ((uint64_t)stream_id << 40) + (uint64_t)t;
        uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        // 2 * (53-bit integer * 2^-53) - 1, exact in FP64
        dst[i * ld + j] = (double)(int64_t)(z >> 11) * 2.220446049250313e-16 - 1.0;
    }
}

cudaError_t fill_uniform(cudaStream_t s, double* dst, int64_t rows, int64_t cols, int64_t ld,
                         uint64_t seed, int32_t sid, int sms) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    fill_uniform_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, rows, cols, ld, seed, sid);
    return cudaGetLastError();
}

// ---- first-fit arena with coalescing ----------------------------------------------
class Arena {
   public:
    void init(size_t bytes) {
        total_ = bytes;
        free_.clear();
        free_[0] = bytes;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 1023) & ~(size_t)1023;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 1023) & ~(size_t)1023;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t total() const { return total_; }
    size_t peak() const { return peak_; }

   private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0, used_ = 0, peak_ = 0;
};

// Native requests of at least 2^31 flops (square n >= 1024, >= 1.7 ms on the whole
// FP64 pipe) take the large lane; a small-lane batch stops growing at 2^33 flops
// of FP64-pipe work (an emulated request counts 1/16 of its flops: its pair
// products run on the tensor pipe).
constexpr double kLargeFlops = 2147483648.0;
constexpr double kBatchCost = 8589934592.0;

struct Request {
    uint64_t id;
    int lane = 0;     // 0 small (grouped batches), 1 large (alone, plain GEMM launch)
    double cost = 0;  // FP64-pipe-equivalent flops
    gb_request r;
    size_t bytes;     // arena footprint
    size_t off = 0;   // arena offset
    Clock::time_point t_submit, t_done;
    gb_status status = GB_OK;
    int state = 0;    // 0 queued, 1 batched, 2 done
    double flops;
    // C in the arena, copied to a pageable C_out when the batch is done (a copy
    // into pageable memory enqueued on the stream would hold the worker thread
    // until the GEMM and the copy finished, and no other batch could start)
    double* late_copy = nullptr;
};

struct Slot {
    int lane = -1;    // lane served; -1: either (a server with one stream)
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* staging = nullptr;   // pinned host tables
    void* tables = nullptr;    // device tables
    unsigned* status = nullptr;
    std::vector<Request*> batch;
    bool busy = false;
};

size_t footprint(const gb_request& r) {
    size_t b = 8 * ((size_t)r.m * r.k + (size_t)r.k * r.n + (size_t)r.m * r.n) + 3 * 1024;
    if (r.precision == GB_PREC_EMULATED) {
        // either orientation (the tuning table may pick the one the padding rule
        // does not): the larger workspace
        const int s = r.slices;  // resolved at submit
        b += std::max(emu_group_layout(s, r.m, r.n, r.k, false).total,
                      emu_group_layout(s, r.m, r.n, r.k, true).total) +
             1024;
    }
    return b;
}

}  // namespace
}  // namespace gb

struct gb_server {
    gb_device* dev;
    uint8_t* arena_base = nullptr;
    gb::Arena arena;
    int max_batch = 64;
    std::vector<gb::Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    int policy = GB_SERVE_LANES;
    std::deque<gb::Request*> fifo[2];  // per lane (FIFO policy: lane 0 only)
    std::unordered_map<uint64_t, gb::Request*> all;
    std::atomic<bool> stop{false};
    std::thread worker;
    uint64_t next_id = 1;
    int64_t submitted = 0, completed = 0, rejected = 0, in_flight = 0, batches = 0, batched_reqs = 0;
    int64_t max_queue = 0;
    int64_t large_launches = 0;
    double done_flops = 0;
    bool have_first = false;
    gb::Clock::time_point t_first, t_last;
    std::vector<double> lat_ms;
    size_t table_bytes = 0;
};

namespace gb {
namespace {

void complete_batch(gb_server* S, Slot& sl) {
    unsigned h = 0;
    cudaMemcpy(&h, sl.status, sizeof(h), cudaMemcpyDeviceToHost);
    if (h) cudaMemset(sl.status, 0, sizeof(h));
    gb_status st = (h & kStatusTimeout) ? GB_ERR_TIMEOUT
                   : (h & kStatusNonfinite) ? GB_ERR_NONFINITE
                                            : GB_OK;
    // results bound for pageable host memory: the batch is done, copy them now
    for (Request* r : sl.batch) {
        if (r->late_copy &&
            cudaMemcpy(r->r.C_out, r->late_copy, 8 * r->r.m * r->r.n, cudaMemcpyDeviceToHost) !=
                cudaSuccess &&
            st == GB_OK)
            st = GB_ERR_CUDA;
        r->late_copy = nullptr;
    }
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request* r : sl.batch) {
        r->t_done = now;
        r->status = st;
        r->state = 2;
        S->arena.release(r->off, r->bytes);
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        S->done_flops += r->flops;
        ++S->completed;
        --S->in_flight;
    }
    S->t_last = now;
    sl.batch.clear();
    sl.busy = false;
    S->cv.notify_all();
}

// Lane a slot takes its next batch from: its own, or for a slot that serves
// either lane, the lane whose head request arrived first.  -1: nothing queued.
int pick_lane(gb_server* S, const Slot& sl) {
    // a large-lane slot starts nothing new while a full small batch waits: the
    // FP64 pipe goes to the short requests first (the GEMMs already running
    // finish, their pending CTAs behind the small batches' in priority)
    if (sl.lane == 1 && (int64_t)S->fifo[0].size() >= S->max_batch) return -1;
    if (sl.lane >= 0) return S->fifo[sl.lane].empty() ? -1 : sl.lane;
    if (S->fifo[0].empty()) return S->fifo[1].empty() ? -1 : 1;
    if (S->fifo[1].empty()) return 0;
    return S->fifo[1].front()->t_submit < S->fifo[0].front()->t_submit ? 1 : 0;
}

// Operands of a request in its arena block: copied from the host or generated.
cudaError_t stage_operands(gb_server* S, const Request* rq, cudaStream_t st, double** pA,
                           double** pB, double** pC, void** emu_ws) {
    const gb_request& q = rq->r;
    const int sms = S->dev->sm_count;
    uint8_t* base = S->arena_base + rq->off;
    double* A = reinterpret_cast<double*>(base);
    double* B = A + q.m * q.k;
    double* C = B + q.k * q.n;
    size_t used = 8 * ((size_t)q.m * q.k + (size_t)q.k * q.n + (size_t)q.m * q.n);
    *emu_ws = base + ((used + 1023) & ~(size_t)1023);
    *pA = A;
    *pB = B;
    *pC = C;
    cudaError_t e;
    if (q.A_host) {
        e = cudaMemcpyAsync(A, q.A_host, 8 * q.m * q.k, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B, q.B_host, 8 * q.k * q.n, cudaMemcpyHostToDevice, st);
    } else {
        e = fill_uniform(st, A, q.m, q.k, q.k, q.seed, 0, sms);
        if (e == cudaSuccess) e = fill_uniform(st, B, q.k, q.n, q.n, q.seed, 1, sms);
    }
    if (e == cudaSuccess && q.beta != 0.0) {
        if (q.C_host)
            e = cudaMemcpyAsync(C, q.C_host, 8 * q.m * q.n, cudaMemcpyHostToDevice, st);
        else if (!q.A_host)
            e = fill_uniform(st, C, q.m, q.n, q.n, q.seed, 2, sms);
        else
            e = cudaMemsetAsync(C, 0, 8 * q.m * q.n, st);
    }
    return e;
}

// A large native request: one ordinary GEMM launch with the library's default
// kernel for its size (16 x 16 shared-memory tiles up to 2048, 4 x 4 register
// tiles above), whose many short CTAs leave their slots to higher-priority work.
cudaError_t launch_large_native(const Launch& L, const gb_request& q, const double* A,
                                const double* B, double* C) {
    const Gemm g{q.m, q.n, q.k, q.alpha, q.beta, A, q.k > 0 ? q.k : 1, B, q.n > 0 ? q.n : 1,
                 C, q.n > 0 ? q.n : 1};
    if (q.m == 0 || q.n == 0) return cudaSuccess;
    if (q.alpha == 0.0 || q.k == 0) return launch_scale(L, g);
    const int64_t mn = q.m < q.n ? q.m : q.n;
    return mn <= 2048 ? launch_tiled(L, g, 16) : launch_dfma(L, g, 4);
}

// Forms one batch from the head of the slot's lane (first in, first out; stops at
// the first request that does not fit the budget) and enqueues it on the slot's
// stream: a large request alone, small ones up to max_batch and the cost cap.
bool launch_batch(gb_server* S, Slot& sl) {
    std::vector<Request*> batch;
    int lane = -1;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        lane = pick_lane(S, sl);
        if (lane < 0) return false;
        std::deque<Request*>& fifo = S->fifo[lane];
        const int cap = lane == 1 ? 1 : S->max_batch;
        double cost = 0;
        while (!fifo.empty() && (int)batch.size() < cap) {
            Request* r = fifo.front();
            if (S->policy == GB_SERVE_LANES && !batch.empty() && cost + r->cost > kBatchCost) break;
            size_t off = 0;
            if (!S->arena.alloc(r->bytes, &off)) break;
            r->off = off;
            r->state = 1;
            fifo.pop_front();
            batch.push_back(r);
            cost += r->cost;
            ++S->in_flight;
        }
    }
    if (batch.empty()) return false;
    const int sms = S->dev->sm_count;
    std::vector<gb_gemm_desc> descs(batch.size());
    std::vector<void*> emu_ws(batch.size(), nullptr);
    std::vector<double*> outC(batch.size(), nullptr);
    cudaError_t e = cudaSuccess;
    gb_status st = GB_OK;
    const Launch L{sl.stream, sl.status, sms};
    for (size_t i = 0; i < batch.size() && e == cudaSuccess; ++i) {
        const gb_request& q = batch[i]->r;
        double *A, *B, *C;
        e = stage_operands(S, batch[i], sl.stream, &A, &B, &C, &emu_ws[i]);
        outC[i] = C;
        if (lane == 1) {
            if (e == cudaSuccess) e = launch_large_native(L, q, A, B, C);
            continue;
        }
        gb_gemm_desc& d = descs[i];
        std::memset(&d, 0, sizeof(d));
        d.m = q.m;
        d.n = q.n;
        d.k = q.k;
        d.alpha = q.alpha;
        d.beta = q.beta;
        d.A = A;
        d.lda = q.k > 0 ? q.k : 1;
        d.B = B;
        d.ldb = q.n > 0 ? q.n : 1;
        d.C = C;
        d.ldc = q.n > 0 ? q.n : 1;
        d.precision = q.precision;
        d.slices = q.slices;
        d.tile = GB_TILE_AUTO;
    }
    if (e == cudaSuccess && lane == 0) {
        int64_t nl = 0;
        st = grouped_enqueue_async(L, descs.data(), (int64_t)descs.size(), sl.tables,
                                   S->table_bytes, sl.staging, emu_ws.data(), &nl);
    }
    for (size_t i = 0; i < batch.size() && e == cudaSuccess && st == GB_OK; ++i) {
        const gb_request& q = batch[i]->r;
        if (!q.C_out) continue;
        // page-locked destinations are copied on the stream; pageable ones when
        // the batch is done (complete_batch)
        cudaPointerAttributes pa{};
        const bool pinned = cudaPointerGetAttributes(&pa, q.C_out) == cudaSuccess &&
                            pa.type == cudaMemoryTypeHost;
        if (pinned)
            e = cudaMemcpyAsync(q.C_out, outC[i], 8 * q.m * q.n, cudaMemcpyDeviceToHost,
                                sl.stream);
        else
            batch[i]->late_copy = outC[i];
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess || st != GB_OK) {
        // the batch never ran: mark its requests failed and give their memory back
        cudaStreamSynchronize(sl.stream);
        std::lock_guard<std::mutex> lock(S->mu);
        for (Request* r : batch) {
            r->status = st != GB_OK ? st : GB_ERR_CUDA;
            r->state = 2;
            r->t_done = Clock::now();
            S->arena.release(r->off, r->bytes);
            --S->in_flight;
            ++S->rejected;
        }
        S->cv.notify_all();
        return true;
    }
    sl.batch = std::move(batch);
    sl.busy = true;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        ++S->batches;
        S->batched_reqs += (int64_t)sl.batch.size();
        if (lane == 1) ++S->large_launches;
    }
    return true;
}

void worker_main(gb_server* S) {
    cudaSetDevice(S->dev->idx);
    for (;;) {
        bool progress = false;
        for (Slot& sl : S->slots) {
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
                complete_batch(S, sl);
                progress = true;
            }
        }
        const bool stopping = S->stop.load();
        if (!stopping) {
            for (Slot& sl : S->slots)
                if (!sl.busy && launch_batch(S, sl)) progress = true;
        }
        bool any_busy = false;
        for (Slot& sl : S->slots) any_busy |= sl.busy;
        if (stopping && !any_busy) break;
        if (!progress) {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv.wait_for(lock, std::chrono::microseconds(50));
        }
    }
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

gb_status gb_fill_uniform(void* cuda_stream, double* dst, int64_t rows, int64_t cols, int64_t ld,
                          uint64_t seed, int32_t stream_id) {
    if (rows < 0 || cols < 0 || ld < (cols > 1 ? cols : 1) || (rows * cols > 0 && !dst)) {
        set_error("gb_fill_uniform: bad size, leading dimension or pointer");
        return GB_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = fill_uniform((cudaStream_t)cuda_stream, dst, rows, cols, ld, seed, stream_id, sms);
    return e == cudaSuccess ? GB_OK : cuda_fail(e, "gb_fill_uniform");
}

gb_status gb_server_create(gb_device* dev, size_t hbm_budget_bytes, int n_streams, int max_batch,
                           gb_server** out) {
    return gb_server_create_ex(dev, hbm_budget_bytes, n_streams, max_batch, GB_SERVE_LANES, out);
}

gb_status gb_server_create_ex(gb_device* dev, size_t hbm_budget_bytes, int n_streams,
                              int max_batch, int policy, gb_server** out) {
    if (!dev || !out || n_streams < 1 || n_streams > 16 || max_batch < 1 || max_batch > 4096 ||
        hbm_budget_bytes < (1u << 20) || (policy != GB_SERVE_LANES && policy != GB_SERVE_FIFO)) {
        set_error("gb_server_create: bad device, budget (>= 1 MiB), streams (1..16), batch "
                  "(1..4096) or policy");
        return GB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    DeviceScope scope(dev->idx);
    gb_server* S = new (std::nothrow) gb_server();
    if (!S) {
        set_error("out of host memory");
        return GB_ERR_INVALID_ARG;
    }
    S->dev = dev;
    S->max_batch = max_batch;
    S->policy = policy;
    S->table_bytes = grouped_table_bytes(max_batch);
    cudaError_t e = cudaMalloc(&S->arena_base, hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "allocating the server arena");
    }
    S->arena.init(hbm_budget_bytes);
    S->slots.resize(n_streams);
    // lanes: half the streams (rounded down) for large requests at the lowest
    // stream priority, the rest for small batches at the highest; one stream
    // serves both lanes at the default priority
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    const int n_large = (policy == GB_SERVE_LANES && n_streams > 1) ? n_streams / 2 : 0;
    for (int i = 0; i < n_streams; ++i) {
        Slot& sl = S->slots[i];
        int prio = 0;
        if (policy == GB_SERVE_FIFO) {
            sl.lane = 0;
        } else if (n_streams == 1) {
            sl.lane = -1;
        } else {
            sl.lane = i < n_large ? 1 : 0;
            prio = sl.lane == 1 ? prio_low : prio_high;
        }
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.staging, S->table_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&sl.tables, S->table_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.status, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(sl.status, 0, sizeof(unsigned));
    }
    if (e != cudaSuccess) {
        gb_status st = cuda_fail(e, "creating the server streams");
        for (Slot& sl : S->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.staging) cudaFreeHost(sl.staging);
            if (sl.tables) cudaFree(sl.tables);
            if (sl.status) cudaFree(sl.status);
        }
        cudaFree(S->arena_base);
        delete S;
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return GB_OK;
}

gb_status gb_server_submit(gb_server* S, const gb_request* req, uint64_t* request_id) {
    if (!S || !req || !request_id) {
        set_error("server, request or id is NULL");
        return GB_ERR_INVALID_ARG;
    }
    const gb_request& q = *req;
    if (q.precision == GB_PREC_EMULATED_BF16 || q.precision == GB_PREC_EMULATED_CRT) {
        set_error("gb_server_submit: requests take native or E4M3-digit precision");
        return GB_ERR_UNSUPPORTED;
    }
    if (q.m < 0 || q.n < 0 || q.k < 0 || (q.precision != GB_PREC_NATIVE && q.precision != GB_PREC_EMULATED) ||
        q.slices < 0 || q.slices > 16 || (q.A_host && !q.B_host) || !(q.alpha == q.alpha) ||
        !(q.beta == q.beta)) {
        set_error("gb_server_submit: bad sizes, precision, slices, operands or scalars");
        return GB_ERR_INVALID_ARG;
    }
    Request* r = new (std::nothrow) Request();
    if (!r) {
        set_error("out of host memory");
        return GB_ERR_INVALID_ARG;
    }
    r->r = q;
    // the slice count the request runs with, fixed now: its footprint and its
    // grouped launch then agree whatever the tuning table holds later
    if (q.precision == GB_PREC_EMULATED && q.slices == 0)
        r->r.slices = default_emulated_slices(q.m, q.n, q.k);
    r->bytes = footprint(r->r);
    r->flops = 2.0 * (double)q.m * (double)q.n * (double)q.k;
    r->cost = q.precision == GB_PREC_EMULATED ? r->flops / 16.0 : r->flops;
    r->lane = (S->policy == GB_SERVE_LANES && q.precision == GB_PREC_NATIVE &&
               r->flops >= kLargeFlops) ? 1 : 0;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    if (r->bytes > S->arena.total()) {
        const size_t bytes = r->bytes;
        delete r;
        ++S->rejected;
        set_error("request of %zu bytes can never fit the %zu-byte budget", bytes,
                  S->arena.total());
        return GB_ERR_OUT_OF_BUDGET;
    }
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->fifo[r->lane].push_back(r);
    ++S->submitted;
    S->max_queue =
        std::max<int64_t>(S->max_queue, (int64_t)(S->fifo[0].size() + S->fifo[1].size()));
    if (!S->have_first) {
        S->have_first = true;
        S->t_first = r->t_submit;
    }
    *request_id = r->id;
    S->cv.notify_all();
    return GB_OK;
}

gb_status gb_server_poll(gb_server* S, uint64_t id, int* done, gb_status* req_status,
                         double* latency_ms) {
    if (!S || !done) {
        set_error("server or done is NULL");
        return GB_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) {
        set_error("unknown request id %llu", (unsigned long long)id);
        return GB_ERR_INVALID_ARG;
    }
    const Request* r = it->second;
    *done = r->state == 2;
    if (req_status) *req_status = r->status;
    if (latency_ms)
        *latency_ms = r->state == 2
                          ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count()
                          : -1.0;
    return GB_OK;
}

gb_status gb_server_drain(gb_server* S, double timeout_s) {
    if (!S) {
        set_error("server is NULL");
        return GB_ERR_INVALID_ARG;
    }
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    std::unique_lock<std::mutex> lock(S->mu);
    auto idle = [&] { return S->fifo[0].empty() && S->fifo[1].empty() && S->in_flight == 0; };
    while (!idle()) {
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout && !idle()) {
            set_error("drain timed out with %zu queued and %lld in flight",
                      S->fifo[0].size() + S->fifo[1].size(), (long long)S->in_flight);
            return GB_ERR_TIMEOUT;
        }
    }
    return GB_OK;
}

gb_status gb_server_stats_get(gb_server* S, gb_server_stats* out) {
    if (!S || !out) {
        set_error("server or out is NULL");
        return GB_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->pending = (int64_t)(S->fifo[0].size() + S->fifo[1].size());
    out->large_launches = S->large_launches;
    out->in_flight = S->in_flight;
    out->max_queue = S->max_queue;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->batched_reqs / (double)S->batches : 0.0;
    out->peak_bytes = S->arena.peak();
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>(v.size() - 1, p * (v.size() - 1) + 0.5);
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        out->max_ms = v.back();
    }
    if (S->have_first && S->completed > 0) {
        out->busy_s = std::chrono::duration<double>(S->t_last - S->t_first).count();
        if (out->busy_s > 0) out->tflops = S->done_flops / out->busy_s / 1e12;
    }
    return GB_OK;
}

gb_status gb_server_destroy(gb_server* S) {
    if (!S) return GB_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        for (auto& fifo : S->fifo) {
            for (Request* r : fifo) {
                r->status = GB_ERR_BUSY;
                r->state = 2;
            }
            fifo.clear();
        }
    }
    S->stop.store(true);
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    DeviceScope scope(S->dev->idx);
    for (Slot& sl : S->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.staging);
        cudaFree(sl.tables);
        cudaFree(sl.status);
    }
    cudaFree(S->arena_base);
    for (auto& kv : S->all) delete kv.second;
    delete S;
    return GB_OK;
}

}  // extern "C"
