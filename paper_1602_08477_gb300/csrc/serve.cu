// GEMM request server (include/gb_serve.h): HBM-budget admission over a device
// arena, FIFO queue, continuous batching into grouped launches on several
// streams, and latency accounting.  All host logic runs on one worker thread.
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

struct Request {
    uint64_t id;
    gb_request r;
    size_t bytes;     // arena footprint
    size_t off = 0;   // arena offset
    Clock::time_point t_submit, t_done;
    gb_status status = GB_OK;
    int state = 0;    // 0 queued, 1 batched, 2 done
    double flops;
};

struct Slot {
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
    if (r.precision == GB_PREC_EMULATED)
        b += emu_group_layout(r.slices == 0 ? 11 : r.slices, r.m, r.n, r.k).total + 1024;
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
    std::deque<gb::Request*> fifo;
    std::unordered_map<uint64_t, gb::Request*> all;
    std::atomic<bool> stop{false};
    std::thread worker;
    uint64_t next_id = 1;
    int64_t submitted = 0, completed = 0, rejected = 0, in_flight = 0, batches = 0, batched_reqs = 0;
    int64_t max_queue = 0;
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
    const gb_status st = (h & kStatusTimeout) ? GB_ERR_TIMEOUT
                         : (h & kStatusNonfinite) ? GB_ERR_NONFINITE
                                                  : GB_OK;
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

// Forms one batch from the FIFO head (first in, first out; stops at the first
// request that does not fit the budget) and enqueues it on the slot's stream.
bool launch_batch(gb_server* S, Slot& sl) {
    std::vector<Request*> batch;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        while (!S->fifo.empty() && (int)batch.size() < S->max_batch) {
            Request* r = S->fifo.front();
            size_t off = 0;
            if (!S->arena.alloc(r->bytes, &off)) break;
            r->off = off;
            r->state = 1;
            S->fifo.pop_front();
            batch.push_back(r);
            ++S->in_flight;
        }
    }
    if (batch.empty()) return false;
    const int sms = S->dev->sm_count;
    std::vector<gb_gemm_desc> descs(batch.size());
    std::vector<void*> emu_ws(batch.size(), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < batch.size() && e == cudaSuccess; ++i) {
        const gb_request& q = batch[i]->r;
        uint8_t* base = S->arena_base + batch[i]->off;
        double* A = reinterpret_cast<double*>(base);
        double* B = A + q.m * q.k;
        double* C = B + q.k * q.n;
        size_t used = 8 * ((size_t)q.m * q.k + (size_t)q.k * q.n + (size_t)q.m * q.n);
        emu_ws[i] = base + ((used + 1023) & ~(size_t)1023);
        if (q.A_host) {
            e = cudaMemcpyAsync(A, q.A_host, 8 * q.m * q.k, cudaMemcpyHostToDevice, sl.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(B, q.B_host, 8 * q.k * q.n, cudaMemcpyHostToDevice, sl.stream);
        } else {
            e = fill_uniform(sl.stream, A, q.m, q.k, q.k, q.seed, 0, sms);
            if (e == cudaSuccess) e = fill_uniform(sl.stream, B, q.k, q.n, q.n, q.seed, 1, sms);
        }
        if (e == cudaSuccess && q.beta != 0.0) {
            if (q.C_host)
                e = cudaMemcpyAsync(C, q.C_host, 8 * q.m * q.n, cudaMemcpyHostToDevice, sl.stream);
            else if (!q.A_host)
                e = fill_uniform(sl.stream, C, q.m, q.n, q.n, q.seed, 2, sms);
            else
                e = cudaMemsetAsync(C, 0, 8 * q.m * q.n, sl.stream);
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
    gb_status st = GB_OK;
    if (e == cudaSuccess) {
        const Launch L{sl.stream, sl.status, sms};
        int64_t nl = 0;
        st = grouped_enqueue_async(L, descs.data(), (int64_t)descs.size(), sl.tables,
                                   S->table_bytes, sl.staging, emu_ws.data(), &nl);
    }
    for (size_t i = 0; i < batch.size() && e == cudaSuccess && st == GB_OK; ++i) {
        const gb_request& q = batch[i]->r;
        if (q.C_out)
            e = cudaMemcpyAsync(q.C_out, descs[i].C, 8 * q.m * q.n, cudaMemcpyDeviceToHost,
                                sl.stream);
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
    if (!dev || !out || n_streams < 1 || n_streams > 16 || max_batch < 1 || max_batch > 4096 ||
        hbm_budget_bytes < (1u << 20)) {
        set_error("gb_server_create: bad device, budget (>= 1 MiB), streams (1..16) or batch (1..4096)");
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
    S->table_bytes = grouped_table_bytes(max_batch);
    cudaError_t e = cudaMalloc(&S->arena_base, hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "allocating the server arena");
    }
    S->arena.init(hbm_budget_bytes);
    S->slots.resize(n_streams);
    for (Slot& sl : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
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
    r->bytes = footprint(q);
    r->flops = 2.0 * (double)q.m * (double)q.n * (double)q.k;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    if (r->bytes > S->arena.total()) {
        delete r;
        ++S->rejected;
        set_error("request of %zu bytes can never fit the %zu-byte budget", footprint(q),
                  S->arena.total());
        return GB_ERR_OUT_OF_BUDGET;
    }
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->fifo.push_back(r);
    ++S->submitted;
    S->max_queue = std::max<int64_t>(S->max_queue, (int64_t)S->fifo.size());
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
    while (!(S->fifo.empty() && S->in_flight == 0)) {
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout &&
            !(S->fifo.empty() && S->in_flight == 0)) {
            set_error("drain timed out with %zu queued and %lld in flight", S->fifo.size(),
                      (long long)S->in_flight);
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
    out->pending = (int64_t)S->fifo.size();
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
        for (Request* r : S->fifo) {
            r->status = GB_ERR_BUSY;
            r->state = 2;
        }
        S->fifo.clear();
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
