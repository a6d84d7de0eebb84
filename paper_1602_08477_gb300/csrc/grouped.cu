// Grouped FP64 GEMMs (include/gb_grouped.h): problem tables, tile map, tuning
// table and the CUDA-graph plan around the persistent grouped kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gb_grouped.h"
#include "handles.h"
#include "internal.h"

struct gb_grouped_plan {
    gb_queue* q;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int use_graph;
    gb::GroupProb* d_native;
    int n_native;
    int64_t native_tiles;
    unsigned long long* d_counter;
    int grid_native;
    gb::EmuProb* d_emu;
    gb::EmuKeys d_keys;
    int n_emu;
    int64_t emu_tiles;
    int max_s;
    std::vector<gb::EmuSRange> s_ranges;  // one per distinct slice count
    int launches;
    double flops;
};

namespace gb {
namespace {

std::mutex g_tune_mu;
std::vector<gb_tune_entry> g_tune;

int default_tile(int64_t m, int64_t n) {
    if (m >= 64 && n >= 64) return kTile64x64;
    if (m >= 64) return kTile64x32;
    if (n >= 64) return kTile32x64;
    return kTile32x32;
}

bool native_tile(int t) { return t >= GB_TILE_64x64 && t <= GB_TILE_32x64; }
bool emu_orientation(int t) { return t == GB_TILE_EMU_ROWS || t == GB_TILE_EMU_COLS; }
bool slice_entry(int t) { return t >= GB_TUNE_SLICES + 1 && t <= GB_TUNE_SLICES + 16; }

// First matching entry of the native kind, else the size rule.
int lookup_tile(int64_t m, int64_t n, int64_t k) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune)
        if (native_tile(e.tile) && m <= e.m_max && n <= e.n_max && k <= e.k_max) return e.tile;
    return default_tile(m, n);
}

}  // namespace

// Slice count of an emulated problem whose descriptor leaves it to the library
// (slices = 0): the first matching slice-count entry, else 11.
int default_emulated_slices(int64_t m, int64_t n, int64_t k) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune)
        if (slice_entry(e.tile) && m <= e.m_max && n <= e.n_max && k <= e.k_max)
            return e.tile - GB_TUNE_SLICES;
    return 11;
}

namespace {

// Orientation of an emulated problem: first matching entry of the emulated
// kind, else the padding rule (emu_group_trans).
int lookup_emu(int s, int64_t m, int64_t n, int64_t k) {
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto& e : g_tune)
            if (emu_orientation(e.tile) && m <= e.m_max && n <= e.n_max && k <= e.k_max)
                return e.tile;
    }
    return emu_group_trans(s, m, n) ? GB_TILE_EMU_COLS : GB_TILE_EMU_ROWS;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

gb_status bad(const char* fmt, long long i) {
    set_error(fmt, i);
    return GB_ERR_INVALID_ARG;
}

// Splits the group into the two tables and computes the workspace layout.
struct Layout {
    std::vector<GroupProb> native;
    std::vector<EmuProb> emu;
    std::vector<EmuLayout> emu_ws;
    std::vector<int64_t> emu_idx;   // descriptor index of each emulated problem
    std::vector<EmuSRange> s_ranges;  // one per distinct slice count
    std::vector<int64_t> keys[kEmuKeys];  // compact prefixes: rows, column strips, tiles
    size_t off_counter = 0, off_native = 0, off_emu = 0, off_keys[kEmuKeys] = {0, 0, 0};
    size_t off_data = 0, total = 0;
    int max_s = 0;
    double flops = 0;
};

gb_status build_layout(const gb_gemm_desc* d, int64_t count, Layout& L) {
    if (count < 0 || (count > 0 && !d)) return bad("descriptor array is NULL or count < 0 (%lld)", count);
    for (int64_t i = 0; i < count; ++i) {
        const gb_gemm_desc& x = d[i];
        const int v = validate_gemm(x.m, x.n, x.k, x.alpha, x.A, x.lda, x.B, x.ldb, x.beta, x.C, x.ldc);
        if (v != GB_OK) {
            char msg[512];
            std::snprintf(msg, sizeof(msg), "problem %lld: %s", (long long)i, gb_last_error());
            set_error("%s", msg);
            return (gb_status)v;
        }
        if (x.precision == GB_PREC_EMULATED_BF16 || x.precision == GB_PREC_EMULATED_CRT) {
            set_error("problem %lld: a group takes native or E4M3-digit precision", (long long)i);
            return GB_ERR_UNSUPPORTED;
        }
        if (x.precision != GB_PREC_NATIVE && x.precision != GB_PREC_EMULATED)
            return bad("problem %lld: unknown precision", (long long)i);
        if (x.reserved != 0) return bad("problem %lld: reserved field must be 0", (long long)i);
        if (x.precision == GB_PREC_NATIVE && x.tile != GB_TILE_AUTO && !native_tile(x.tile))
            return bad("problem %lld: unknown native tile variant", (long long)i);
        if (x.precision == GB_PREC_EMULATED && x.tile != GB_TILE_AUTO && !emu_orientation(x.tile))
            return bad("problem %lld: an emulated problem's tile is AUTO, EMU_ROWS or EMU_COLS",
                       (long long)i);
        const int s = x.slices == 0 ? default_emulated_slices(x.m, x.n, x.k) : x.slices;
        if (x.precision == GB_PREC_EMULATED && (s < 1 || s > 16))
            return bad("problem %lld: slices must be in [1, 16] (or 0)", (long long)i);
        if (x.m == 0 || x.n == 0) continue;
        L.flops += 2.0 * (double)x.m * (double)x.n * (double)x.k;
        const bool trivial = x.alpha == 0.0 || x.k == 0;  // C <- beta C, A and B unread
        if (x.precision == GB_PREC_NATIVE || trivial) {
            GroupProb p{};
            p.m = x.m;
            p.n = x.n;
            p.k = trivial ? 0 : x.k;
            p.lda = x.lda;
            p.ldb = x.ldb;
            p.ldc = x.ldc;
            p.A = x.A;
            p.B = x.B;
            p.C = x.C;
            p.alpha = x.alpha;
            p.beta = x.beta;
            p.tile = native_tile(x.tile) ? x.tile : lookup_tile(x.m, x.n, x.k);
            p.tiles_n = (int32_t)((x.n + tile_bn(p.tile) - 1) / tile_bn(p.tile));
            L.native.push_back(p);
        } else {
            EmuProb e{};
            e.m = x.m;
            e.n = x.n;
            e.k = x.k;
            e.lda = x.lda;
            e.ldb = x.ldb;
            e.ldc = x.ldc;
            e.A = x.A;
            e.B = x.B;
            e.C = x.C;
            e.alpha = x.alpha;
            e.beta = x.beta;
            e.s = s;
            const int orient = x.tile != GB_TILE_AUTO ? x.tile : lookup_emu(s, x.m, x.n, x.k);
            e.trans = orient == GB_TILE_EMU_COLS ? 1 : 0;
            e.ra = e.trans ? emu_bn(s) : kEmuBM;
            e.rb = e.trans ? kEmuBM : emu_bn(s);
            // output tiles: 128 lines of the row side x emu_bn(s) of the column side
            const int64_t cols = e.trans ? x.m : x.n;
            e.tiles_n = (int32_t)((cols + emu_bn(s) - 1) / emu_bn(s));
            L.emu.push_back(e);
            L.emu_ws.push_back(emu_group_layout(s, x.m, x.n, x.k, e.trans != 0));
            L.emu_idx.push_back(i);
            L.max_s = std::max(L.max_s, s);
        }
    }
    // expensive tiles first: the persistent CTAs take tiles in table order
    std::stable_sort(L.native.begin(), L.native.end(), [](const GroupProb& a, const GroupProb& b) {
        const int64_t ca = (int64_t)tile_bm(a.tile) * tile_bn(a.tile) * (a.k + 8);
        const int64_t cb = (int64_t)tile_bm(b.tile) * tile_bn(b.tile) * (b.k + 8);
        return ca > cb;
    });
    int64_t t = 0;
    for (auto& p : L.native) {
        p.first_tile = t;
        t += ((p.m + tile_bm(p.tile) - 1) / tile_bm(p.tile)) * p.tiles_n;
    }
    // emulated problems of equal slice count together (one launch set each),
    // long-K problems first within a slice count (their tiles cost the most)
    {
        std::vector<size_t> perm(L.emu.size());
        for (size_t i = 0; i < perm.size(); ++i) perm[i] = i;
        std::stable_sort(perm.begin(), perm.end(), [&](size_t a, size_t b) {
            if (L.emu[a].s != L.emu[b].s) return L.emu[a].s < L.emu[b].s;
            return L.emu_ws[a].kp > L.emu_ws[b].kp;
        });
        std::vector<EmuProb> e2;
        std::vector<EmuLayout> w2;
        std::vector<int64_t> i2;
        for (size_t i : perm) {
            e2.push_back(L.emu[i]);
            w2.push_back(L.emu_ws[i]);
            i2.push_back(L.emu_idx[i]);
        }
        L.emu.swap(e2);
        L.emu_ws.swap(w2);
        L.emu_idx.swap(i2);
    }
    L.off_counter = 0;
    L.off_native = 256;
    L.off_emu = up256(L.off_native + sizeof(GroupProb) * L.native.size());
    size_t kend = up256(L.off_emu + sizeof(EmuProb) * L.emu.size());
    for (int a = 0; a < kEmuKeys; ++a) {
        L.off_keys[a] = kend;
        kend = up256(kend + sizeof(int64_t) * L.emu.size());
    }
    L.off_data = (kend + 1023) & ~(size_t)1023;
    size_t off = L.off_data;
    int64_t rows = 0, colblks = 0, tiles = 0;
    for (size_t i = 0; i < L.emu.size(); ++i) {
        EmuProb& e = L.emu[i];
        const EmuLayout& w = L.emu_ws[i];
        e.kp = w.kp;
        // device pointers are filled in once the workspace base is known
        e.first_row = rows;
        e.first_colblk = colblks;
        e.first_tile = tiles;
        L.keys[0].push_back(rows);
        L.keys[1].push_back(colblks);
        L.keys[2].push_back(tiles);
        const int64_t ncbp = ((e.n + e.rb - 1) / e.rb * e.rb + 31) / 32;     // padded to tiles
        rows += (e.m + kEmuBM - 1) / kEmuBM * kEmuBM;  // 128-row blocks of the split of A
        colblks += ncbp;
        const int64_t row_side = e.trans ? e.n : e.m;
        const int64_t nt = ((row_side + kEmuBM - 1) / kEmuBM) * e.tiles_n;
        tiles += nt;
        if (L.s_ranges.empty() || L.s_ranges.back().s != e.s)
            L.s_ranges.push_back(EmuSRange{e.s, (int)i, 0, e.first_row, 0, e.first_colblk, 0,
                                           e.first_tile, 0, 0});
        EmuSRange& r = L.s_ranges.back();
        r.q_end = (int)i + 1;
        r.kp_max = std::max(r.kp_max, w.kp);
        r.row_end = rows;
        r.cb_end = colblks;
        r.t_end = tiles;
        off += w.total;
    }
    L.total = off;
    return GB_OK;
}

EmuKeys keys_at(uint8_t* base, const Layout& L) {
    return EmuKeys{reinterpret_cast<const int64_t*>(base + L.off_keys[0]),
                   reinterpret_cast<const int64_t*>(base + L.off_keys[1]),
                   reinterpret_cast<const int64_t*>(base + L.off_keys[2])};
}

}  // namespace

size_t grouped_table_bytes(int64_t count) {
    const size_t c = (size_t)count;
    return 256 + up256(sizeof(GroupProb) * c) + up256(sizeof(EmuProb) * c) +
           kEmuKeys * up256(sizeof(int64_t) * c) + 1024;
}

gb_status grouped_enqueue_async(const Launch& L, const gb_gemm_desc* descs, int64_t count,
                                void* tables, size_t table_bytes, void* staging,
                                void* const* emu_ws, int64_t* launches) {
    Layout lay;
    gb_status st = build_layout(descs, count, lay);
    if (st != GB_OK) return st;
    if (lay.off_data > table_bytes) {
        set_error("grouped table space %zu < %zu", table_bytes, lay.off_data);
        return GB_ERR_WORKSPACE;
    }
    // each emulated problem uses the workspace of its own descriptor
    for (size_t ei = 0; ei < lay.emu.size(); ++ei) {
        uint8_t* w = static_cast<uint8_t*>(emu_ws[lay.emu_idx[ei]]);
        emu_group_assign(lay.emu[ei], w, lay.emu_ws[ei]);
    }
    uint8_t* stg = static_cast<uint8_t*>(staging);
    uint8_t* dev = static_cast<uint8_t*>(tables);
    std::memset(stg, 0, 256);
    if (!lay.native.empty())
        std::memcpy(stg + lay.off_native, lay.native.data(), sizeof(GroupProb) * lay.native.size());
    if (!lay.emu.empty()) {
        std::memcpy(stg + lay.off_emu, lay.emu.data(), sizeof(EmuProb) * lay.emu.size());
        for (int a = 0; a < kEmuKeys; ++a)
            std::memcpy(stg + lay.off_keys[a], lay.keys[a].data(), sizeof(int64_t) * lay.emu.size());
    }
    cudaError_t e = cudaMemcpyAsync(dev, stg, lay.off_data, cudaMemcpyHostToDevice, L.stream);
    int64_t nl = 0;
    if (e == cudaSuccess && !lay.native.empty()) {
        const GroupProb& last = lay.native.back();
        const int64_t tiles = last.first_tile +
                              ((last.m + tile_bm(last.tile) - 1) / tile_bm(last.tile)) * last.tiles_n;
        int64_t grid = (int64_t)L.sm_count * grouped_native_occupancy();
        if (grid > tiles) grid = tiles;
        e = launch_grouped_native(L, reinterpret_cast<GroupProb*>(dev + lay.off_native),
                                  (int)lay.native.size(), tiles,
                                  reinterpret_cast<unsigned long long*>(dev), (int)grid);
        ++nl;
    }
    if (e == cudaSuccess && !lay.emu.empty()) {
        EmuProb* d = reinterpret_cast<EmuProb*>(dev + lay.off_emu);
        const EmuKeys keys = keys_at(dev, lay);
        for (size_t r = 0; r < lay.s_ranges.size() && e == cudaSuccess; ++r) {
            e = launch_grouped_split(L, d, keys, lay.s_ranges[r]);
            if (e == cudaSuccess) e = launch_grouped_products(L, d, keys, lay.s_ranges[r]);
            nl += 3;
        }
    }
    if (launches) *launches = nl;
    if (e != cudaSuccess) return cuda_fail(e, "grouped enqueue");
    return GB_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

gb_status gb_tune_set(const gb_tune_entry* entries, int64_t count) {
    if (count < 0 || (count > 0 && !entries)) {
        set_error("tuning entries NULL or count < 0");
        return GB_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < count; ++i) {
        if (!native_tile(entries[i].tile) && !emu_orientation(entries[i].tile) &&
            !slice_entry(entries[i].tile)) {
            set_error("tuning entry %lld: tile must be a concrete variant (1..6) or a slice "
                      "count (GB_TUNE_SLICES + 1..16)", (long long)i);
            return GB_ERR_INVALID_ARG;
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.assign(entries, entries + count);
    return GB_OK;
}

gb_status gb_tune_get(gb_tune_entry* entries, int64_t capacity, int64_t* count) {
    if (!count) {
        set_error("count is NULL");
        return GB_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    *count = (int64_t)g_tune.size();
    for (int64_t i = 0; i < capacity && i < (int64_t)g_tune.size(); ++i) entries[i] = g_tune[i];
    return GB_OK;
}

gb_status gb_tune_lookup(int64_t m, int64_t n, int64_t k, int32_t* tile) {
    if (!tile || m < 0 || n < 0 || k < 0) {
        set_error("tile is NULL or a size is negative");
        return GB_ERR_INVALID_ARG;
    }
    *tile = lookup_tile(m, n, k);
    return GB_OK;
}

gb_status gb_tune_lookup_slices(int64_t m, int64_t n, int64_t k, int32_t* slices) {
    if (!slices || m < 0 || n < 0 || k < 0) {
        set_error("slices is NULL or a size is negative");
        return GB_ERR_INVALID_ARG;
    }
    *slices = default_emulated_slices(m, n, k);
    return GB_OK;
}

gb_status gb_tune_lookup_emulated(int slices, int64_t m, int64_t n, int64_t k, int32_t* tile) {
    if (m < 0 || n < 0 || k < 0) {
        set_error("a size is negative");
        return GB_ERR_INVALID_ARG;
    }
    const int s = slices == 0 ? default_emulated_slices(m, n, k) : slices;
    if (!tile || m < 0 || n < 0 || k < 0 || s < 1 || s > 16) {
        set_error("tile is NULL, a size is negative or slices is outside [0, 16]");
        return GB_ERR_INVALID_ARG;
    }
    *tile = lookup_emu(s, m, n, k);
    return GB_OK;
}

gb_status gb_grouped_workspace_size(const gb_gemm_desc* descs, int64_t count, size_t* out) {
    if (!out) {
        set_error("out is NULL");
        return GB_ERR_INVALID_ARG;
    }
    Layout L;
    gb_status st = build_layout(descs, count, L);
    if (st != GB_OK) return st;
    *out = L.total;
    return GB_OK;
}

static gb_status enqueue_plan(gb_grouped_plan* p, cudaStream_t stream,
                              const SplitFork* fk = nullptr) {
    const Launch L{stream, p->q->status, p->q->dev->sm_count};
    cudaError_t e = cudaSuccess;
    if (p->native_tiles > 0) {
        e = cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), stream);
        if (e == cudaSuccess)
            e = launch_grouped_native(L, p->d_native, p->n_native, p->native_tiles, p->d_counter,
                                      p->grid_native);
    }
    for (size_t r = 0; r < p->s_ranges.size() && e == cudaSuccess; ++r) {
        e = launch_grouped_split(L, p->d_emu, p->d_keys, p->s_ranges[r], fk);
        if (e == cudaSuccess) e = launch_grouped_products(L, p->d_emu, p->d_keys, p->s_ranges[r]);
    }
    if (e != cudaSuccess) return cuda_fail(e, "grouped launch");
    return GB_OK;
}

gb_status gb_grouped_plan_create(gb_queue* q, const gb_gemm_desc* descs, int64_t count,
                                 void* workspace, size_t workspace_bytes, int use_graph,
                                 gb_grouped_plan** out) {
    if (!q || !out) {
        set_error("queue or out is NULL");
        return GB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    Layout L;
    gb_status st = build_layout(descs, count, L);
    if (st != GB_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 || workspace_bytes < L.total) {
        set_error("grouped workspace missing, misaligned or below %zu bytes", L.total);
        return GB_ERR_WORKSPACE;
    }
    DeviceScope scope(q->dev->idx);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    size_t off = L.off_data;
    for (size_t i = 0; i < L.emu.size(); ++i) {
        const EmuLayout& w = L.emu_ws[i];
        emu_group_assign(L.emu[i], ws + off, w);
        off += w.total;
    }
    gb_grouped_plan* p = new (std::nothrow) gb_grouped_plan();
    if (!p) {
        set_error("out of host memory");
        return GB_ERR_INVALID_ARG;
    }
    p->q = q;
    p->use_graph = use_graph;
    p->d_counter = reinterpret_cast<unsigned long long*>(ws + L.off_counter);
    p->d_native = reinterpret_cast<GroupProb*>(ws + L.off_native);
    p->n_native = (int)L.native.size();
    p->native_tiles = 0;
    if (!L.native.empty()) {
        const GroupProb& last = L.native.back();
        p->native_tiles = last.first_tile +
                          ((last.m + tile_bm(last.tile) - 1) / tile_bm(last.tile)) * last.tiles_n;
    }
    p->d_emu = reinterpret_cast<EmuProb*>(ws + L.off_emu);
    p->d_keys = keys_at(ws, L);
    p->n_emu = (int)L.emu.size();
    p->emu_tiles = L.s_ranges.empty() ? 0 : L.s_ranges.back().t_end;
    p->max_s = L.max_s;
    p->s_ranges = L.s_ranges;
    p->flops = L.flops;
    const int occ = grouped_native_occupancy();
    int64_t grid = (int64_t)q->dev->sm_count * occ;
    if (grid > p->native_tiles) grid = p->native_tiles;
    p->grid_native = (int)(grid > 0 ? grid : 1);
    p->launches = (p->native_tiles > 0 ? 1 : 0) +
                  3 * (int)L.s_ranges.size();

    cudaError_t e = cudaSuccess;
    if (!L.native.empty())
        e = cudaMemcpyAsync(p->d_native, L.native.data(), sizeof(GroupProb) * L.native.size(),
                            cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess && !L.emu.empty())
        e = cudaMemcpyAsync(p->d_emu, L.emu.data(), sizeof(EmuProb) * L.emu.size(),
                            cudaMemcpyHostToDevice, q->stream);
    for (int a = 0; a < kEmuKeys && e == cudaSuccess && !L.emu.empty(); ++a)
        e = cudaMemcpyAsync(ws + L.off_keys[a], L.keys[a].data(), sizeof(int64_t) * L.emu.size(),
                            cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "uploading the grouped tables");
    }
    if (use_graph) {
        // captured with the split of A on a second stream beside that of B: in the
        // graph the two are parallel branches that join before the products
        cudaStream_t cs = nullptr;
        SplitFork fk{nullptr, nullptr, nullptr};
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&fk.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fk.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fk.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue_plan(p, cs, &fk);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (st == GB_OK && e2 == cudaSuccess) {
                p->graph = g;
                e = cudaGraphInstantiate(&p->exec, g, 0);
            } else {
                if (g) cudaGraphDestroy(g);
                if (st == GB_OK) e = e2;
            }
        }
        if (cs) cudaStreamDestroy(cs);
        if (fk.side) cudaStreamDestroy(fk.side);
        if (fk.fork) cudaEventDestroy(fk.fork);
        if (fk.join) cudaEventDestroy(fk.join);
        if (st != GB_OK || e != cudaSuccess) {
            if (p->exec) cudaGraphExecDestroy(p->exec);
            if (p->graph) cudaGraphDestroy(p->graph);
            delete p;
            return st != GB_OK ? st : cuda_fail(e, "capturing the grouped graph");
        }
    }
    *out = p;
    return GB_OK;
}

gb_status gb_grouped_plan_run(gb_grouped_plan* p) {
    if (!p) {
        set_error("plan is NULL");
        return GB_ERR_INVALID_ARG;
    }
    DeviceScope scope(p->q->dev->idx);
    if (p->use_graph) {
        cudaError_t e = cudaGraphLaunch(p->exec, p->q->stream);
        return finish_call(p->q, e, "grouped graph launch");
    }
    gb_status st = enqueue_plan(p, p->q->stream);
    if (st != GB_OK) return st;
    return finish_call(p->q, cudaSuccess, "grouped launch");
}

gb_status gb_grouped_plan_info(const gb_grouped_plan* p, int64_t* native_tiles,
                               int64_t* emulated_tiles, int* launches, double* flops) {
    if (!p) {
        set_error("plan is NULL");
        return GB_ERR_INVALID_ARG;
    }
    if (native_tiles) *native_tiles = p->native_tiles;
    if (emulated_tiles) *emulated_tiles = p->emu_tiles;
    if (launches) *launches = p->launches;
    if (flops) *flops = p->flops;
    return GB_OK;
}

gb_status gb_grouped_plan_destroy(gb_grouped_plan* p) {
    if (!p) return GB_OK;
    DeviceScope scope(p->q->dev->idx);
    cudaStreamSynchronize(p->q->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
    return GB_OK;
}

gb_status gb_dgemm_grouped(gb_queue* q, const gb_gemm_desc* descs, int64_t count,
                           void* workspace, size_t workspace_bytes) {
    gb_grouped_plan* p = nullptr;
    gb_status st = gb_grouped_plan_create(q, descs, count, workspace, workspace_bytes, 0, &p);
    if (st != GB_OK) return st;
    st = gb_grouped_plan_run(p);
    gb_grouped_plan_destroy(p);
    return st;
}

}  // extern "C"
