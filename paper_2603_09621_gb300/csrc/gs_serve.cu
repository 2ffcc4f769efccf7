// gs_serve.cu -- continuous-batching serving runtime: a best-fit host allocator over one
// device arena, admission by that budget, one stream per resident request, fitting steps in
// graph-captured chunks, bins grown between chunks when a step overflowed them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <iterator>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "gs_common.cuh"
#include "gs_serve.h"

// ------------------------------------------------------------------ arena
struct gs_arena {
    uintptr_t base = 0;
    size_t bytes = 0;
    size_t used = 0;
    size_t peak = 0;
    std::map<size_t, size_t> holes;  // offset -> size (sorted by offset, coalesced)
    std::map<size_t, size_t> live;   // offset -> size
};

namespace {

constexpr size_t kAlign = 256;
inline size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

extern "C" gs_status gs_arena_create(void* base, size_t bytes, gs_arena** out) {
    if (!base || !out) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(base) % kAlign != 0) return GS_ERR_INVALID_ARG;
    gs_arena* a = new (std::nothrow) gs_arena;
    if (!a) return GS_ERR_INVALID_ARG;
    a->base = reinterpret_cast<uintptr_t>(base);
    a->bytes = bytes / kAlign * kAlign;
    if (a->bytes) a->holes[0] = a->bytes;
    *out = a;
    return GS_OK;
}

extern "C" gs_status gs_arena_alloc(gs_arena* a, size_t bytes, void** out) {
    if (!a || !out || bytes == 0) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (bytes > a->bytes) return GS_ERR_CAPACITY;
    const size_t need = round_up(bytes);
    auto best = a->holes.end();
    for (auto it = a->holes.begin(); it != a->holes.end(); ++it)
        if (it->second >= need && (best == a->holes.end() || it->second < best->second)) best = it;
    if (best == a->holes.end()) return GS_ERR_CAPACITY;
    const size_t off = best->first, hole = best->second;
    a->holes.erase(best);
    if (hole > need) a->holes[off + need] = hole - need;
    a->live[off] = need;
    a->used += need;
    a->peak = std::max(a->peak, a->used);
    *out = reinterpret_cast<void*>(a->base + off);
    return GS_OK;
}

extern "C" gs_status gs_arena_alloc_top(gs_arena* a, size_t bytes, void** out) {
    if (!a || !out || bytes == 0) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (bytes > a->bytes) return GS_ERR_CAPACITY;
    const size_t need = round_up(bytes);
    for (auto it = a->holes.rbegin(); it != a->holes.rend(); ++it) {
        if (it->second < need) continue;
        const size_t hole_off = it->first, hole = it->second;
        const size_t off = hole_off + hole - need;
        if (hole > need)
            it->second = hole - need;
        else
            a->holes.erase(hole_off);
        a->live[off] = need;
        a->used += need;
        a->peak = std::max(a->peak, a->used);
        *out = reinterpret_cast<void*>(a->base + off);
        return GS_OK;
    }
    return GS_ERR_CAPACITY;
}

extern "C" gs_status gs_arena_free(gs_arena* a, void* p) {
    if (!a || !p) return GS_ERR_INVALID_ARG;
    const uintptr_t u = reinterpret_cast<uintptr_t>(p);
    if (u < a->base) return GS_ERR_INVALID_ARG;
    auto it = a->live.find(u - a->base);
    if (it == a->live.end()) return GS_ERR_INVALID_ARG;
    size_t off = it->first, len = it->second;
    a->live.erase(it);
    a->used -= len;
    auto nxt = a->holes.lower_bound(off);
    if (nxt != a->holes.end() && off + len == nxt->first) {  // merge with the following hole
        len += nxt->second;
        nxt = a->holes.erase(nxt);
    }
    if (nxt != a->holes.begin()) {  // merge with the preceding hole
        auto prv = std::prev(nxt);
        if (prv->first + prv->second == off) {
            prv->second += len;
            return GS_OK;
        }
    }
    a->holes[off] = len;
    return GS_OK;
}

extern "C" gs_status gs_arena_stats(const gs_arena* a, size_t* used, size_t* peak,
                                    size_t* largest_free, int64_t* n_live) {
    if (!a) return GS_ERR_INVALID_ARG;
    if (used) *used = a->used;
    if (peak) *peak = a->peak;
    if (largest_free) {
        size_t m = 0;
        for (const auto& h : a->holes) m = std::max(m, h.second);
        *largest_free = m;
    }
    if (n_live) *n_live = static_cast<int64_t>(a->live.size());
    return GS_OK;
}

extern "C" void gs_arena_destroy(gs_arena* a) { delete a; }

// ------------------------------------------------------------------ server
namespace {

using Clock = std::chrono::steady_clock;

// Host slot the end of every chunk copies into (pinned memory, one per stream).
struct Slot {
    int32_t status;
    int32_t step;
    int64_t npairs;
    float loss;
    int32_t pad[11];
};
static_assert(sizeof(Slot) == 64, "slot is one 64-byte line");

struct Sizes {
    size_t persist = 0;  // output: fitted params (fit) or volume I (render)
    size_t state = 0;    // fit: grad, m, v, I, W, lr_pred, lr_target, loss, step; render: W (+ params)
    size_t bins = 0;     // bins + workspace at the given capacity
};

struct Job {
    int64_t id = 0;
    gs_request req{};
    int32_t state = GS_REQ_PENDING;
    gs_status error = GS_OK;
    int32_t status_bits = 0;
    int32_t steps_done = 0;
    int32_t grows = 0;
    int32_t chunks = 0;
    int32_t bypassed = 0;
    float loss = 0.f;
    double admit_s = 0.0, done_s = 0.0;
    int64_t capacity = 0;
    int64_t need = 0;         // pairs needed after an overflow (0: none pending)
    bool inflight = false;
    int slot = -1;            // stream / event / host slot index while resident
    void* persist = nullptr;  // output block
    void* state_blk = nullptr;
    void* bins_blk = nullptr;
    size_t persist_bytes = 0, state_bytes = 0, bins_bytes = 0;
    gs_fit_state fs{};        // fit: the step state (pointers into the blocks)
    gs_bins bins{};
    void* ws = nullptr;
    size_t ws_bytes = 0;
    float* I = nullptr;
    float* W = nullptr;
    const float* render_params = nullptr;
    cudaGraphExec_t graph = nullptr;
};

struct Carver {
    char* p;
    size_t off = 0;
    explicit Carver(void* base) : p(static_cast<char*>(base)) {}
    void* take(size_t bytes) {
        void* r = p + off;
        off += round_up(bytes);
        return r;
    }
};

bool grid_ok(const gs_grid& g) {
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0) return false;
    for (int k = 0; k < 3; ++k)
        if (!(g.h[k] > 0.f) || !std::isfinite(g.h[k]) || !std::isfinite(g.origin[k])) return false;
    return true;
}

int64_t voxels(const gs_grid& g) { return int64_t(g.nx) * g.ny * g.nz; }

int64_t initial_capacity(const gs_server_config& c, int64_t n) {
    const double cap = std::ceil(double(c.pairs_per_gauss) * double(n)) + 4096.0;
    return static_cast<int64_t>(std::min(cap, double(gs::kMaxCapacity)));
}

size_t bins_block_bytes(const gs_server_config& c, int64_t n, int64_t cap, const gs_grid& g) {
    const size_t b = gs_bins_bytes(n, cap, &g, &c.cfg);
    const size_t w = gs_workspace_bytes(n, cap, &g, &c.cfg);
    if (!b || !w) return 0;
    return round_up(b) + round_up(w);
}

bool request_ok(const gs_request& r) {
    if (!grid_ok(r.grid) || r.n_gauss < 1 || !std::isfinite(r.arrival_s)) return false;
    if (r.kind == GS_REQ_FIT) {
        if (r.iters < 1 || !r.params || !r.lr_target) return false;
        if (r.lr_model == GS_LR_TRILINEAR)
            return r.lr_nx >= 1 && r.lr_ny >= 1 && r.lr_nz >= 1;
        return r.lr_model == GS_LR_ZBOX && r.s >= 1 && r.grid.nz / r.s >= 1;
    }
    if (r.kind == GS_REQ_RENDER) return r.source >= 0 || r.params;
    return false;
}

// Voxels of a fit request's LR scan.
size_t lr_voxels(const gs_request& r) {
    if (r.lr_model == GS_LR_TRILINEAR) return size_t(r.lr_nz) * r.lr_ny * r.lr_nx;
    return size_t(r.grid.nz / r.s) * r.grid.ny * r.grid.nx;
}

// Block sizes of a request at capacity `cap`; false if the request is invalid.
bool sizes_of(const gs_server_config& c, const gs_request& r, int64_t cap, Sizes* s) {
    if (!request_ok(r)) return false;
    const size_t pbytes = size_t(r.n_gauss) * 12 * sizeof(float);
    const size_t vbytes = size_t(voxels(r.grid)) * sizeof(float);
    s->bins = bins_block_bytes(c, r.n_gauss, cap, r.grid);
    if (!s->bins) return false;
    if (r.kind == GS_REQ_FIT) {
        const size_t lbytes = lr_voxels(r) * sizeof(float);
        s->persist = round_up(pbytes);
        s->state = 3 * round_up(pbytes) + 2 * round_up(vbytes) + 2 * round_up(lbytes) + 2 * kAlign;
    } else {
        s->persist = round_up(vbytes);
        s->state = round_up(vbytes) + (r.source < 0 ? round_up(pbytes) : 0);
    }
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct gs_server {
    gs_server_config cfg{};
    int device = 0;
    void* dmem = nullptr;
    gs_arena* arena = nullptr;
    Slot* host = nullptr;  // pinned [max_active]
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<int> free_slots;
    std::vector<Job> jobs;
    Clock::time_point t0;
    int64_t chunks_launched = 0, graphs_captured = 0, grows = 0;
    bool stuck = false;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void free_block(void*& p, size_t& bytes) {
        if (p) gs_arena_free(arena, p);
        p = nullptr;
        bytes = 0;
    }

    void drop_graph(Job& j) {
        if (j.graph) cudaGraphExecDestroy(j.graph);
        j.graph = nullptr;
    }

    // Leave residency: free the transient blocks and the stream slot (the output stays).
    void retire(Job& j, int32_t final_state, gs_status err) {
        // a failed launch may have left work queued that still uses the blocks
        if (j.slot >= 0) cudaStreamSynchronize(streams[j.slot]);
        drop_graph(j);
        free_block(j.state_blk, j.state_bytes);
        free_block(j.bins_blk, j.bins_bytes);
        if (final_state == GS_REQ_FAILED) free_block(j.persist, j.persist_bytes);
        if (j.slot >= 0) free_slots.push_back(j.slot);
        j.slot = -1;
        j.inflight = false;
        j.need = 0;
        j.state = final_state;
        j.error = err;
        j.done_s = now();
    }

    // Bind the bins and workspace of a request to its bins block at capacity j.capacity.
    gs_status bind_bins(Job& j) {
        const gs_grid& g = j.req.grid;
        const size_t b = gs_bins_bytes(j.req.n_gauss, j.capacity, &g, &cfg.cfg);
        gs_status s = gs_bins_bind(j.bins_blk, b, j.req.n_gauss, j.capacity, &g, &cfg.cfg, &j.bins);
        if (s != GS_OK) return s;
        j.ws = static_cast<char*>(j.bins_blk) + round_up(b);
        j.ws_bytes = j.bins_bytes - round_up(b);
        if (j.req.kind == GS_REQ_FIT) {
            j.fs.bins = j.bins;
            j.fs.ws = j.ws;
            j.fs.ws_bytes = j.ws_bytes;
        }
        return GS_OK;
    }

    // Replace the bins block by one for `cap` pairs. false if the arena has no room now.
    bool grow_to(Job& j, int64_t cap) {
        const size_t nb = bins_block_bytes(cfg, j.req.n_gauss, cap, j.req.grid);
        if (!nb) return false;
        void* blk = nullptr;
        if (gs_arena_alloc(arena, nb, &blk) != GS_OK) {
            // the old block's space may be what makes room: free it first, and take the old
            // size back if the new one still does not fit
            void* old = j.bins_blk;
            const size_t old_bytes = j.bins_bytes;
            gs_arena_free(arena, old);
            if (gs_arena_alloc(arena, nb, &blk) != GS_OK) {
                void* back = nullptr;
                gs_arena_alloc(arena, old_bytes, &back);  // cannot fail: the space was just freed
                j.bins_blk = back;
                bind_bins(j);
                drop_graph(j);
                return false;
            }
        } else {
            gs_arena_free(arena, j.bins_blk);
        }
        j.bins_blk = blk;
        j.bins_bytes = nb;
        j.capacity = cap;
        drop_graph(j);
        ++j.grows;
        ++grows;
        return bind_bins(j) == GS_OK;
    }

    bool admit(Job& j) {
        Sizes sz;
        j.capacity = initial_capacity(cfg, j.req.n_gauss);
        if (!sizes_of(cfg, j.req, j.capacity, &sz)) return false;
        if (gs_arena_alloc_top(arena, sz.persist, &j.persist) != GS_OK) return false;
        if (gs_arena_alloc(arena, sz.state, &j.state_blk) != GS_OK) {
            free_block(j.persist, sz.persist);
            return false;
        }
        if (gs_arena_alloc(arena, sz.bins, &j.bins_blk) != GS_OK) {
            free_block(j.state_blk, sz.state);
            free_block(j.persist, sz.persist);
            return false;
        }
        j.persist_bytes = sz.persist;
        j.state_bytes = sz.state;
        j.bins_bytes = sz.bins;
        j.slot = free_slots.back();
        free_slots.pop_back();
        j.state = GS_REQ_ACTIVE;
        j.admit_s = now();
        cudaStream_t st = streams[j.slot];
        const gs_grid& g = j.req.grid;
        const size_t pbytes = size_t(j.req.n_gauss) * 12 * sizeof(float);
        const size_t vbytes = size_t(voxels(g)) * sizeof(float);
        Carver c(j.state_blk);
        bool ok = true;
        if (j.req.kind == GS_REQ_FIT) {
            const size_t lbytes = lr_voxels(j.req) * sizeof(float);
            gs_fit_state& f = j.fs;
            f = gs_fit_state{};
            f.lr_model = j.req.lr_model;
            f.lr_nx = j.req.lr_nx;
            f.lr_ny = j.req.lr_ny;
            f.lr_nz = j.req.lr_nz;
            f.grid = g;
            f.cfg = cfg.cfg;
            f.adam = cfg.adam;
            f.n_gauss = j.req.n_gauss;
            f.s = j.req.s;
            f.params = static_cast<float*>(j.persist);
            f.grad = static_cast<float*>(c.take(pbytes));
            f.m = static_cast<float*>(c.take(pbytes));
            f.v = static_cast<float*>(c.take(pbytes));
            f.I = static_cast<float*>(c.take(vbytes));
            f.W = static_cast<float*>(c.take(vbytes));
            f.lr_pred = static_cast<float*>(c.take(lbytes));
            float* tgt = static_cast<float*>(c.take(lbytes));
            f.lr_target = tgt;
            f.d_loss = static_cast<float*>(c.take(sizeof(float)));
            f.d_step = static_cast<int32_t*>(c.take(sizeof(int32_t)));
            ok = cudaMemcpyAsync(f.params, j.req.params, pbytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(tgt, j.req.lr_target, lbytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemsetAsync(f.m, 0, pbytes, st) == cudaSuccess &&
                 cudaMemsetAsync(f.v, 0, pbytes, st) == cudaSuccess &&
                 cudaMemsetAsync(f.d_step, 0, sizeof(int32_t), st) == cudaSuccess &&
                 cudaMemsetAsync(f.d_loss, 0, sizeof(float), st) == cudaSuccess;
        } else {
            j.I = static_cast<float*>(j.persist);
            j.W = static_cast<float*>(c.take(vbytes));
            if (j.req.source >= 0) {
                j.render_params = static_cast<const float*>(jobs[j.req.source].persist);
            } else {
                float* p = static_cast<float*>(c.take(pbytes));
                ok = cudaMemcpyAsync(p, j.req.params, pbytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
                j.render_params = p;
            }
        }
        if (!ok || bind_bins(j) != GS_OK) {
            retire(j, GS_REQ_FAILED, ok ? GS_ERR_INVALID_ARG : GS_ERR_CUDA);
            return true;  // admitted and failed: the caller moves on
        }
        return true;
    }

    gs_status capture(Job& j) {
        cudaStream_t st = streams[j.slot];
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GS_ERR_CUDA;
        gs_status s = GS_OK;
        for (int k = 0; k < cfg.chunk_steps && s == GS_OK; ++k) s = gs_fit_step(&j.fs, st);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s == GS_OK && e != cudaSuccess) s = GS_ERR_CUDA;
        if (s == GS_OK && cudaGraphInstantiate(&j.graph, graph, 0) != cudaSuccess) {
            j.graph = nullptr;
            s = GS_ERR_CUDA;
        }
        if (graph) cudaGraphDestroy(graph);
        if (s == GS_OK) ++graphs_captured;
        return s;
    }

    gs_status launch(Job& j) {
        cudaStream_t st = streams[j.slot];
        Slot* h = host + j.slot;
        gs_status s = GS_OK;
        if (j.req.kind == GS_REQ_FIT) {
            const int n = std::min(cfg.chunk_steps, j.req.iters - j.steps_done);
            if (cfg.use_graphs && n == cfg.chunk_steps) {
                if (!j.graph) s = capture(j);
                if (s == GS_OK && cudaGraphLaunch(j.graph, st) != cudaSuccess) s = GS_ERR_CUDA;
            } else {
                for (int k = 0; k < n && s == GS_OK; ++k) s = gs_fit_step(&j.fs, st);
            }
            if (s == GS_OK &&
                (cudaMemcpyAsync(&h->step, j.fs.d_step, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(&h->loss, j.fs.d_loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess))
                s = GS_ERR_CUDA;
        } else {
            s = gs_bin_bricks(j.render_params, &j.req.grid, &cfg.cfg, &j.bins, j.ws, j.ws_bytes, st);
            if (s == GS_OK) s = gs_render_fwd(&j.bins, &j.req.grid, &cfg.cfg, j.I, j.W, nullptr, st);
        }
        if (s != GS_OK) return s;
        if (cudaMemcpyAsync(&h->status, j.bins.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&h->npairs, j.bins.d_npairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(events[j.slot], st) != cudaSuccess)
            return GS_ERR_CUDA;
        j.inflight = true;
        ++j.chunks;
        ++chunks_launched;
        return GS_OK;
    }

    // Collect a finished chunk. Returns true if the job left residency.
    bool collect(Job& j) {
        const Slot& h = host[j.slot];
        j.inflight = false;
        j.status_bits |= h.status;
        if (j.req.kind == GS_REQ_FIT) {
            j.steps_done = h.step;
            j.loss = h.loss;
        }
        if (h.status & GS_STATUS_CAPACITY) {
            if (h.npairs > gs::kMaxCapacity) {
                retire(j, GS_REQ_FAILED, GS_ERR_CAPACITY);
                return true;
            }
            j.need = std::max<int64_t>(h.npairs, j.capacity + 1);
            return false;
        }
        if (j.req.kind == GS_REQ_RENDER || j.steps_done >= j.req.iters) {
            retire(j, GS_REQ_DONE, GS_OK);
            return true;
        }
        return false;
    }

    bool source_ready(const Job& j, bool* failed) const {
        *failed = false;
        if (j.req.kind != GS_REQ_RENDER || j.req.source < 0) return true;
        const Job& src = jobs[j.req.source];
        if (src.state == GS_REQ_FAILED || (src.state == GS_REQ_DONE && !src.persist)) {
            *failed = true;
            return false;
        }
        return src.state == GS_REQ_DONE;
    }

    gs_status poll(bool* changed) {
        *changed = false;
        const double t = now();
        // 1. finished chunks
        for (Job& j : jobs) {
            if (j.state != GS_REQ_ACTIVE || !j.inflight) continue;
            const cudaError_t e = cudaEventQuery(events[j.slot]);
            if (e == cudaErrorNotReady) continue;
            *changed = true;
            if (e != cudaSuccess) {
                retire(j, GS_REQ_FAILED, GS_ERR_CUDA);
                continue;
            }
            collect(j);
        }
        // 2. bins to grow
        int n_active = 0, n_stalled = 0;
        Job* newest_stalled = nullptr;
        for (Job& j : jobs) {
            if (j.state != GS_REQ_ACTIVE) continue;
            ++n_active;
            if (j.need > 0 && !j.inflight) {
                const int64_t cap = std::min<int64_t>(gs::kMaxCapacity, j.need + j.need / 8 + 4096);
                if (grow_to(j, cap)) {
                    j.need = 0;
                    *changed = true;
                } else {
                    ++n_stalled;
                    if (!newest_stalled || j.admit_s >= newest_stalled->admit_s) newest_stalled = &j;
                }
            }
        }
        bool any_inflight = false;
        for (const Job& j : jobs) any_inflight |= (j.state == GS_REQ_ACTIVE && j.inflight);
        if (n_stalled && n_stalled == n_active && !any_inflight) {
            // every resident request waits for room that only its peers hold: give up the newest
            retire(*newest_stalled, GS_REQ_FAILED, GS_ERR_CAPACITY);
            *changed = true;
            --n_active;
        }
        // 3. admission in arrival order, with bounded overtaking of the oldest blocked request
        std::vector<Job*> waiting;
        for (Job& j : jobs) {
            if (j.state != GS_REQ_PENDING || j.req.arrival_s > t) continue;
            bool failed = false;
            if (!source_ready(j, &failed)) {
                if (failed) {
                    j.state = GS_REQ_FAILED;
                    j.error = GS_ERR_INVALID_ARG;
                    j.done_s = t;
                    *changed = true;
                }
                continue;
            }
            waiting.push_back(&j);
        }
        std::stable_sort(waiting.begin(), waiting.end(),
                         [](const Job* a, const Job* b) { return a->req.arrival_s < b->req.arrival_s; });
        Job* blocked = nullptr;
        int admitted = 0;
        for (Job* j : waiting) {
            if (free_slots.empty()) break;
            if (blocked && blocked->bypassed >= cfg.max_bypass) break;
            if (admit(*j)) {
                *changed = true;
                ++admitted;
                if (blocked) ++blocked->bypassed;
            } else if (!blocked) {
                blocked = j;
            }
        }
        // nothing resident and nothing admitted although requests wait: only releasing
        // finished outputs can make room
        stuck = blocked && admitted == 0 && n_active == 0;
        // 4. next chunk of every idle resident request
        for (Job& j : jobs) {
            if (j.state != GS_REQ_ACTIVE || j.inflight || j.need > 0) continue;
            const gs_status s = launch(j);
            *changed = true;
            if (s != GS_OK) retire(j, GS_REQ_FAILED, s);
        }
        return stuck ? GS_ERR_CAPACITY : GS_OK;
    }

    int32_t unfinished() const {
        int32_t n = 0;
        for (const Job& j : jobs) n += (j.state == GS_REQ_PENDING || j.state == GS_REQ_ACTIVE);
        return n;
    }
};

extern "C" size_t gs_server_request_bytes(const gs_server_config* cfg, const gs_request* req) {
    if (!cfg || !req) return 0;
    Sizes s;
    if (!sizes_of(*cfg, *req, initial_capacity(*cfg, req->n_gauss), &s)) return 0;
    return s.persist + s.state + s.bins;
}

extern "C" gs_status gs_server_create(const gs_server_config* cfg, gs_server** out) {
    if (!cfg || !out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->hbm_budget < kAlign || cfg->max_active < 1 || cfg->max_active > 64 ||
        cfg->chunk_steps < 1 || cfg->max_bypass < 0 || !(cfg->pairs_per_gauss > 0.f) ||
        !std::isfinite(cfg->pairs_per_gauss))
        return GS_ERR_INVALID_ARG;
    if (!(cfg->adam.beta1 >= 0.0 && cfg->adam.beta1 < 1.0 && cfg->adam.beta2 >= 0.0 &&
          cfg->adam.beta2 < 1.0 && cfg->adam.eps > 0.0))
        return GS_ERR_INVALID_ARG;
    gs_server* sv = new (std::nothrow) gs_server;
    if (!sv) return GS_ERR_INVALID_ARG;
    sv->cfg = *cfg;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return GS_ERR_CUDA;
    }
    bool ok = cudaMalloc(&sv->dmem, cfg->hbm_budget) == cudaSuccess &&
              gs_arena_create(sv->dmem, cfg->hbm_budget, &sv->arena) == GS_OK &&
              cudaHostAlloc(reinterpret_cast<void**>(&sv->host), sizeof(Slot) * cfg->max_active,
                            cudaHostAllocDefault) == cudaSuccess;
    for (int i = 0; ok && i < cfg->max_active; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) sv->streams.push_back(s);
        ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) sv->events.push_back(e);
    }
    if (!ok) {
        cudaGetLastError();
        gs_server_destroy(sv);
        return GS_ERR_CUDA;
    }
    for (int i = cfg->max_active - 1; i >= 0; --i) sv->free_slots.push_back(i);
    sv->t0 = Clock::now();
    *out = sv;
    return GS_OK;
}

extern "C" gs_status gs_server_submit(gs_server* sv, const gs_request* req, int64_t* id) {
    if (!sv || !req || !id) return GS_ERR_INVALID_ARG;
    Sizes s;
    if (!sizes_of(sv->cfg, *req, initial_capacity(sv->cfg, req->n_gauss), &s)) return GS_ERR_INVALID_ARG;
    if (req->kind == GS_REQ_RENDER && req->source >= 0) {
        if (req->source >= static_cast<int64_t>(sv->jobs.size())) return GS_ERR_INVALID_ARG;
        const Job& src = sv->jobs[req->source];
        if (src.req.kind != GS_REQ_FIT || src.req.n_gauss != req->n_gauss) return GS_ERR_INVALID_ARG;
    }
    if (s.persist + s.state + s.bins > sv->arena->bytes) return GS_ERR_CAPACITY;
    Job j;
    j.id = static_cast<int64_t>(sv->jobs.size());
    j.req = *req;
    sv->jobs.push_back(j);
    *id = j.id;
    return GS_OK;
}

extern "C" gs_status gs_server_poll(gs_server* sv, int32_t* n_unfinished) {
    if (!sv) return GS_ERR_INVALID_ARG;
    DeviceGuard guard(sv->device);
    bool changed = false;
    const gs_status s = sv->poll(&changed);
    if (n_unfinished) *n_unfinished = sv->unfinished();
    return s;
}

extern "C" gs_status gs_server_run(gs_server* sv, double timeout_s, int32_t poll_us) {
    if (!sv || !(timeout_s >= 0.0) || poll_us < 0) return GS_ERR_INVALID_ARG;
    DeviceGuard guard(sv->device);
    const auto t_end = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
    for (;;) {
        bool changed = false;
        const gs_status s = sv->poll(&changed);
        if (s != GS_OK) return s;
        if (sv->unfinished() == 0) return GS_OK;
        if (Clock::now() >= t_end) return GS_ERR_TIMEOUT;
        if (!changed && poll_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(poll_us));
    }
}

extern "C" gs_status gs_server_result(const gs_server* sv, int64_t id, gs_result* out) {
    if (!sv || !out || id < 0 || id >= static_cast<int64_t>(sv->jobs.size())) return GS_ERR_INVALID_ARG;
    const Job& j = sv->jobs[id];
    gs_result r{};
    r.state = j.state;
    r.error = j.error;
    r.status_bits = j.status_bits;
    r.steps_done = j.steps_done;
    r.capacity = j.capacity;
    r.grows = j.grows;
    r.chunks = j.chunks;
    r.loss = j.loss;
    r.arrival_s = j.req.arrival_s;
    r.admit_s = j.admit_s;
    r.done_s = j.done_s;
    r.output = (j.state == GS_REQ_DONE) ? j.persist : nullptr;
    r.bytes = j.persist_bytes + j.state_bytes + j.bins_bytes;
    *out = r;
    return GS_OK;
}

extern "C" gs_status gs_server_release(gs_server* sv, int64_t id) {
    if (!sv || id < 0 || id >= static_cast<int64_t>(sv->jobs.size())) return GS_ERR_INVALID_ARG;
    Job& j = sv->jobs[id];
    if (j.state != GS_REQ_DONE && j.state != GS_REQ_FAILED) return GS_ERR_INVALID_ARG;
    for (const Job& d : sv->jobs)
        if (d.req.kind == GS_REQ_RENDER && d.req.source == id &&
            (d.state == GS_REQ_PENDING || d.state == GS_REQ_ACTIVE))
            return GS_ERR_INVALID_ARG;
    sv->free_block(j.persist, j.persist_bytes);
    return GS_OK;
}

extern "C" gs_status gs_server_stats_read(const gs_server* sv, gs_server_stats* out) {
    if (!sv || !out) return GS_ERR_INVALID_ARG;
    gs_server_stats s{};
    s.now_s = sv->now();
    for (const Job& j : sv->jobs) {
        s.n_pending += j.state == GS_REQ_PENDING;
        s.n_active += j.state == GS_REQ_ACTIVE;
        s.n_done += j.state == GS_REQ_DONE;
        s.n_failed += j.state == GS_REQ_FAILED;
    }
    s.arena_bytes = sv->arena ? sv->arena->bytes : 0;
    if (sv->arena) gs_arena_stats(sv->arena, &s.used_bytes, &s.peak_bytes, nullptr, nullptr);
    s.chunks_launched = sv->chunks_launched;
    s.graphs_captured = sv->graphs_captured;
    s.grows = sv->grows;
    *out = s;
    return GS_OK;
}

extern "C" void gs_server_destroy(gs_server* sv) {
    if (!sv) return;
    {
        DeviceGuard guard(sv->device);
        for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
        for (Job& j : sv->jobs) sv->drop_graph(j);
        for (cudaEvent_t e : sv->events) cudaEventDestroy(e);
        for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
        if (sv->host) cudaFreeHost(sv->host);
        if (sv->dmem) cudaFree(sv->dmem);
        gs_arena_destroy(sv->arena);
    }
    delete sv;
}
