// gs_volume.cu -- slice-profile forward model (box average of s slices along z), its
// adjoint, the deterministic L1 loss, the fused fitting step and the small host utilities of
// the C ABI.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include <atomic>

#include "gs_common.cuh"

namespace gs {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

__global__ void __launch_bounds__(256) k_downsample_fwd(const float* __restrict__ hr, int ny, int nx,
                                                        int nzl, int s, float inv_s,
                                                        float* __restrict__ lr) {
    pdl_enter();
    const int64_t plane = int64_t(ny) * nx;
    const int64_t n = plane * nzl;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = i / plane, r = i - k * plane;
        const float* src = hr + (k * s) * plane + r;
        float acc = 0.f;
        for (int j = 0; j < s; ++j) acc += src[j * plane];
        lr[i] = acc * inv_s;
    }
}

__global__ void __launch_bounds__(256) k_downsample_bwd(const float* __restrict__ dlr, int nz, int ny,
                                                        int nx, int s, float inv_s,
                                                        float* __restrict__ dhr) {
    pdl_enter();
    const int64_t plane = int64_t(ny) * nx;
    const int64_t n = plane * nz;
    const int zmax = s * (nz / s);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t z = i / plane, r = i - z * plane;
        dhr[i] = (z < zmax) ? dlr[(z / s) * plane + r] * inv_s : 0.0f;
    }
}

// Stage 1: fixed grid of kL1Blocks blocks; each thread sums |pred - target| over a fixed
// stride, then a fixed-shape block tree. Optionally writes sign(pred - target) / n.
__global__ void __launch_bounds__(256) k_l1_partial(const float* __restrict__ pred,
                                                    const float* __restrict__ target, int64_t n,
                                                    float inv_n, float* __restrict__ dpred,
                                                    float* __restrict__ partials) {
    pdl_enter();
    __shared__ float sm[256];
    float acc = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float d = pred[i] - target[i];
        acc += fabsf(d);
        if (dpred) dpred[i] = (d > 0.f) ? inv_n : ((d < 0.f) ? -inv_n : 0.f);
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(1024) k_l1_final(const float* __restrict__ partials, float inv_n,
                                                   float* __restrict__ loss) {
    pdl_enter();
    __shared__ float sm[kL1Blocks];
    sm[threadIdx.x] = partials[threadIdx.x];
    __syncthreads();
    for (int o = kL1Blocks / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sm[0] * inv_n;
}

static unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    return static_cast<unsigned>(b < 65536 ? b : 65536);
}

// The slice profile and its adjoint-factor kernel over a 2D grid (blockIdx.y = LR or HR
// slice) with four voxels per thread, for planes of a multiple of 4 voxels and at most 65,535 slices: no index division
// per voxel, 16-byte accesses. Same arithmetic, same results.
__global__ void __launch_bounds__(256) k_downsample_fwd4(const float4* __restrict__ hr, int plane4,
                                                         int s, float inv_s,
                                                         float4* __restrict__ lr) {
    pdl_enter();
    const int k = blockIdx.y;
    const float4* src = hr + int64_t(k) * s * plane4;
    float4* dst = lr + int64_t(k) * plane4;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < plane4; r += gridDim.x * blockDim.x) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < s; ++j) {
            const float4 v = src[int64_t(j) * plane4 + r];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        dst[r] = make_float4(acc.x * inv_s, acc.y * inv_s, acc.z * inv_s, acc.w * inv_s);
    }
}

__device__ __forceinline__ float2 adj_factor(float gI, float w, float iv, float eps) {
    const float al = gI / (w > eps ? w : eps);
    return make_float2(al, (w > eps) ? al * iv : 0.0f);
}

__global__ void __launch_bounds__(256) k_profile_adj_prep4(const float4* __restrict__ dlr,
                                                           const float4* __restrict__ Iv,
                                                           const float4* __restrict__ Wv,
                                                           int plane4, int zmax, int s, float inv_s,
                                                           float eps, float4* __restrict__ aip) {
    pdl_enter();
    const int z = blockIdx.y;
    const bool in = z < zmax;
    const int64_t base = int64_t(z) * plane4;
    const float4* g4 = dlr + int64_t(in ? z / s : 0) * plane4;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < plane4; r += gridDim.x * blockDim.x) {
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) {
            const float4 d = g4[r];
            g = make_float4(d.x * inv_s, d.y * inv_s, d.z * inv_s, d.w * inv_s);
        }
        const float4 w = Wv[base + r], iv = Iv[base + r];
        const float2 a0 = adj_factor(g.x, w.x, iv.x, eps), a1 = adj_factor(g.y, w.y, iv.y, eps);
        const float2 a2 = adj_factor(g.z, w.z, iv.z, eps), a3 = adj_factor(g.w, w.w, iv.w, eps);
        aip[2 * (base + r)] = make_float4(a0.x, a0.y, a1.x, a1.y);
        aip[2 * (base + r) + 1] = make_float4(a2.x, a2.y, a3.x, a3.y);
    }
}

static dim3 grid2d(int plane4, int slices) {
    const int bx = (plane4 + 255) / 256;
    return dim3(static_cast<unsigned>(bx < 64 ? bx : 64), static_cast<unsigned>(slices));
}

static bool vec_ok(const void* a, const void* b, int64_t plane, int slices) {
    return plane % 4 == 0 && slices <= 65535 && reinterpret_cast<uintptr_t>(a) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(b) % 16 == 0;
}

gs_status launch_l1(const float* pred, const float* target, int64_t n, float* d_loss, float* dpred,
                    float* partials, cudaStream_t st, int64_t n_norm) {
    // the mean's normaliser: n, or n_norm > 0 when these values are one part of a larger mean
    const int64_t nn = n_norm > 0 ? n_norm : n;
    const float inv_n = nn > 0 ? 1.0f / float(nn) : 0.0f;
    launch_k(k_l1_partial, dim3(kL1Blocks), dim3(256), 0, st, pred, target, n, inv_n, dpred,
        partials);
    gs_status s = last_launch_status();
    if (s != GS_OK) return s;
    launch_k(k_l1_final, dim3(1), dim3(kL1Blocks), 0, st, partials, inv_n, d_loss);
    return last_launch_status();
}

gs_status downsample_fwd_impl(const float* hr, int nz, int ny, int nx, int s, float* lr,
                              cudaStream_t st) {
    const int nzl = nz / s;
    const int64_t n = int64_t(nzl) * ny * nx;
    if (n == 0) return GS_OK;
    const int64_t plane = int64_t(ny) * nx;
    if (vec_ok(hr, lr, plane, nzl) && plane / 4 <= (int64_t(1) << 30)) {
        const int plane4 = static_cast<int>(plane / 4);
        launch_k(k_downsample_fwd4, dim3(grid2d(plane4, nzl)), dim3(256), 0, st,
            reinterpret_cast<const float4*>(hr), plane4, s, 1.0f / float(s),
            reinterpret_cast<float4*>(lr));
    } else {
        launch_k(k_downsample_fwd, dim3(grid_for(n)), dim3(256), 0, st, hr, ny, nx, nzl, s,
            1.0f / float(s), lr);
    }
    return last_launch_status();
}

gs_status downsample_bwd_impl(const float* dlr, int nz, int ny, int nx, int s, float* dhr,
                              cudaStream_t st) {
    const int64_t n = int64_t(nz) * ny * nx;
    launch_k(k_downsample_bwd, dim3(grid_for(n)), dim3(256), 0, st, dlr, nz, ny, nx, s,
        1.0f / float(s), dhr);
    return last_launch_status();
}

// Provided by the other translation units.
gs_status bind_workspace(void* base, size_t bytes, int64_t n_gauss, int64_t capacity,
                         const gs_grid* grid, const gs_config* cfg, Workspace* ws);
bool bins_match(const gs_bins* b, const gs_grid* grid, const gs_config* cfg);
gs_status bin_bricks_impl(const float* params, const gs_grid* grid, const gs_config* cfg,
                          gs_bins* bins, const Workspace& ws, cudaStream_t st);
gs_status render_fwd_impl(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg, float* I,
                          float* W, unsigned long long* stats, cudaStream_t st);
gs_status launch_adjoint_pairs(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                               const Workspace& ws, cudaStream_t st);
gs_status launch_chain_adam(float* params, float* grad, float* m, float* v, const float* part,
                            const float* gacc, const gs_bins* bins, int64_t n,
                            const gs_grid* grid, const gs_config* cfg, const gs_adam* hp,
                            int32_t* d_step, cudaStream_t st);

// Slice-profile adjoint fused with the adjoint render's per-voxel factors: for each HR voxel
// dL/dI = dL/dLR[z / s] / s (0 below the last full slab), alpha = dL/dI / max(W, eps) and
// I' = I where W > eps, else 0; stored as (alpha, alpha I').
__global__ void __launch_bounds__(256) k_profile_adj_prep(const float* __restrict__ dlr,
                                                          const float* __restrict__ Iv,
                                                          const float* __restrict__ Wv, int nz,
                                                          int ny, int nx, int s, float inv_s,
                                                          float eps, float2* __restrict__ aip) {
    pdl_enter();
    const int64_t plane = int64_t(ny) * nx;
    const int64_t n = plane * nz;
    const int zmax = s * (nz / s);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t z = i / plane, r = i - z * plane;
        const float gI = (z < zmax) ? dlr[(z / s) * plane + r] * inv_s : 0.0f;
        const float w = Wv[i];
        const float al = gI / (w > eps ? w : eps);
        aip[i] = make_float2(al, (w > eps) ? al * Iv[i] : 0.0f);
    }
}

}  // namespace gs

using namespace gs;

static bool vol_args_ok(const void* a, const void* b, int32_t nz, int32_t ny, int32_t nx, int32_t s) {
    return a && b && nz > 0 && ny > 0 && nx > 0 && s > 0 &&
           int64_t(nz) * ny * nx <= (int64_t(1) << 31) - 1;
}

extern "C" gs_status gs_downsample_fwd(const float* hr, int32_t nz, int32_t ny, int32_t nx,
                                       int32_t s, float* lr, gs_stream stream) {
    if (!vol_args_ok(hr, lr, nz, ny, nx, s)) return GS_ERR_INVALID_ARG;
    return downsample_fwd_impl(hr, nz, ny, nx, s, lr, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_downsample_bwd(const float* dlr, int32_t nz, int32_t ny, int32_t nx,
                                       int32_t s, float* dhr, gs_stream stream) {
    if (!vol_args_ok(dlr, dhr, nz, ny, nx, s)) return GS_ERR_INVALID_ARG;
    return downsample_bwd_impl(dlr, nz, ny, nx, s, dhr, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_l1_loss(const float* pred, const float* target, int64_t n, float* d_loss,
                                float* dpred, void* ws, size_t ws_bytes, gs_stream stream) {
    if (!pred || !target || !d_loss || !ws || n <= 0) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return GS_ERR_INVALID_ARG;
    if (ws_bytes < sizeof(float) * kL1Blocks) return GS_ERR_WORKSPACE;
    return launch_l1(pred, target, n, d_loss, dpred, static_cast<float*>(ws),
                     reinterpret_cast<cudaStream_t>(stream));
}

namespace {

// One fitting iteration's common part: validation, workspace and phase events.
struct FitRun {
    gs_fit_state* st = nullptr;
    Workspace w = {};
    cudaStream_t cs = nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaEvent_t lr_ready = nullptr;  // if set: the LR target is ready when this event is

    // Phase events: during stream capture they must be external event-record nodes, or they
    // would only serve as capture-internal dependencies.
    bool mark(int phase) const {
        if (!st->n_phase_events) return true;
        cudaEvent_t ev = static_cast<cudaEvent_t>(st->phase_events[phase]);
        if (cap == cudaStreamCaptureStatusActive)
            return cudaEventRecordWithFlags(ev, cs, cudaEventRecordExternal) == cudaSuccess;
        return cudaEventRecord(ev, cs) == cudaSuccess;
    }
};

gs_status fit_prepare(gs_fit_state* st, gs_stream stream, FitRun* run) {
    if (!st) return GS_ERR_INVALID_ARG;
    gs_status s = validate_grid_cfg(&st->grid, &st->cfg);
    if (s != GS_OK) return s;
    if (st->n_gauss <= 0) return GS_ERR_INVALID_ARG;
    const bool trilinear = st->lr_model == GS_LR_TRILINEAR;
    if (trilinear) {
        const int32_t lim = 1 << 23;
        if (st->lr_nx <= 0 || st->lr_ny <= 0 || st->lr_nz <= 0 || st->lr_nx >= lim ||
            st->lr_ny >= lim || st->lr_nz >= lim || st->grid.nx >= lim || st->grid.ny >= lim ||
            st->grid.nz >= lim)
            return GS_ERR_INVALID_ARG;
    } else if (st->lr_model != GS_LR_ZBOX || st->s <= 0 || st->grid.nz / st->s <= 0) {
        return GS_ERR_INVALID_ARG;
    }
    if (!st->params || !st->grad || !st->m || !st->v || !st->d_step || !st->I || !st->W ||
        !st->lr_pred || !st->lr_target || !st->d_loss)
        return GS_ERR_INVALID_ARG;
    if (!bins_match(&st->bins, &st->grid, &st->cfg) || st->bins.n_gauss != st->n_gauss)
        return GS_ERR_INVALID_ARG;
    s = bind_workspace(st->ws, st->ws_bytes, st->n_gauss, st->bins.capacity, &st->grid, &st->cfg,
                       &run->w);
    if (s != GS_OK) return s;
    if (st->n_phase_events != 0 && (st->n_phase_events != GS_FIT_PHASES || !st->phase_events))
        return GS_ERR_INVALID_ARG;
    run->st = st;
    run->cs = reinterpret_cast<cudaStream_t>(stream);
    if (st->n_phase_events && cudaStreamIsCapturing(run->cs, &run->cap) != cudaSuccess)
        return GS_ERR_CUDA;
    return GS_OK;
}

// Bin, render, LR forward model, L1 (normalised by n_norm LR values when n_norm > 0, else by
// the state's own count), its adjoint with the adjoint render's per-voxel factors, and the
// adjoint render kernel; phase events 0-4.
gs_status fit_front(const FitRun& run, int64_t n_norm) {
    gs_fit_state* st = run.st;
    const Workspace& w = run.w;
    cudaStream_t cs = run.cs;
    const bool trilinear = st->lr_model == GS_LR_TRILINEAR;
    const gs_grid& g = st->grid;
    if (!run.mark(0)) return GS_ERR_CUDA;
    gs_status s = bin_bricks_impl(st->params, &g, &st->cfg, &st->bins, w, cs);
    if (s != GS_OK) return s;
    if (!run.mark(1)) return GS_ERR_CUDA;
    s = render_fwd_impl(&st->bins, &g, &st->cfg, st->I, st->W, nullptr, cs);
    if (s != GS_OK) return s;
    if (!run.mark(2)) return GS_ERR_CUDA;
    if (run.lr_ready && cudaStreamWaitEvent(cs, run.lr_ready, 0) != cudaSuccess) return GS_ERR_CUDA;
    if (trilinear)
        s = resample_fwd_impl(st->I, g.nz, g.ny, g.nx, st->lr_pred, st->lr_nz, st->lr_ny, st->lr_nx, cs);
    else
        s = downsample_fwd_impl(st->I, g.nz, g.ny, g.nx, st->s, st->lr_pred, cs);
    if (s != GS_OK) return s;
    const int64_t n_lr = trilinear ? int64_t(st->lr_nz) * st->lr_ny * st->lr_nx
                                   : int64_t(g.nz / st->s) * g.ny * g.nx;
    // L1 loss; its gradient overwrites lr_pred in place.
    s = launch_l1(st->lr_pred, st->lr_target, n_lr, st->d_loss, st->lr_pred, w.l1_part, cs, n_norm);
    if (s != GS_OK) return s;
    if (trilinear) {
        s = resample_adj_prep_impl(st->lr_pred, st->lr_nz, st->lr_ny, st->lr_nx, st->I, st->W, g.nz,
                                   g.ny, g.nx, st->cfg.eps, w.aip, cs);
        if (s != GS_OK) return s;
    } else {
        const int64_t nv = int64_t(g.nz) * g.ny * g.nx;
        const int64_t plane = int64_t(g.ny) * g.nx;
        if (vec_ok(st->lr_pred, st->I, plane, g.nz) && vec_ok(st->W, w.aip, plane, g.nz) &&
            plane / 4 <= (int64_t(1) << 30)) {
            const int plane4 = static_cast<int>(plane / 4);
            launch_k(k_profile_adj_prep4, dim3(grid2d(plane4, g.nz)), dim3(256), 0, cs,
                reinterpret_cast<const float4*>(st->lr_pred),
                reinterpret_cast<const float4*>(st->I), reinterpret_cast<const float4*>(st->W),
                plane4, st->s * (g.nz / st->s), st->s, 1.0f / float(st->s), st->cfg.eps,
                reinterpret_cast<float4*>(w.aip));
        } else {
            launch_k(k_profile_adj_prep, dim3(grid_for(nv)), dim3(256), 0, cs, st->lr_pred, st->I,
                st->W, g.nz, g.ny, g.nx, st->s, 1.0f / float(st->s), st->cfg.eps, w.aip);
        }
        s = last_launch_status();
        if (s != GS_OK) return s;
    }
    if (!run.mark(3)) return GS_ERR_CUDA;
    s = launch_adjoint_pairs(&st->bins, &g, &st->cfg, w, cs);
    if (s != GS_OK) return s;
    if (!run.mark(4)) return GS_ERR_CUDA;
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_fit_step(gs_fit_state* st, gs_stream stream) {
    FitRun run;
    gs_status s = fit_prepare(st, stream, &run);
    if (s != GS_OK) return s;
    s = fit_front(run, 0);
    if (s != GS_OK) return s;
    s = launch_chain_adam(st->params, st->grad, st->m, st->v, run.w.part, run.w.gacc, &st->bins,
                          st->n_gauss, &st->grid, &st->cfg, &st->adam, st->d_step, run.cs);
    if (s != GS_OK) return s;
    if (!run.mark(5)) return GS_ERR_CUDA;
    if (!run.mark(6)) return GS_ERR_CUDA;
    return GS_OK;
}

namespace {

// Per-device side stream and events of gs_fit_step_host, created once with that device current.
struct HostCopyRes {
    cudaStream_t side = nullptr;
    cudaEvent_t entry = nullptr, lr_done = nullptr;
};
constexpr int kMaxHostDevices = 64;
std::mutex g_host_res_mutex;
HostCopyRes g_host_res[kMaxHostDevices];

gs_status host_copy_res(HostCopyRes** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxHostDevices) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_host_res_mutex);
    HostCopyRes& r = g_host_res[dev];
    if (!r.side) {
        if (cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.entry, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.lr_done, cudaEventDisableTiming) != cudaSuccess)
            return GS_ERR_CUDA;
    }
    *out = &r;
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_fit_step_host(gs_fit_state* st, const float* h_params,
                                      const float* h_lr_target, float* h_loss, gs_stream stream) {
    if (!st || st->n_gauss <= 0 || !st->params || !st->lr_target || !st->d_loss)
        return GS_ERR_INVALID_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_lr = st->lr_model == GS_LR_TRILINEAR
                             ? int64_t(st->lr_nz) * st->lr_ny * st->lr_nx
                             : (st->s > 0 ? int64_t(st->grid.nz / st->s) * st->grid.ny * st->grid.nx : 0);
    if (n_lr <= 0) return GS_ERR_INVALID_ARG;
    FitRun run;
    gs_status s = fit_prepare(st, stream, &run);
    if (s != GS_OK) return s;
    // The parameters go first, alone on the link, since binning waits for them; the LR target
    // follows on a side stream while the step bins and renders, and the step waits for it
    // only before the LR model. The side stream starts after everything issued on `stream`
    // so far (the parameter copy included), so an earlier step still reading lr_target is
    // not overwritten.
    if (h_params && cudaMemcpyAsync(st->params, h_params, sizeof(float) * 12 * st->n_gauss,
                                    cudaMemcpyHostToDevice, cs) != cudaSuccess)
        return GS_ERR_CUDA;
    if (h_lr_target) {
        HostCopyRes* r = nullptr;
        s = host_copy_res(&r);
        if (s != GS_OK) return s;
        if (cudaEventRecord(r->entry, cs) != cudaSuccess ||
            cudaStreamWaitEvent(r->side, r->entry, 0) != cudaSuccess ||
            cudaMemcpyAsync(const_cast<float*>(st->lr_target), h_lr_target, sizeof(float) * n_lr,
                            cudaMemcpyHostToDevice, r->side) != cudaSuccess ||
            cudaEventRecord(r->lr_done, r->side) != cudaSuccess)
            return GS_ERR_CUDA;
        run.lr_ready = r->lr_done;
    }
    s = fit_front(run, 0);
    if (s != GS_OK) return s;
    s = launch_chain_adam(st->params, st->grad, st->m, st->v, run.w.part, run.w.gacc, &st->bins,
                          st->n_gauss, &st->grid, &st->cfg, &st->adam, st->d_step, cs);
    if (s != GS_OK) return s;
    if (!run.mark(5) || !run.mark(6)) return GS_ERR_CUDA;
    if (h_loss && cudaMemcpyAsync(h_loss, st->d_loss, sizeof(float), cudaMemcpyDeviceToHost,
                                  cs) != cudaSuccess)
        return GS_ERR_CUDA;
    return GS_OK;
}

extern "C" gs_status gs_fit_grad(gs_fit_state* st, int64_t n_lr_total, gs_stream stream) {
    if (n_lr_total < 0) return GS_ERR_INVALID_ARG;
    FitRun run;
    gs_status s = fit_prepare(st, stream, &run);
    if (s != GS_OK) return s;
    s = fit_front(run, n_lr_total);
    if (s != GS_OK) return s;
    s = launch_chain_grad(st->params, st->grad, run.w.part, run.w.gacc, &st->bins, st->n_gauss,
                          &st->grid, &st->cfg, run.cs);
    if (s != GS_OK) return s;
    if (!run.mark(5)) return GS_ERR_CUDA;
    if (!run.mark(6)) return GS_ERR_CUDA;
    return GS_OK;
}

extern "C" gs_status gs_fit_apply(gs_fit_state* st, const int32_t* d_skip, gs_stream stream) {
    if (!st || st->n_gauss <= 0 || !st->params || !st->grad || !st->m || !st->v || !st->d_step)
        return GS_ERR_INVALID_ARG;
    return launch_adam(st->params, st->grad, st->m, st->v, st->n_gauss, &st->adam, st->d_step,
                       d_skip, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_status_read(const int32_t* d_status, int32_t* h_status, gs_stream stream) {
    if (!d_status || !h_status) return GS_ERR_INVALID_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h_status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(cs) != cudaSuccess) return GS_ERR_CUDA;
    if (*h_status & GS_STATUS_CAPACITY) return GS_ERR_CAPACITY;
    if (*h_status & GS_STATUS_NONFINITE) return GS_ERR_NONFINITE;
    return GS_OK;
}

extern "C" const char* gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "pair capacity exceeded";
        case GS_ERR_WORKSPACE: return "workspace too small";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_TIMEOUT: return "device wait timed out";
        case GS_ERR_NONFINITE: return "invalid Gaussian parameters";
    }
    return "unknown status";
}

extern "C" unsigned long long gs_launch_count(void) { return g_launches.load(); }

extern "C" const char* gs_version(void) { return "gsmri 0.1.0 (sm_103a)"; }
