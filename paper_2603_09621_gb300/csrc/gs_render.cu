// gs_render.cu -- Eq. 3-4 forward render and its Eq. 5-6 adjoint, one CTA per brick
// (Sec. 3.3: "each handled by one CUDA thread block"; the brick's Gaussians are staged into
// shared memory).
//
// Both kernels split a brick into 4 x 4 x 4 voxel footprints. A footprint F is skipped for a
// Gaussian when the Mahalanobis triangle inequality proves that no voxel of F has
// d^2 <= trunc_sigma^2: with centre c and |p - c|_inf <= 3/2 voxel,
//     |p - mu|_M >= |c - mu|_M - |p - c|_M,   |p - c|_M^2 <= (3/2)^2 sum_ab |M_ab|,
// so the skip adds exactly nothing (a small margin absorbs FP32 rounding). Skipped and
// truncated pairs contribute exact zeros, so results do not depend on the brick shape.
//
// Forward: lane <-> 2 voxels of its warp's footprint, warp-ballot over the staged Gaussians,
// per-voxel S and W accumulated in registers in ascending Gaussian id (deterministic).
// Adjoint: each warp takes 32 staged Gaussians; their (Gaussian, footprint) hits become
// work items spread over the lanes; every item sums its footprint's 64 voxels into 11
// render-space partials; the owner lane of the Gaussian adds its items in footprint order.
// The per-(brick, Gaussian) result goes to a per-pair slot (deterministic mode, reduced
// later in Gaussian-major order) or to one float atomic per value (fast mode).
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "gs_common.cuh"

namespace gs {

constexpr int kFwdChunk = 128;  // Gaussians staged per forward round
constexpr int kBwdChunk = 256;  // Gaussians staged per adjoint round (8 warps x 32)
constexpr int kMaxFoot = 16;    // footprints per brick (brick volume <= 1024)

struct RenderGeo {
    int nx, ny, nz;
    int bsx, bsy, bsz;  // brick shape
    int fx, fy, fz;     // footprints per brick along each axis
    int nbx, nby;
    float thr;          // -(log2 e / 2) trunc_sigma^2: a pair contributes when e >= thr
    float cull;         // sqrt(-thr) * (1 + 1e-3) + 1e-3: footprint skip bound
    float eps;
};

__device__ __forceinline__ int64_t valid_pairs_r(const int64_t* npairs, int64_t capacity) {
    int64_t P = *npairs;
    return (P > capacity || P < 0) ? 0 : P;
}

// True if the Gaussian (record r0..r2) may reach a voxel of the footprint whose first voxel
// has index (ox, oy, oz) (see the file comment).
__device__ __forceinline__ bool foot_hit(const float4& r0, const float4& r1, const float4& r2,
                                         float ox, float oy, float oz, float cull) {
    const float dx = ((ox + 1.5f) - r0.x) - r0.w;
    const float dy = ((oy + 1.5f) - r0.y) - r1.x;
    const float dz = ((oz + 1.5f) - r0.z) - r1.y;
    const float Qxx = r1.z, Qyy = r1.w, Qzz = r2.x, Q2xy = r2.y, Q2xz = r2.z, Q2yz = r2.w;
    float e = Qxx * dx * dx + Qyy * dy * dy + Qzz * dz * dz + Q2xy * dx * dy + Q2xz * dx * dz +
              Q2yz * dy * dz;
    float mc = sqrtf(fmaxf(-e, 0.0f));
    float rq = 2.25f * (fabsf(Qxx) + fabsf(Qyy) + fabsf(Qzz) + fabsf(Q2xy) + fabsf(Q2xz) +
                        fabsf(Q2yz));
    return mc - sqrtf(rq) <= cull;
}

// ------------------------------------------------------------------------ forward

template <bool kStats>
__global__ void __launch_bounds__(512) k_render_fwd(const int32_t* __restrict__ brick_off,
                                                    const int32_t* __restrict__ pair_gid,
                                                    const float4* __restrict__ rec4,
                                                    RenderGeo G, float* __restrict__ I,
                                                    float* __restrict__ W,
                                                    unsigned long long* __restrict__ stats) {
    __shared__ float4 srec[kFwdChunk][4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int b = blockIdx.x;
    const int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    const int wx = warp % G.fx, wy = (warp / G.fx) % G.fy, wz = warp / (G.fx * G.fy);
    const int ox = bx * G.bsx + wx * 4, oy = by * G.bsy + wy * 4, oz = bz * G.bsz + wz * 4;
    const int x0 = ox + 2 * (lane & 1), y = oy + ((lane >> 1) & 3), z = oz + (lane >> 3);
    const float fx0 = static_cast<float>(x0), fy = static_cast<float>(y), fz = static_cast<float>(z);
    const float fox = static_cast<float>(ox), foy = static_cast<float>(oy), foz = static_cast<float>(oz);

    float S0 = 0.f, W0 = 0.f, S1 = 0.f, W1 = 0.f;
    unsigned long long n_eff = 0, n_eval = 0;
    const int start = brick_off[b], end = brick_off[b + 1];
    for (int c0 = start; c0 < end; c0 += kFwdChunk) {
        const int cnt = min(kFwdChunk, end - c0);
        __syncthreads();
        for (int i = tid; i < cnt * 4; i += nthreads) {
            const int k = i >> 2, part = i & 3;
            const int gid = pair_gid[c0 + k];
            srec[k][part] = rec4[int64_t(gid) * 4 + part];
        }
        __syncthreads();
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            const int k = k0 + lane;
            bool hit = false;
            if (k < cnt) hit = foot_hit(srec[k][0], srec[k][1], srec[k][2], fox, foy, foz, G.cull);
            unsigned mask = __ballot_sync(0xffffffffu, hit);
            while (mask) {
                const int kk = k0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 r0 = srec[kk][0], r1 = srec[kk][1], r2 = srec[kk][2], r3 = srec[kk][3];
                const float dy = (fy - r0.y) - r1.x;
                const float dz = (fz - r0.z) - r1.y;
                const float u0 = (fx0 - r0.x) - r0.w;
                const float u1 = u0 + 1.0f;
                const float Qxx = r1.z, Qyy = r1.w, Qzz = r2.x, Q2xy = r2.y, Q2xz = r2.z, Q2yz = r2.w;
                const float cb = fmaf(Q2xy, dy, Q2xz * dz);
                const float cc = fmaf(fmaf(Qyy, dy, Q2yz * dz), dy, Qzz * dz * dz);
                const float e0 = fmaf(fmaf(Qxx, u0, cb), u0, cc);
                const float e1 = fmaf(fmaf(Qxx, u1, cb), u1, cc);
                float g0 = ex2_approx(e0), g1 = ex2_approx(e1);
                g0 = (e0 >= G.thr) ? g0 : 0.0f;
                g1 = (e1 >= G.thr) ? g1 : 0.0f;
                S0 = fmaf(r3.x, g0, S0);
                W0 = fmaf(r3.y, g0, W0);
                S1 = fmaf(r3.x, g1, S1);
                W1 = fmaf(r3.y, g1, W1);
                if (kStats) {
                    const bool in_yz = y < G.ny && z < G.nz;
                    n_eff += (in_yz && x0 < G.nx && e0 >= G.thr) ? 1 : 0;
                    n_eff += (in_yz && x0 + 1 < G.nx && e1 >= G.thr) ? 1 : 0;
                    n_eval += 2;
                }
            }
        }
    }
    if (y < G.ny && z < G.nz) {
        const int64_t row = (int64_t(z) * G.ny + y) * G.nx;
        if (x0 < G.nx) {
            I[row + x0] = S0 / (W0 > G.eps ? W0 : G.eps);
            W[row + x0] = W0;
        }
        if (x0 + 1 < G.nx) {
            I[row + x0 + 1] = S1 / (W1 > G.eps ? W1 : G.eps);
            W[row + x0 + 1] = W1;
        }
    }
    if (kStats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_eff += __shfl_xor_sync(0xffffffffu, n_eff, o);
            n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
        }
        if (lane == 0) {
            atomicAdd(&stats[0], n_eff);
            atomicAdd(&stats[1], n_eval);
        }
    }
}

// ------------------------------------------------------------------------ adjoint

template <bool kDet>
__global__ void __launch_bounds__(256) k_render_bwd(
    const int32_t* __restrict__ brick_off, const int32_t* __restrict__ pair_gid,
    const int32_t* __restrict__ pair_gmj, const float4* __restrict__ rec4, RenderGeo G,
    const float* __restrict__ Iv, const float* __restrict__ Wv, const float* __restrict__ dIv,
    float* __restrict__ part, float* __restrict__ gacc) {
    __shared__ float4 srec[kBwdChunk][4];
    __shared__ float2 ab[kMaxFoot][66];              // (dL/dI / W', I') per footprint voxel
    __shared__ unsigned short items[8][32 * kMaxFoot];
    __shared__ float ipart[8][32][12];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    const int nf = G.fx * G.fy * G.fz;
    const int bx0 = bx * G.bsx, by0 = by * G.bsy, bz0 = bz * G.bsz;

    // Prologue: per-voxel factors. gamma = dL/dw_i = (v_i - I') * alpha with
    // alpha = dL/dI / max(W, eps) and I' = I where W > eps, else 0 (Eq. 5; I = S / eps below
    // the floor gives dI/dw_i = v_i / eps).
    for (int i = tid; i < nf * 64; i += blockDim.x) {
        const int f = i >> 6, v = i & 63;
        const int fx = f % G.fx, fy = (f / G.fx) % G.fy, fz = f / (G.fx * G.fy);
        const int x = bx0 + fx * 4 + (v & 3), y = by0 + fy * 4 + ((v >> 2) & 3),
                  z = bz0 + fz * 4 + (v >> 4);
        float alpha = 0.f, ip = 0.f;
        if (x < G.nx && y < G.ny && z < G.nz) {
            const int64_t idx = (int64_t(z) * G.ny + y) * G.nx + x;
            const float w = Wv[idx], gI = dIv[idx];
            alpha = gI / (w > G.eps ? w : G.eps);
            ip = (w > G.eps) ? Iv[idx] : 0.0f;
        }
        ab[f][v] = make_float2(alpha, ip);
    }

    const int start = brick_off[b], end = brick_off[b + 1];
    for (int c0 = start; c0 < end; c0 += kBwdChunk) {
        const int cnt = min(kBwdChunk, end - c0);
        __syncthreads();
        for (int i = tid; i < cnt * 4; i += blockDim.x) {
            const int k = i >> 2, prt = i & 3;
            srec[k][prt] = rec4[int64_t(pair_gid[c0 + k]) * 4 + prt];
        }
        __syncthreads();

        const int k = warp * 32 + lane;  // chunk-local Gaussian owned by this lane
        const bool own = k < cnt;
        unsigned fmask = 0;
        if (own) {
            const float4 r0 = srec[k][0], r1 = srec[k][1], r2 = srec[k][2];
            for (int f = 0; f < nf; ++f) {
                const int fx = f % G.fx, fy = (f / G.fx) % G.fy, fz = f / (G.fx * G.fy);
                if (foot_hit(r0, r1, r2, float(bx0 + fx * 4), float(by0 + fy * 4),
                             float(bz0 + fz * 4), G.cull))
                    fmask |= 1u << f;
            }
        }
        const int nmine = __popc(fmask);
        int incl = nmine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int mstart = incl - nmine;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        {
            unsigned m = fmask;
            int pos = mstart;
            while (m) {
                const int f = __ffs(m) - 1;
                m &= m - 1;
                items[warp][pos++] = static_cast<unsigned short>((lane << 4) | f);
            }
        }
        __syncwarp();

        float acc[11];
#pragma unroll
        for (int q = 0; q < 11; ++q) acc[q] = 0.f;

        for (int b0 = 0; b0 < total; b0 += 32) {
            const int it_idx = b0 + lane;
            if (it_idx < total) {
                const unsigned it = items[warp][it_idx];
                const int jl = it >> 4, f = it & 15;
                const int kk = warp * 32 + jl;
                const float4 r0 = srec[kk][0], r1 = srec[kk][1], r2 = srec[kk][2], r3 = srec[kk][3];
                const int fx = f % G.fx, fy = (f / G.fx) % G.fy, fz = f / (G.fx * G.fy);
                const float ux = (float(bx0 + fx * 4) - r0.x) - r0.w;
                const float uy0 = (float(by0 + fy * 4) - r0.y) - r1.x;
                const float uz0 = (float(bz0 + fz * 4) - r0.z) - r1.y;
                const float Qxx = r1.z, Qyy = r1.w, Qzz = r2.x, Q2xy = r2.y, Q2xz = r2.z, Q2yz = r2.w;
                const float rr = r3.y, vv = r3.z;
                float m1x = 0.f, m1y = 0.f, m1z = 0.f, m2xx = 0.f, m2yy = 0.f, m2zz = 0.f;
                float m2xy = 0.f, m2xz = 0.f, m2yz = 0.f, dv = 0.f, dr = 0.f;
                const float2* abf = ab[f];
#pragma unroll
                for (int vz = 0; vz < 4; ++vz) {
                    const float dz = uz0 + float(vz);
#pragma unroll
                    for (int vy = 0; vy < 4; ++vy) {
                        const float dy = uy0 + float(vy);
                        const float cb = fmaf(Q2xy, dy, Q2xz * dz);
                        const float cc = fmaf(fmaf(Qyy, dy, Q2yz * dz), dy, Qzz * dz * dz);
                        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
                        for (int vx = 0; vx < 4; ++vx) {
                            const float u = ux + float(vx);
                            const float e = fmaf(fmaf(Qxx, u, cb), u, cc);
                            float g = ex2_approx(e);
                            g = (e >= G.thr) ? g : 0.0f;
                            const float2 a = abf[(vz * 4 + vy) * 4 + vx];
                            const float w = rr * g;
                            const float gam = (vv - a.y) * a.x;
                            dv = fmaf(a.x, w, dv);
                            dr = fmaf(gam, g, dr);
                            const float Gw = gam * w;
                            s0 += Gw;
                            const float t = Gw * u;
                            s1 += t;
                            s2 = fmaf(t, u, s2);
                        }
                        m1x += s1;
                        m1y = fmaf(dy, s0, m1y);
                        m1z = fmaf(dz, s0, m1z);
                        m2xx += s2;
                        m2xy = fmaf(dy, s1, m2xy);
                        m2xz = fmaf(dz, s1, m2xz);
                        const float ty = dy * s0;
                        m2yy = fmaf(ty, dy, m2yy);
                        m2yz = fmaf(ty, dz, m2yz);
                        m2zz = fmaf(dz * s0, dz, m2zz);
                    }
                }
                float* ip = ipart[warp][lane];
                ip[G_M1X] = m1x; ip[G_M1Y] = m1y; ip[G_M1Z] = m1z;
                ip[G_M2XX] = m2xx; ip[G_M2YY] = m2yy; ip[G_M2ZZ] = m2zz;
                ip[G_M2XY] = m2xy; ip[G_M2XZ] = m2xz; ip[G_M2YZ] = m2yz;
                ip[G_DV] = dv; ip[G_DR] = dr;
            }
            __syncwarp();
            if (own) {
                const int lo = max(mstart, b0), hi = min(mstart + nmine, b0 + 32);
                for (int q = lo; q < hi; ++q) {
                    const float* ip = ipart[warp][q - b0];
#pragma unroll
                    for (int m = 0; m < 11; ++m) acc[m] += ip[m];
                }
            }
            __syncwarp();
        }

        if (own) {
            const int64_t pos = int64_t(c0) + k;
            if (kDet) {
                const int64_t j = pair_gmj[pos];
                float4* dst = reinterpret_cast<float4*>(part + j * GRAD_FLOATS);
                dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                dst[2] = make_float4(acc[8], acc[9], acc[10], 0.f);
            } else if (nmine > 0) {
                float* dst = gacc + int64_t(pair_gid[pos]) * GRAD_FLOATS;
#pragma unroll
                for (int m = 0; m < 11; ++m) atomicAdd(dst + m, acc[m]);
            }
        }
    }
}

// Deterministic reduction: per Gaussian, sum its per-brick partials in Gaussian-major order
// (ascending brick index).
__global__ void __launch_bounds__(256) k_pair_reduce(const float* __restrict__ part,
                                                     const int32_t* __restrict__ gm_off,
                                                     const int64_t* __restrict__ npairs,
                                                     int64_t capacity, int64_t N,
                                                     float* __restrict__ gacc) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float acc[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) acc[m] = 0.f;
    if (valid_pairs_r(npairs, capacity) > 0) {
        const int a = gm_off[g], e = gm_off[g + 1];
        for (int j = a; j < e; ++j) {
            const float4* src = reinterpret_cast<const float4*>(part + int64_t(j) * GRAD_FLOATS);
            const float4 p0 = src[0], p1 = src[1], p2 = src[2];
            acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w;
            acc[4] += p1.x; acc[5] += p1.y; acc[6] += p1.z; acc[7] += p1.w;
            acc[8] += p2.x; acc[9] += p2.y; acc[10] += p2.z;
        }
    }
    float4* dst = reinterpret_cast<float4*>(gacc + g * GRAD_FLOATS);
    dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    dst[2] = make_float4(acc[8], acc[9], acc[10], 0.f);
}

// ------------------------------------------------------------------------ host side

RenderGeo make_geo(const gs_grid* grid, const gs_config* cfg) {
    BrickGeom b = brick_geom(grid, cfg);
    RenderGeo G;
    G.nx = grid->nx; G.ny = grid->ny; G.nz = grid->nz;
    G.bsx = b.bx; G.bsy = b.by; G.bsz = b.bz;
    G.fx = b.bx / 4; G.fy = b.by / 4; G.fz = b.bz / 4;
    G.nbx = b.nbx; G.nby = b.nby;
    G.thr = -kHalfLog2e * cfg->trunc_sigma * cfg->trunc_sigma;
    G.cull = sqrtf(-G.thr) * (1.0f + 1e-3f) + 1e-3f;
    G.eps = cfg->eps;
    return G;
}

gs_status render_fwd_impl(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                          float* I, float* W, unsigned long long* stats, cudaStream_t st) {
    RenderGeo G = make_geo(grid, cfg);
    const int threads = 32 * G.fx * G.fy * G.fz;
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    if (stats)
        k_render_fwd<true><<<bins->n_bricks, threads, 0, st>>>(bins->brick_off, bins->pair_gid, rec4,
                                                               G, I, W, stats);
    else
        k_render_fwd<false><<<bins->n_bricks, threads, 0, st>>>(bins->brick_off, bins->pair_gid,
                                                                rec4, G, I, W, nullptr);
    return last_launch_status();
}

gs_status bind_workspace(void* base, size_t bytes, int64_t n_gauss, int64_t capacity,
                         const gs_grid* grid, const gs_config* cfg, Workspace* ws);
bool bins_match(const gs_bins* b, const gs_grid* grid, const gs_config* cfg);

// Render-space adjoint into ws.gacc [N, 12] (no parameter chain).
gs_status render_bwd_geo(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                         const float* I, const float* W, const float* dI, const Workspace& ws,
                         cudaStream_t st, const std::function<bool()>& after_kernel) {
    RenderGeo G = make_geo(grid, cfg);
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    const int64_t N = bins->n_gauss;
    if (cfg->deterministic) {
        k_render_bwd<true><<<bins->n_bricks, 256, 0, st>>>(bins->brick_off, bins->pair_gid,
                                                           bins->pair_gmj, rec4, G, I, W, dI,
                                                           ws.part, nullptr);
        gs_status s = last_launch_status();
        if (s != GS_OK) return s;
        if (after_kernel && !after_kernel()) return GS_ERR_CUDA;
        if (N > 0) {
            k_pair_reduce<<<static_cast<unsigned>((N + 255) / 256), 256, 0, st>>>(
                ws.part, bins->gm_off, bins->d_npairs, bins->capacity, N, ws.gacc);
            s = last_launch_status();
        }
        return s;
    }
    if (N > 0 && cudaMemsetAsync(ws.gacc, 0, sizeof(float) * GRAD_FLOATS * N, st) != cudaSuccess)
        return GS_ERR_CUDA;
    k_render_bwd<false><<<bins->n_bricks, 256, 0, st>>>(bins->brick_off, bins->pair_gid,
                                                        bins->pair_gmj, rec4, G, I, W, dI, nullptr,
                                                        ws.gacc);
    gs_status s = last_launch_status();
    if (s != GS_OK) return s;
    if (after_kernel && !after_kernel()) return GS_ERR_CUDA;
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_render_fwd(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                                   float* I, float* W, unsigned long long* d_stats,
                                   gs_stream stream) {
    gs_status s = validate_grid_cfg(grid, cfg);
    if (s != GS_OK) return s;
    if (!bins_match(bins, grid, cfg) || !I || !W) return GS_ERR_INVALID_ARG;
    return render_fwd_impl(bins, grid, cfg, I, W, d_stats, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_render_bwd(const float* params, const gs_bins* bins, const gs_grid* grid,
                                   const gs_config* cfg, const float* I, const float* W,
                                   const float* dI, float* dparams, void* ws, size_t ws_bytes,
                                   gs_stream stream) {
    gs_status s = validate_grid_cfg(grid, cfg);
    if (s != GS_OK) return s;
    if (!bins_match(bins, grid, cfg) || !I || !W || !dI) return GS_ERR_INVALID_ARG;
    if (bins->n_gauss > 0 && (!params || !dparams)) return GS_ERR_INVALID_ARG;
    Workspace w;
    s = bind_workspace(ws, ws_bytes, bins->n_gauss, bins->capacity, grid, cfg, &w);
    if (s != GS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s = render_bwd_geo(bins, grid, cfg, I, W, dI, w, st, nullptr);
    if (s != GS_OK) return s;
    if (bins->n_gauss == 0) return GS_OK;
    return launch_param_bwd(params, w.gacc, bins->n_gauss, grid, cfg, dparams, st);
}
