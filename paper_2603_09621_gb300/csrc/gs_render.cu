// gs_render.cu -- Eq. 3-4 forward render and its Eq. 5-6 adjoint, one CTA per brick
// (Sec. 3.3: "each handled by one CUDA thread block"; the brick's Gaussians are staged into
// shared memory and no depth order is needed).
//
// A brick of bx x by x bz voxels is treated as by * bz rows of bx voxels along x. For a
// Gaussian and a row through (dy, dz) (offsets from the mean, voxel units) the exponent
// along the row is q(dx) = |z_row + dx m0|^2 with z_row = m1 dy + m2 dz (whitened
// coordinates, see the record layout). Two exact, conservative culls decide which rows a
// Gaussian can reach:
//   * slab: |M (p - c)| <= sum_j h_j |m_j| over a box of half-extents h around c, so the
//     box is missed when |M (c - mu)| - sum_j h_j |m_j| > sqrt(T) (triangle inequality);
//   * row shadow: min over dx of q = Pyy dy^2 + P2yz dy dz + Pzz dz^2 (the Gram form of m1,
//     m2 projected orthogonally to m0), so the row is missed when that exceeds T.
// (T = (log2 e / 2) trunc_sigma^2; margins absorb FP32 rounding.) A pair contributes only
// where q <= T, evaluated per voxel, so culled pairs contribute exact zeros.
//
// Per (row, Gaussian) the exponent is expanded around the row's nearest integer voxel x_c to
// the Gaussian's closest point: q(x) = q_c + t (a t + 2 b_c), t = x - x_c, a = |m0|^2,
// q_c = |z_c|^2, b_c = z_c . m0. x_c depends only on the Gaussian and the row, never on the
// brick, so every voxel's value is the same for any brick shape, and every term stays of the
// size of q itself for the voxels inside the ellipsoid (no cancellation).
//
// Forward: lane <-> row; the row's bx S and W accumulate in registers in ascending Gaussian
// id (deterministic). A warp tests 32 staged Gaussians against its slab with one ballot;
// each lane then keeps a 64-bit mask of the chunk's Gaussians that reach its row and walks
// it in order.
// Adjoint: each warp owns 32 staged Gaussians; an owner lane builds its Gaussian's row mask
// from the row shadow, the warp turns the (Gaussian, row) hits into work items by a prefix
// sum, and each lane evaluates one item: the row's bx voxels, summed into 11 render-space
// partials. The owner adds its items in row order. The per-(brick, Gaussian) result goes to
// a per-pair slot (deterministic mode, reduced later in Gaussian-major order) or to one
// float atomic per value (fast mode).
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>

#include "gs_common.cuh"

namespace gs {

constexpr int kFwdChunk = 64;    // Gaussians staged per forward round (one 64-bit mask)
constexpr int kBwdChunk = 256;   // Gaussians staged per adjoint round (8 warps x 32)
constexpr int kMaxRows = 64;     // rows per brick (by * bz)
constexpr int kBwdThreads = 256;

struct RenderGeo {
    int nx, ny, nz;
    int bsx, bsy, bsz;  // brick shape
    int nbx, nby;
    float T;            // (log2 e / 2) trunc_sigma^2: a pair contributes when q <= T
    float Trow;         // row / slab cull bound on q: T (1 + 1e-2) + 1e-3
    float sqrtTcull;    // sqrt(Trow)
    float eps;
};

struct Rec {
    float mhx, mhy, mhz, mlx, mly, mlz;
    float m0x, m0y, m0z, m1x, m1y, m1z, m2x, m2y, m2z;
    float n0, n1, n2, inva, pyy, p2yz, pzz, vr, r, v;
};

__device__ __forceinline__ Rec load_rec(const float4* s) {
    const float4 a = s[0], b = s[1], c = s[2], d = s[3], e = s[4], f = s[5], g = s[6];
    Rec R;
    R.mhx = a.x; R.mhy = a.y; R.mhz = a.z; R.mlx = a.w;
    R.mly = b.x; R.mlz = b.y; R.m0x = b.z; R.m0y = b.w;
    R.m0z = c.x; R.m1x = c.y; R.m1y = c.z; R.m1z = c.w;
    R.m2x = d.x; R.m2y = d.y; R.m2z = d.z; R.n0 = d.w;
    R.n1 = e.x; R.n2 = e.y; R.inva = e.z; R.pyy = e.w;
    R.p2yz = f.x; R.pzz = f.y; R.vr = f.z; R.r = f.w;
    R.v = g.x;
    return R;
}

// Slab cull: may the Gaussian reach a voxel centre in [xa, xb] x [ya, yb] x [za, zb]?
__device__ __forceinline__ bool slab_hit(const float4* s, float xa, float xb, float ya, float yb,
                                         float za, float zb, float sqrtTcull) {
    const float4 a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    const float cx = 0.5f * (xa + xb), cy = 0.5f * (ya + yb), cz = 0.5f * (za + zb);
    const float dx = (cx - a.x) - a.w, dy = (cy - a.y) - b.x, dz = (cz - a.z) - b.y;
    // z_c = M (c - mu) = m0 dx + m1 dy + m2 dz
    const float zx = b.z * dx + c.y * dy + d.x * dz;
    const float zy = b.w * dx + c.z * dy + d.y * dz;
    const float zz = c.x * dx + c.w * dy + d.z * dz;
    const float zc = sqrtf(zx * zx + zy * zy + zz * zz);
    const float rad = 0.5f * ((xb - xa) * d.w + (yb - ya) * e.x + (zb - za) * e.y);
    return zc - rad <= sqrtTcull;
}

// Row-shadow cull for the row through voxel centres (., y, z).
__device__ __forceinline__ bool row_hit(const float4* s, float fy, float fz, float Trow) {
    const float4 a = s[0], b = s[1], e = s[4], f = s[5];
    const float dy = (fy - a.y) - b.x, dz = (fz - a.z) - b.y;
    const float q = fmaf(e.w * dy, dy, fmaf(f.x * dy, dz, f.y * dz * dz));
    return q <= Trow;
}

// Row set-up: the expansion point of the exponent along the row through (y, z).
struct RowExp {
    float qc, twob, a, t0;  // q(x) = qc + t (a t + twob), t = x - x_c = t0 + xb
    float dy, dz, dxc;      // offsets from the mean; dxc = x_c - mu_x
};

__device__ __forceinline__ RowExp row_setup(const Rec& R, float fy, float fz, float fx0) {
    RowExp E;
    E.dy = (fy - R.mhy) - R.mly;
    E.dz = (fz - R.mhz) - R.mlz;
    const float zrx = fmaf(R.m1x, E.dy, R.m2x * E.dz);
    const float zry = fmaf(R.m1y, E.dy, R.m2y * E.dz);
    const float zrz = fmaf(R.m1z, E.dy, R.m2z * E.dz);
    const float b0 = zrx * R.m0x + zry * R.m0y + zrz * R.m0z;
    // nearest integer voxel to the row's closest point x* = mu_x - b0 / a (brick independent)
    float xc = rintf((R.mhx - b0 * R.inva) + R.mlx);
    xc = fminf(fmaxf(xc, -8388608.0f), 8388608.0f);
    E.dxc = (xc - R.mhx) - R.mlx;
    const float zcx = fmaf(E.dxc, R.m0x, zrx);
    const float zcy = fmaf(E.dxc, R.m0y, zry);
    const float zcz = fmaf(E.dxc, R.m0z, zrz);
    E.qc = zcx * zcx + zcy * zcy + zcz * zcz;
    E.twob = 2.0f * (zcx * R.m0x + zcy * R.m0y + zcz * R.m0z);
    E.a = R.m0x * R.m0x + R.m0y * R.m0y + R.m0z * R.m0z;
    E.t0 = fx0 - xc;
    return E;
}

// ------------------------------------------------------------------------ forward

template <int BX, bool kStats>
__global__ void __launch_bounds__(64) k_render_fwd(const int32_t* __restrict__ brick_off,
                                                   const int32_t* __restrict__ pair_gid,
                                                   const float4* __restrict__ rec4, RenderGeo G,
                                                   float* __restrict__ I, float* __restrict__ W,
                                                   unsigned long long* __restrict__ stats) {
    __shared__ float4 srec[kFwdChunk][REC_F4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrows = G.bsy * G.bsz;
    const int b = blockIdx.x;
    const int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    const int x0 = bx * BX, y0 = by * G.bsy, z0 = bz * G.bsz;
    const bool row_ok = tid < nrows;
    const int y = y0 + tid % G.bsy, z = z0 + tid / G.bsy;
    const float fy = float(y), fz = float(z), fx0 = float(x0);
    // this warp's slab of voxel centres
    const int r_first = warp * 32, r_last = min(nrows, warp * 32 + 32) - 1;
    const float sxa = fx0, sxb = float(x0 + BX - 1);
    const float sya = float(y0), syb = float(y0 + G.bsy - 1);
    const float sza = float(z0 + r_first / G.bsy), szb = float(z0 + r_last / G.bsy);

    float S[BX], Wa[BX];
#pragma unroll
    for (int i = 0; i < BX; ++i) {
        S[i] = 0.f;
        Wa[i] = 0.f;
    }
    unsigned long long n_eff = 0, n_eval = 0;
    const int start = brick_off[b], end = brick_off[b + 1];
    for (int c0 = start; c0 < end; c0 += kFwdChunk) {
        const int cnt = min(kFwdChunk, end - c0);
        __syncthreads();
        for (int i = tid; i < cnt * REC_F4; i += blockDim.x) {
            const int k = i / REC_F4, part = i - k * REC_F4;
            srec[k][part] = rec4[int64_t(pair_gid[c0 + k]) * REC_F4 + part];
        }
        __syncthreads();
        unsigned long long hits = 0;
        for (int h = 0; h < cnt; h += 32) {
            const int k = h + lane;
            const bool sh = (k < cnt) && slab_hit(srec[k], sxa, sxb, sya, syb, sza, szb, G.sqrtTcull);
            unsigned m = __ballot_sync(0xffffffffu, sh);
            while (m) {
                const int kk = h + __ffs(m) - 1;
                m &= m - 1;
                if (row_ok && row_hit(srec[kk], fy, fz, G.Trow)) hits |= 1ull << kk;
            }
        }
        while (hits) {
            const int kk = __ffsll(static_cast<long long>(hits)) - 1;
            hits &= hits - 1;
            const Rec R = load_rec(srec[kk]);
            const RowExp E = row_setup(R, fy, fz, fx0);
#pragma unroll
            for (int i = 0; i < BX; ++i) {
                const float t = E.t0 + float(i);
                const float q = fmaf(t, fmaf(E.a, t, E.twob), E.qc);
                float g = ex2_approx(-q);
                g = (q <= G.T) ? g : 0.0f;
                S[i] = fmaf(R.vr, g, S[i]);
                Wa[i] = fmaf(R.r, g, Wa[i]);
                if (kStats) n_eff += (q <= G.T && x0 + i < G.nx) ? 1 : 0;
            }
            if (kStats) n_eval += BX;
        }
    }
    if (row_ok && y < G.ny && z < G.nz) {
        const int64_t row = (int64_t(z) * G.ny + y) * G.nx;
#pragma unroll
        for (int i = 0; i < BX; ++i) {
            if (x0 + i < G.nx) {
                I[row + x0 + i] = S[i] / (Wa[i] > G.eps ? Wa[i] : G.eps);
                W[row + x0 + i] = Wa[i];
            }
        }
    } else {
        n_eff = 0;
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

// Position of the k-th set bit (k counted from 0) of a 64-bit mask that has more than k.
__device__ __forceinline__ int select_bit64(unsigned long long m, int k) {
    int pos = 0;
    unsigned w = static_cast<unsigned>(m);
    int c = __popc(w);
    if (k >= c) {
        k -= c;
        w = static_cast<unsigned>(m >> 32);
        pos = 32;
    }
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const unsigned lowmask = (1u << half) - 1u;
        c = __popc(w & lowmask);
        if (k >= c) {
            k -= c;
            w >>= half;
            pos += half;
        }
    }
    return pos;
}

// Rows of the brick (index rz * bsy + ry) that the Gaussian may reach: per z-row the row
// shadow is a quadratic in dy, solved for its y-interval (padded by a margin).
__device__ __forceinline__ unsigned long long brick_row_mask(const Rec& R, const RenderGeo& G,
                                                             int y0, int z0) {
    unsigned long long mask = 0;
    const float mu_y = R.mhy + R.mly;
    const float inv2a = 0.5f / R.pyy;
    for (int rz = 0; rz < G.bsz; ++rz) {
        const float dz = (float(z0 + rz) - R.mhz) - R.mlz;
        const float bq = R.p2yz * dz;
        const float cq = R.pzz * dz * dz - G.Trow;
        const float disc = bq * bq - 4.0f * R.pyy * cq;
        if (!(disc >= 0.0f)) continue;
        const float sq = sqrtf(disc);
        const float ylo = mu_y + (-bq - sq) * inv2a;
        const float yhi = mu_y + (-bq + sq) * inv2a;
        const float pad = 1e-3f + 1e-5f * fabsf(mu_y);
        int ia = static_cast<int>(ceilf(fmaxf(ylo - pad, float(y0) - 1.0f))) - y0;
        int ib = static_cast<int>(floorf(fminf(yhi + pad, float(y0 + G.bsy)))) - y0;
        ia = max(ia, 0);
        ib = min(ib, G.bsy - 1);
        if (ia > ib) continue;
        const unsigned long long bits = ((2ull << (ib - ia)) - 1ull) << (rz * G.bsy + ia);
        mask |= bits;
    }
    return mask;
}

template <int BX, bool kDet>
__global__ void __launch_bounds__(kBwdThreads) k_render_bwd(
    const int32_t* __restrict__ brick_off, const int32_t* __restrict__ pair_gid,
    const int32_t* __restrict__ pair_gmj, const float4* __restrict__ rec4, RenderGeo G,
    const float* __restrict__ Iv, const float* __restrict__ Wv, const float* __restrict__ dIv,
    float* __restrict__ part, float* __restrict__ gacc) {
    extern __shared__ float4 smem4[];
    float4(*srec)[REC_F4] = reinterpret_cast<float4(*)[REC_F4]>(smem4);              // [256][7]
    float2* ab = reinterpret_cast<float2*>(smem4 + kBwdChunk * REC_F4);                  // [rows][BX+1]
    float(*ipart)[32][12] = reinterpret_cast<float(*)[32][12]>(ab + kMaxRows * (BX + 1));  // [8][32][12]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    const int x0 = bx * BX, y0 = by * G.bsy, z0 = bz * G.bsz;
    const int nrows = G.bsy * G.bsz;
    const float fx0 = float(x0);

    // Prologue: per-voxel factors. dL/dw_i = (v_i - I') alpha with alpha = dL/dI / max(W, eps)
    // and I' = I where W > eps, else 0 (Eq. 5; below the floor I = S / eps, dI/dw_i = v_i / eps).
    for (int i = tid; i < nrows * BX; i += blockDim.x) {
        const int r = i / BX, xb = i - r * BX;
        const int x = x0 + xb, y = y0 + r % G.bsy, z = z0 + r / G.bsy;
        float alpha = 0.f, ip = 0.f;
        if (x < G.nx && y < G.ny && z < G.nz) {
            const int64_t idx = (int64_t(z) * G.ny + y) * G.nx + x;
            const float w = Wv[idx], gI = dIv[idx];
            alpha = gI / (w > G.eps ? w : G.eps);
            ip = (w > G.eps) ? Iv[idx] : 0.0f;
        }
        ab[r * (BX + 1) + xb] = make_float2(alpha, ip);
    }

    const int start = brick_off[b], end = brick_off[b + 1];
    for (int c0 = start; c0 < end; c0 += kBwdChunk) {
        const int cnt = min(kBwdChunk, end - c0);
        __syncthreads();
        for (int i = tid; i < cnt * REC_F4; i += blockDim.x) {
            const int k = i / REC_F4, prt = i - k * REC_F4;
            srec[k][prt] = rec4[int64_t(pair_gid[c0 + k]) * REC_F4 + prt];
        }
        __syncthreads();

        const int k = warp * 32 + lane;  // chunk-local Gaussian owned by this lane
        const bool own = k < cnt;
        unsigned long long rmask = 0;
        if (own) rmask = brick_row_mask(load_rec(srec[k]), G, y0, z0);
        const int nmine = __popcll(static_cast<long long>(rmask));
        int incl = nmine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int mstart = incl - nmine;
        const int total = __shfl_sync(0xffffffffu, incl, 31);

        float acc[11];
#pragma unroll
        for (int q = 0; q < 11; ++q) acc[q] = 0.f;

        for (int b0 = 0; b0 < total; b0 += 32) {
            const int it = b0 + lane;
            // owner of item `it`: the last lane whose start is <= it
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = j + step;
                const int sc = __shfl_sync(0xffffffffu, mstart, cand & 31);
                if (cand < 32 && sc <= it) j = cand;
            }
            const unsigned mlo = __shfl_sync(0xffffffffu, static_cast<unsigned>(rmask), j);
            const unsigned mhi = __shfl_sync(0xffffffffu, static_cast<unsigned>(rmask >> 32), j);
            const int jstart = __shfl_sync(0xffffffffu, mstart, j);
            if (it < total) {
                const unsigned long long om = (static_cast<unsigned long long>(mhi) << 32) | mlo;
                const int r = select_bit64(om, it - jstart);
                const int ry = r % G.bsy, rz = r / G.bsy;
                const Rec R = load_rec(srec[warp * 32 + j]);
                const RowExp E = row_setup(R, float(y0 + ry), float(z0 + rz), fx0);
                const float2* abr = ab + r * (BX + 1);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, dv = 0.f, dr = 0.f;
#pragma unroll
                for (int i = 0; i < BX; ++i) {
                    const float t = E.t0 + float(i);
                    const float q = fmaf(t, fmaf(E.a, t, E.twob), E.qc);
                    float g = ex2_approx(-q);
                    g = (q <= G.T) ? g : 0.0f;
                    const float2 av = abr[i];
                    const float w = R.r * g;
                    const float gam = (R.v - av.y) * av.x;
                    dv = fmaf(av.x, w, dv);
                    dr = fmaf(gam, g, dr);
                    const float Gw = gam * w;
                    const float dx = E.dxc + t;
                    s0 += Gw;
                    const float tg = Gw * dx;
                    s1 += tg;
                    s2 = fmaf(tg, dx, s2);
                }
                const float dy = E.dy, dz = E.dz;
                float* ip = ipart[warp][lane];
                ip[G_M1X] = s1;
                ip[G_M1Y] = dy * s0;
                ip[G_M1Z] = dz * s0;
                ip[G_M2XX] = s2;
                ip[G_M2YY] = dy * dy * s0;
                ip[G_M2ZZ] = dz * dz * s0;
                ip[G_M2XY] = dy * s1;
                ip[G_M2XZ] = dz * s1;
                ip[G_M2YZ] = dy * dz * s0;
                ip[G_DV] = dv;
                ip[G_DR] = dr;
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

template <int BX>
constexpr size_t bwd_smem_bytes() {
    return sizeof(float4) * kBwdChunk * REC_F4 + sizeof(float2) * kMaxRows * (BX + 1) +
           sizeof(float) * 8 * 32 * 12;
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
    const int64_t P = *npairs;
    if (P >= 0 && P <= capacity) {
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
    G.nbx = b.nbx; G.nby = b.nby;
    G.T = kHalfLog2e * cfg->trunc_sigma * cfg->trunc_sigma;
    G.Trow = G.T * (1.0f + 1e-2f) + 1e-3f;
    G.sqrtTcull = sqrtf(G.Trow);
    G.eps = cfg->eps;
    return G;
}

template <int BX>
static gs_status launch_fwd(const gs_bins* bins, const RenderGeo& G, float* I, float* W,
                            unsigned long long* stats, cudaStream_t st) {
    const int threads = ((G.bsy * G.bsz + 31) / 32) * 32;
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    if (stats)
        k_render_fwd<BX, true><<<bins->n_bricks, threads, 0, st>>>(bins->brick_off, bins->pair_gid,
                                                                   rec4, G, I, W, stats);
    else
        k_render_fwd<BX, false><<<bins->n_bricks, threads, 0, st>>>(bins->brick_off, bins->pair_gid,
                                                                    rec4, G, I, W, nullptr);
    return last_launch_status();
}

gs_status render_fwd_impl(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                          float* I, float* W, unsigned long long* stats, cudaStream_t st) {
    RenderGeo G = make_geo(grid, cfg);
    switch (G.bsx) {
        case 4: return launch_fwd<4>(bins, G, I, W, stats, st);
        case 8: return launch_fwd<8>(bins, G, I, W, stats, st);
        case 16: return launch_fwd<16>(bins, G, I, W, stats, st);
    }
    return GS_ERR_INVALID_ARG;
}

gs_status bind_workspace(void* base, size_t bytes, int64_t n_gauss, int64_t capacity,
                         const gs_grid* grid, const gs_config* cfg, Workspace* ws);
bool bins_match(const gs_bins* b, const gs_grid* grid, const gs_config* cfg);

template <int BX, bool kDet>
static gs_status launch_bwd(const gs_bins* bins, const RenderGeo& G, const float* I, const float* W,
                            const float* dI, const Workspace& ws, cudaStream_t st) {
    const size_t smem = bwd_smem_bytes<BX>();
    // Opt in to more than 48 KB of dynamic shared memory once per device.
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        if (cudaFuncSetAttribute(k_render_bwd<BX, kDet>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) != cudaSuccess)
            return GS_ERR_CUDA;
        attr_done.fetch_or(bit);
    }
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    k_render_bwd<BX, kDet><<<bins->n_bricks, kBwdThreads, smem, st>>>(
        bins->brick_off, bins->pair_gid, bins->pair_gmj, rec4, G, I, W, dI,
        kDet ? ws.part : nullptr, kDet ? nullptr : ws.gacc);
    return last_launch_status();
}

template <bool kDet>
static gs_status launch_bwd_bx(const gs_bins* bins, const RenderGeo& G, const float* I,
                               const float* W, const float* dI, const Workspace& ws,
                               cudaStream_t st) {
    switch (G.bsx) {
        case 4: return launch_bwd<4, kDet>(bins, G, I, W, dI, ws, st);
        case 8: return launch_bwd<8, kDet>(bins, G, I, W, dI, ws, st);
        case 16: return launch_bwd<16, kDet>(bins, G, I, W, dI, ws, st);
    }
    return GS_ERR_INVALID_ARG;
}

// Render-space adjoint into ws.gacc [N, 12] (no parameter chain).
gs_status render_bwd_geo(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                         const float* I, const float* W, const float* dI, const Workspace& ws,
                         cudaStream_t st, const std::function<bool()>& after_kernel) {
    RenderGeo G = make_geo(grid, cfg);
    const int64_t N = bins->n_gauss;
    if (cfg->deterministic) {
        gs_status s = launch_bwd_bx<true>(bins, G, I, W, dI, ws, st);
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
    gs_status s = launch_bwd_bx<false>(bins, G, I, W, dI, ws, st);
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
