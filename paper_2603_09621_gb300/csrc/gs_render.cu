// gs_render.cu -- Eq. 3-4 forward render and its Eq. 5-6 adjoint, one CTA per brick
// (Sec. 3.3: "each handled by one CUDA thread block"; the brick's Gaussians are staged into
// shared memory and no depth order is needed).
//
// Exponent of a pair (voxel p, Gaussian i) in voxel units: q = S(dy, dz) + (sa (dx - dx*))^2
// (record layout in gs_common.cuh), the Gaussian kernel is 2^-q and the pair contributes
// only where q <= T = (log2 e / 2) trunc_sigma^2. q is computed by the same operation sequence
// in both kernels from the voxel's global index and the Gaussian alone, so forward and
// adjoint agree on every inclusion decision and no result depends on the brick shape.
//
// Forward: the brick is split into 4 x 4 x 4 footprints, one half-warp each; a lane owns one
// x-row of four voxels. The block stages the brick's list in rounds of about 28 records per
// footprint (224 for an 8^3 brick), so most lists take one round and smaller bricks, with
// shorter lists, keep more blocks resident. A half-warp tests 16 staged Gaussians against
// its footprint with one ballot and three conservative tests: the triangle inequality in
// whitened space (|M (p - mu)| >= |M (c - mu)| - rho4, with rho4 the whitened radius of the
// footprint around its centre c, so a footprint whose centre is farther than sqrt(T) + rho4
// is missed), the truncated ellipsoid's bounding box widened by 3/2 along each axis, and q's
// lower bound from the smallest eigenvalue at the footprint's nearest point; a margin
// absorbs FP32 rounding. It evaluates the hits in ascending Gaussian id, accumulating S and W in registers
// (deterministic; one packed FFMA2 updates a voxel's (S, W) with (v r, r) g).
// Adjoint: one thread per (brick, Gaussian) pair evaluates the brick rows the Gaussian
// reaches (the row shadow, per z-row a quadratic in dy; z-planes whose section of the
// ellipsoid misses the brick's x range are skipped), each row as bx predicated voxel slots in
// packed FP32x2 pairs, so lanes never diverge inside a row. A block takes 256 consecutive
// brick-major pairs (one to three bricks), computes their row masks and counting-sorts them
// by number of rows in shared memory; its four warps then take 32-pair chunks of the sorted
// list, longest first, from a shared counter, so the lanes of a warp run pairs of equal length
// and a warp that drew short pairs moves on to the next chunk (64 registers without spills,
// 8 blocks per SM, 7 for 16-voxel-wide bricks; the y and z cross moments are summed over both
// FP32x2 elements per row to keep the accumulators that small). The per-voxel factors (alpha, alpha I'), alpha = dL/dI / max(W, eps), are
// precomputed into one float2 volume; a block copies those of its first four bricks into
// shared memory (zero outside the grid), so rows read them without range tests; a 16-byte pad
// after every 128 bytes and a 32-byte offset between staged bricks spread the rows that the
// lanes of a warp read at once over the shared-memory banks. Each pair's partial is summed by
// one thread in a fixed voxel order (the processing order does not change results) and goes
// to a per-pair slot (deterministic mode, reduced later in Gaussian-major order) or to one
// float atomic per value (fast mode).
#include <cuda_runtime.h>
#include <stdint.h>


#include "gs_common.cuh"

namespace gs {

constexpr int kFwdChunkPerFoot = 28;  // Gaussians staged per forward round and 4^3 footprint
                                      // (in steps of a factor 2: 56, 112 or 224 records)
constexpr int kBwdThreads = 128;
constexpr int kBwdPairs = 256;        // pairs per adjoint block, taken by warps 32 at a time
constexpr int kBwdStage = 4;          // bricks of per-voxel factors staged per adjoint block
constexpr int kMaxBrickVoxels = 512;  // brick volume limit (x * y * z <= 512)

// Packed FP32x2 arithmetic (one FFMA2 / FADD2 / FMUL2 instruction for two single-precision
// operations; each element is rounded exactly as the scalar fmaf / + / *).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

struct RenderGeo {
    int nx, ny, nz;
    int bsx, bsy, bsz;  // brick shape
    int fx, fy, fz;     // 4^3 footprints per brick along each axis
    int nbx, nby;
    int bsy_shift, bsy_mask;  // row r of a brick is (y, z) = (r & mask, r >> shift)
    float T;            // (log2 e / 2) trunc_sigma^2: a pair contributes when q <= T
    float Tcull;        // cull bound on q: T (1 + 1e-2) + 1e-3
    float sqrtTcull;    // sqrt(Tcull)
    float eps;
    FastDiv dnbx, dnby;  // division by the brick counts along x and y
};

// Brick coordinates (along x, y, z) of brick index b (x fastest).
__device__ __forceinline__ void brick_xyz(int b, const RenderGeo& G, int& bx, int& by, int& bz) {
    const unsigned q = fast_div(static_cast<unsigned>(b), G.dnbx);
    bx = b - static_cast<int>(q) * G.nbx;
    const unsigned r = fast_div(q, G.dnby);
    by = static_cast<int>(q - r * static_cast<unsigned>(G.nby));
    bz = static_cast<int>(r);
}

struct Rec {
    float nmhx, nmlx;        // minus the mean's x head and tail
    float2 nmh_yz, nml_yz;   // minus the mean's (y, z) head and tail
    float2 pc2;              // (P2yz, c2): the dz coefficients of the row terms
    float2 pyc1;             // (Pyy, c1): their dy coefficients
    float pzz, sa, rho4, vr, r, v;
    float lam;               // q per squared voxel distance from the mean, at the least (culling)
    float ex, ey, ez;        // footprint-centre box half-extents (culling)
};

__device__ __forceinline__ Rec load_rec(const float4* s) {
    const float4 a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    Rec R;
    R.nmhx = a.x; R.nmlx = a.y; R.nmh_yz = make_float2(a.z, a.w);
    R.nml_yz = make_float2(b.x, b.y); R.pc2 = make_float2(b.z, b.w);
    R.pyc1 = make_float2(c.x, c.y); R.pzz = c.z; R.sa = c.w;
    R.rho4 = d.y;
    R.ex = d.x; R.ey = d.z; R.ez = d.w;
    R.vr = e.x; R.r = e.y; R.v = e.z; R.lam = e.w;
    return R;
}

// The adjoint's copy of a record: quads 0, 1, 2 and 4 (it never reads quad 3, the footprint
// radius). Slots keep the full 80-byte stride: a 64-byte stride puts the pairs' quads into
// two bank groups and the shared-memory loads conflict.
__device__ __forceinline__ Rec load_rec_bwd(const float4* s) {
    const float4 a = s[0], b = s[1], c = s[2], e = s[4];
    Rec R;
    R.nmhx = a.x; R.nmlx = a.y; R.nmh_yz = make_float2(a.z, a.w);
    R.nml_yz = make_float2(b.x, b.y); R.pc2 = make_float2(b.z, b.w);
    R.pyc1 = make_float2(c.x, c.y); R.pzz = c.z; R.sa = c.w;
    R.rho4 = 0.f;
    R.ex = R.ey = R.ez = 0.f;
    R.vr = e.x; R.r = e.y; R.v = e.z; R.lam = 0.f;
    return R;
}

// Row quantities of the Gaussian for the row through voxel centres (., y, z): the row shadow
// S and the position dx* of the row minimum. One operation sequence for both kernels.
__device__ __forceinline__ void row_terms(const Rec& R, float2 fyz, float& dy, float& dz,
                                          float& S, float& dxs) {
    // (dy, dz) = ((y, z) - head) - tail as one packed pair of additions of the negated mean
    const float2 d = add2(add2(fyz, R.nmh_yz), R.nml_yz);
    dy = d.x;
    dz = d.y;
    // (Pyy dy + P2yz dz, c1 dy + c2 dz) as one packed multiply and one packed FMA
    const float2 t = fma2(R.pyc1, f2(dy, dy), mul2(R.pc2, f2(dz, dz)));
    S = fmaf(dy, t.x, R.pzz * dz * dz);
    dxs = t.y;
}

// x offset of voxel x from the mean, u = ux_base(R, x & ~3) + (x & 3).
__device__ __forceinline__ float ux_base(const Rec& R, int x4) {
    return (float(x4) + R.nmhx) + R.nmlx;
}

// Scaled x offset of voxel x = x4 + k (x4 = x & ~3) from the row minimum, tq = sa (u - dx*),
// taken as tq = fma(k, sa, tq0) from the group's tq0 = sa (ux_base(R, x4) - dx*); then
// q = fma(tq, tq, S). Every kernel uses this operation sequence, so forward and adjoint agree
// on every inclusion q <= T.
__device__ __forceinline__ float tq_base(const Rec& R, int x4, float dxs) {
    return R.sa * (ux_base(R, x4) - dxs);
}

__device__ __forceinline__ float q_of_k(const Rec& R, float tq0, int k, float S) {
    const float tq = (k == 0) ? tq0 : fmaf(float(k), R.sa, tq0);
    return fmaf(tq, tq, S);
}

// Footprint cull: may the Gaussian reach a voxel centre within 3/2 of (cx, cy, cz) per axis?
// Three conservative tests: the whitened triangle inequality; the footprint centre's offset
// from the mean against the truncated ellipsoid's box widened by the footprint's half-width;
// and q's lower bound lam |p - mu|^2 at the footprint's voxel box's nearest point (exact for
// isotropic Gaussians, it drops footprints that only a corner of the ellipsoid grazes between
// voxel centres). (An approximate square root suffices: Tcull carries a 1 % margin over T.)
__device__ __forceinline__ bool foot_hit(const float4* s, float cx, float cy, float cz,
                                         float sqrtTcull) {
    const Rec R = load_rec(s);
    float dy, dz, S, dxs;
    row_terms(R, f2(cy, cz), dy, dz, S, dxs);
    const float ux = (cx + R.nmhx) + R.nmlx;
    const float tq = R.sa * (ux - dxs);
    const float qc = fmaf(tq, tq, S);
    const float ax = fmaxf(fabsf(ux) - 1.5f, 0.0f), ay = fmaxf(fabsf(dy) - 1.5f, 0.0f);
    const float az = fmaxf(fabsf(dz) - 1.5f, 0.0f);
    const float dist2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
    return (sqrt_approx(fmaxf(qc, 0.0f)) - R.rho4 <= sqrtTcull) & (fabsf(ux) <= R.ex) &
           (fabsf(dy) <= R.ey) & (fabsf(dz) <= R.ez) & (R.lam * dist2 <= sqrtTcull * sqrtTcull);
}

// ------------------------------------------------------------------------ forward

template <bool kStats, int kChunk>
__global__ void __launch_bounds__(128, 10) k_render_fwd(const int32_t* __restrict__ brick_off,
                                                    const int32_t* __restrict__ pair_gid,
                                                    const float4* __restrict__ rec4, RenderGeo G,
                                                    float* __restrict__ I, float* __restrict__ W,
                                                    unsigned long long* __restrict__ stats) {
    pdl_enter();
    __shared__ float4 srec[kChunk][REC_F4];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nthreads = blockDim.x;
    const int b = blockIdx.x;
    int bx, by, bz;
    brick_xyz(b, G, bx, by, bz);
    // half-warp per 4^3 footprint; a lane owns one x-row of 4 voxels
    const int foot = tid >> 4, l16 = lane & 15;
    const int n_foot = G.fx * G.fy * G.fz;
    const bool foot_ok = foot < n_foot;
    const int f = foot_ok ? foot : 0;
    const int wx = f % G.fx, wy = (f / G.fx) % G.fy, wz = f / (G.fx * G.fy);
    const int ox = bx * G.bsx + wx * 4, oy = by * G.bsy + wy * 4, oz = bz * G.bsz + wz * 4;
    const int y = oy + (l16 & 3), z = oz + (l16 >> 2);
    const float2 fyz = f2(float(y), float(z));
    const float cx = float(ox) + 1.5f, cy = float(oy) + 1.5f, cz = float(oz) + 1.5f;
    const unsigned half_sel = (lane < 16) ? 0x0000ffffu : 0xffff0000u;

    float2 SW[4];  // (S, W) of the lane's four voxels
#pragma unroll
    for (int xi = 0; xi < 4; ++xi) SW[xi] = f2(0.f, 0.f);
    unsigned long long n_eff = 0, n_eval = 0;
    const int start = brick_off[b], end = brick_off[b + 1];
    for (int c0 = start; c0 < end; c0 += kChunk) {
        const int cnt = min(kChunk, end - c0);
        if (c0 != start) __syncthreads();  // the previous chunk's records are no longer read
        for (int k = tid; k < cnt; k += nthreads) {  // a thread stages one record
            const float4* src = rec4 + int64_t(pair_gid[c0 + k]) * REC_F4;
#pragma unroll
            for (int part = 0; part < REC_F4; ++part) srec[k][part] = src[part];
        }
        __syncthreads();
        for (int k0 = 0; k0 < cnt; k0 += 16) {
            // lane l16 of each half tests Gaussian k0 + l16 against the half's footprint
            const int k = k0 + l16;
            const bool hit = foot_ok && (k < cnt) && foot_hit(srec[k], cx, cy, cz, G.sqrtTcull);
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            unsigned mask = (bal & half_sel) >> (lane & 16);
            // each half takes its hits in ascending Gaussian id (per voxel the order of Eq. 3);
            // the halves run their own trip counts and meet again at the next ballot
            while (mask) {
                {
                    const int kk = k0 + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const Rec R = load_rec(srec[kk]);
                    float dy, dz, Sr, dxs;
                    row_terms(R, fyz, dy, dz, Sr, dxs);
                    const float tq0 = tq_base(R, ox, dxs);
                    const float2 vrr = f2(R.vr, R.r);
#pragma unroll
                    for (int xi = 0; xi < 4; ++xi) {
                        const float q = q_of_k(R, tq0, xi, Sr);
                        if (q <= G.T) {
                            const float g = ex2_approx(-q);
                            SW[xi] = fma2(vrr, f2(g, g), SW[xi]);
                        }
                        if (kStats) {
                            n_eff += (y < G.ny && z < G.nz && ox + xi < G.nx && q <= G.T) ? 1 : 0;
                            n_eval += 1;
                        }
                    }
                }
            }
        }
    }
    if (foot_ok && y < G.ny && z < G.nz) {
        const int64_t row = (int64_t(z) * G.ny + y) * G.nx + ox;
        float Iv[4];
#pragma unroll
        for (int xi = 0; xi < 4; ++xi) Iv[xi] = SW[xi].x / (SW[xi].y > G.eps ? SW[xi].y : G.eps);
        if (ox + 3 < G.nx && (G.nx & 3) == 0) {
            *reinterpret_cast<float4*>(I + row) = make_float4(Iv[0], Iv[1], Iv[2], Iv[3]);
            *reinterpret_cast<float4*>(W + row) = make_float4(SW[0].y, SW[1].y, SW[2].y, SW[3].y);
        } else {
#pragma unroll
            for (int xi = 0; xi < 4; ++xi)
                if (ox + xi < G.nx) {
                    I[row + xi] = Iv[xi];
                    W[row + xi] = SW[xi].y;
                }
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

// Rows of the brick (index rz * bsy + ry) that the Gaussian may reach: per z-row the row
// shadow S(dy, dz) <= Tcull holds on the y-interval yc(dz) +- hw(dz), with
// yc = mu_y - (P2yz / 2 Pyy) dz and hw^2 = Tcull / Pyy - c3 dz^2,
// c3 = (Pzz - P2yz^2 / 4 Pyy) / Pyy (the interval is padded; Tcull carries a 1 % margin).
// A z-plane whose section of the truncated ellipsoid misses the brick's x range is skipped.
// The mask is a conservative superset only (the rows themselves test q <= T), so the plane
// offsets are taken as dz(z0) + rz and positions relative to the brick, inside the padding.
// kBY, kBZ: the brick's y and z sizes at compile time (0: taken from G); the fitting
// workload's 8^3 bricks and the paper's 8 x 8 x 4 ones have their own unrolled copies.
template <int kBY, int kBZ>
__device__ __forceinline__ unsigned long long brick_row_mask(const Rec& R, const RenderGeo& G,
                                                             int x0, int y0, int z0) {
    const int bsy = kBY > 0 ? kBY : G.bsy;
    const int bsz = kBZ > 0 ? kBZ : G.bsz;
    unsigned long long mask = 0;
    const float ipyy = __fdividef(1.0f, R.pyc1.x);
    const float k1 = -0.5f * (R.pc2.x * ipyy);
    const float nc3 = -(R.pzz - 0.25f * R.pc2.x * (R.pc2.x * ipyy)) * ipyy;
    const float h0 = G.Tcull * ipyy;
    const float mu_y = -(R.nmh_yz.x + R.nml_yz.x);
    const float mu_x = -(R.nmhx + R.nmlx);
    const float pad = 1e-3f + 1e-5f * fabsf(mu_y);
    // the section's x extent through plane dz: centre mu_x + (c1 k1 + c2) dz, half-width
    // hw_y sqrt(Pyy / a + c1^2) (hw_y the y half-width of the same section); tested as
    // |centre - brick centre| <= half-width + brick half-width
    const float kx = fmaf(R.pyc1.y, k1, R.pc2.y);
    const float lam = sqrt_approx(fmaf(R.pyc1.x, __fdividef(1.0f, R.sa * R.sa), R.pyc1.y * R.pyc1.y));
    const float half_bx = 0.5f * float(G.bsx - 1);
    const float xrel = mu_x - (float(x0) + half_bx);
    const float padx = 1e-3f + 1e-5f * fabsf(mu_x) + half_bx;
    const float yrel = mu_y - float(y0);
    const float dz0 = (float(z0) + R.nmh_yz.y) + R.nml_yz.y;
    const unsigned full = (1u << bsy) - 1u;
#pragma unroll (kBZ > 0 ? kBZ : 1)
    for (int rz = 0; rz < bsz; ++rz) {
        const float dz = dz0 + float(rz);
        const float hw2 = fmaf(nc3 * dz, dz, h0);
        const float sh = sqrt_approx(fmaxf(hw2, 0.0f));
        const bool in_x = fabsf(fmaf(kx, dz, xrel)) <= fmaf(sh, lam, padx);
        const float yc = fmaf(k1, dz, yrel);
        const float hw = sh + pad;
        // rows ceil(yc - hw) .. floor(yc + hw), clamped to the brick; empty when ia > ib
        const int ia = min(max(__float2int_ru(yc - hw), 0), bsy);
        const int ib = min(max(__float2int_rd(yc + hw), -1), bsy - 1);
        const unsigned bits = (full << ia) & (full >> (bsy - 1 - ib));
        if (hw2 >= 0.0f && in_x) mask |= static_cast<unsigned long long>(bits) << (rz * bsy);
    }
    return mask;
}

// Per-voxel adjoint factors (alpha, alpha I'): dL/dw_i = v_i alpha - alpha I' with
// alpha = dL/dI / max(W, eps) and I' = I where W > eps, else 0 (Eq. 5; below the floor
// I = S / eps, so dI/dw_i = v_i / eps).
__global__ void __launch_bounds__(256) k_bwd_prep(const float* __restrict__ Iv,
                                                  const float* __restrict__ Wv,
                                                  const float* __restrict__ dIv, int64_t n,
                                                  float eps, float2* __restrict__ aip) {
    pdl_enter();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float w = Wv[i], gI = dIv[i];
        const float al = gI / (w > eps ? w : eps);
        aip[i] = make_float2(al, (w > eps) ? al * Iv[i] : 0.0f);
    }
}

// Adjoint sums of one (brick, Gaussian) pair, with h = gamma g (gamma = dL/dw) per voxel.
// A brick row of bx voxels is taken as bx/2 voxel pairs (p, p + bx/2); element e of a float2
// holds the sums over the voxels p + e bx/2 (offset u = uc_e + p from the mean along x).
struct AdjAcc {
    float2 h, p1;         // sum h, sum h p
    float2 pq;            // sum h p (p + 1) / 2  (so sum h p^2 = 2 pq - p1)
    float2 ag;            // sum alpha g
    float hy, hz;         // sum h dy, sum h dz over both elements
    float oy, oz;         // sum h o dy, sum h o dz, o = p + e bx/2 the slot's offset from uc_0
    float yy, zz, yz;     // sum h dy^2, sum h dz^2, sum h dy dz
};

// The rows of one (brick, Gaussian) pair: for each row in the mask, bx voxel slots in bx/2
// packed pairs, with the factors read from the block's staged copy (kStaged: per row, float4
// (alpha_p, alpha_{p+bx/2}, -alpha I'_p, -alpha I'_{p+bx/2}) for p < bx/2) or from the volume.
// The exponent of every slot takes the forward's operation sequence element by element, so
// both kernels agree on every inclusion q <= T. The slot moments along x are running sums
// over p (descending), which need no per-slot constants.
template <int BX, bool kStaged>
__device__ __forceinline__ void adjoint_rows(const Rec& R, unsigned long long m, const RenderGeo& G,
                                             int x0, int y0, int z0,
                                             const float4* __restrict__ sfac_b,
                                             const float2* __restrict__ aip, AdjAcc& A) {
    constexpr int P = BX / 2;                    // voxel pairs per row
    constexpr int NT = (BX >= 8) ? BX / 8 : 1;   // packed group bases per row
    const int x1 = min(x0 + BX, G.nx) - 1;
    const float2 sa2 = f2(R.sa, R.sa), v2 = f2(R.v, R.v);
    // x offsets of the 4-voxel groups that pair p reads: (group p/4, group p/4 + bx/8)
    float2 uxp[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j)
        uxp[j] = (BX >= 8) ? f2(ux_base(R, x0 + 4 * j), ux_base(R, x0 + 4 * j + P))
                           : f2(ux_base(R, x0), ux_base(R, x0));
    while (m) {
        const int r = __ffsll(static_cast<long long>(m)) - 1;
        m &= m - 1;
        const int y = y0 + (r & G.bsy_mask), z = z0 + (r >> G.bsy_shift);
        float dy, dz, S, dxs;
        row_terms(R, f2(float(y), float(z)), dy, dz, S, dxs);
        const float2 S2 = f2(S, S), nd2 = f2(-dxs, -dxs);
        float2 tq0[NT];  // tq_base of each group, the forward's sa * (ux - dx*)
#pragma unroll
        for (int j = 0; j < NT; ++j) tq0[j] = mul2(sa2, add2(uxp[j], nd2));
        const bool row_in = kStaged || ((y < G.ny) && (z < G.nz));
        const float2* arow = kStaged ? nullptr
                                     : aip + (int64_t(min(z, G.nz - 1)) * G.ny + min(y, G.ny - 1)) * G.nx + x0;
        float2 rs = f2(0.f, 0.f), m1 = f2(0.f, 0.f), qs = f2(0.f, 0.f);
#pragma unroll
        for (int p = P - 1; p >= 0; --p) {
            // exponent of the two slots: in-group index k, group base tq0
            float2 tq;
            if (BX >= 8) {
                const int k = p & 3;
                tq = (k == 0) ? tq0[p >> 2] : fma2(f2(float(k), float(k)), sa2, tq0[p >> 2]);
            } else {
                tq = fma2(f2(float(p), float(p + 2)), sa2, tq0[0]);
            }
            const float2 q = fma2(tq, tq, S2);
            const float2 g = f2((q.x <= G.T) ? ex2_approx(-q.x) : 0.0f,
                                (q.y <= G.T) ? ex2_approx(-q.y) : 0.0f);
            float2 al, nai;  // (alpha, -alpha I') of the two slots, zero outside the grid
            if (kStaged) {
                const float4 f = sfac_b[r * P + ((r * P) >> 3) + p];
                al = f2(f.x, f.y);
                nai = f2(f.z, f.w);
            } else {
                const float2 fa = (row_in && x0 + p <= x1) ? arow[p] : f2(0.f, 0.f);
                const float2 fb = (row_in && x0 + p + P <= x1) ? arow[p + P] : f2(0.f, 0.f);
                al = f2(fa.x, fb.x);
                nai = f2(-fa.y, -fb.y);
            }
            const float2 h = mul2(fma2(v2, al, nai), g);
            A.ag = fma2(al, g, A.ag);
            rs = add2(rs, h);            // sum over slots >= p
            if (p >= 1) {
                m1 = add2(m1, rs);       // ends as sum h p
                qs = add2(qs, m1);       // ends as sum h p (p + 1) / 2
            }
        }
        A.h = add2(A.h, rs);
        A.p1 = add2(A.p1, m1);
        A.pq = add2(A.pq, qs);
        const float s0 = rs.x + rs.y;
        const float s1 = fmaf(float(P), rs.y, m1.x + m1.y);  // sum h o over the row
        A.hy = fmaf(s0, dy, A.hy);
        A.hz = fmaf(s0, dz, A.hz);
        A.oy = fmaf(s1, dy, A.oy);
        A.oz = fmaf(s1, dz, A.oz);
        const float ty = dy * s0;
        A.yy = fmaf(ty, dy, A.yy);
        A.yz = fmaf(ty, dz, A.yz);
        A.zz = fmaf(dz * s0, dz, A.zz);
    }
}

template <int BX, bool kDet>
__global__ void __launch_bounds__(kBwdThreads, (BX == 16 ? 7 : 8)) k_render_bwd(
    const int32_t* __restrict__ pair_gid, const int32_t* __restrict__ pair_gmj,
    const int32_t* __restrict__ pair_brick, const int64_t* __restrict__ npairs, int64_t capacity,
    const float4* __restrict__ rec4, RenderGeo G, const float2* __restrict__ aip,
    float* __restrict__ part, float* __restrict__ gacc) {
    pdl_enter();
    constexpr int kPer = kBwdPairs / kBwdThreads;  // pairs per thread in the prologue
    constexpr int kWarps = kBwdThreads / 32;
    // staged bricks 2 float4 apart beyond their padded size: rows of different bricks that the
    // lanes of a warp read at once fall on different banks
    constexpr int kStageStride = kMaxBrickVoxels / 2 + kMaxBrickVoxels / 16 + 2;
    __shared__ float4 sfac[kBwdStage * kStageStride];
    __shared__ unsigned long long smask[kBwdPairs];
    __shared__ int sgid[kBwdPairs];
    __shared__ unsigned short sorder[kBwdPairs];
    __shared__ unsigned char sstage[kBwdPairs];
    __shared__ int hist[66];
    __shared__ int cursor[66];
    __shared__ int sbrick[kBwdStage];
    __shared__ int gcount[kBwdPairs / 32];
    __shared__ int chunk_next;
    int64_t P = *npairs;
    if (P < 0 || P > capacity) P = 0;
    const int64_t base = int64_t(blockIdx.x) * kBwdPairs;
    if (base >= P) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nvalid = static_cast<int>(min(int64_t(kBwdPairs), P - base));
    for (int k = tid; k < 66; k += kBwdThreads) {
        hist[k] = 0;
        cursor[k] = 0;
    }
    if (tid == 0) chunk_next = 0;
    // distinct bricks of the block's pairs (brick-major order: a new brick starts a run);
    // thread tid holds pairs tid + h * 128 (32-pair group warp + 4 h)
    int b_t[kPer], gidv[kPer];
    unsigned bal[kPer];
    bool newb[kPer];
#pragma unroll
    for (int h = 0; h < kPer; ++h) {
        const int q = tid + h * kBwdThreads;
        b_t[h] = 0;
        gidv[h] = 0;
        newb[h] = false;
        if (q < nvalid) {
            b_t[h] = pair_brick[base + q];
            gidv[h] = pair_gid[base + q];
            newb[h] = (q == 0) || (b_t[h] != pair_brick[base + q - 1]);
        }
        bal[h] = __ballot_sync(0xffffffffu, newb[h]);
        if (lane == 0) gcount[warp + h * kWarps] = __popc(bal[h]);
    }
    __syncthreads();
    int n_bricks = 0;
#pragma unroll
    for (int g = 0; g < kBwdPairs / 32; ++g) n_bricks += gcount[g];
    // row mask of each pair, its staged brick, histogram of row counts (most first)
    int bucket[kPer];
#pragma unroll
    for (int h = 0; h < kPer; ++h) {
        const int q = tid + h * kBwdThreads;
        const int grp = warp + h * kWarps;
        bucket[h] = 0;
        if (q < nvalid) {
            int run_before = 0;
            for (int g = 0; g < grp; ++g) run_before += gcount[g];
            const int kb = run_before + __popc(bal[h] & ((1u << lane) - 1u)) + (newb[h] ? 1 : 0) - 1;
            if (newb[h] && kb < kBwdStage) sbrick[kb] = b_t[h];
            sstage[q] = static_cast<unsigned char>(min(kb, kBwdStage));
            const int gid = gidv[h];
            sgid[q] = gid;
            int bxx, by, bz;
            brick_xyz(b_t[h], G, bxx, by, bz);
            const Rec Rm = load_rec_bwd(rec4 + int64_t(gid) * REC_F4);
            const int mx0 = bxx * G.bsx, my0 = by * G.bsy, mz0 = bz * G.bsz;
            const unsigned long long m = (G.bsy == 8 && G.bsz == 8)
                                             ? brick_row_mask<8, 8>(Rm, G, mx0, my0, mz0)
                                             : (G.bsy == 8 && G.bsz == 4)
                                                   ? brick_row_mask<8, 4>(Rm, G, mx0, my0, mz0)
                                                   : brick_row_mask<0, 0>(Rm, G, mx0, my0, mz0);
            smask[q] = m;
            bucket[h] = 64 - __popcll(static_cast<long long>(m));
            atomicAdd(&hist[bucket[h]], 1);
        }
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix of the 65 bucket counts: lane l owns buckets 3l..3l+2
        int c[3], t = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int bk = 3 * lane + k;
            c[k] = bk <= 64 ? hist[bk] : 0;
            t += c[k];
        }
        int incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int bk = 3 * lane + k;
            if (bk <= 64) hist[bk] = run;
            run += c[k];
        }
    }
    // per-voxel factors of the first kBwdStage bricks into shared memory, zero outside the
    // grid, so the row loop needs no range tests; per row and voxel pair (p, p + bx/2) one
    // float4 (alpha_p, alpha_{p+bx/2}, -alpha I'_p, -alpha I'_{p+bx/2}), float4 index
    // i = row * bx/2 + p stored at i + i/8 (rows of the lanes of a warp fall on other banks)
    const int n_stage = min(n_bricks, kBwdStage);
    constexpr int kPairs = BX / 2;
    const int bpairs = kPairs * G.bsy * G.bsz;
    for (int k = 0; k < n_stage; ++k) {
        const int b = sbrick[k];
        int bxx, byy, bzz;
        brick_xyz(b, G, bxx, byy, bzz);
        const int x0 = bxx * BX, y0 = byy * G.bsy, z0 = bzz * G.bsz;
        float4* dst = &sfac[k * kStageStride];
        if (x0 + BX <= G.nx && y0 + G.bsy <= G.ny && z0 + G.bsz <= G.nz && (G.nx & 1) == 0) {
            // brick inside the grid, rows 16-byte aligned: float4 loads of voxels (2c, 2c+1)
            // and (2c+P, 2c+P+1) give the entries of pairs 2c and 2c+1
            constexpr int kHalf = kPairs / 2;
            for (int e = tid; e < bpairs / 2; e += kBwdThreads) {
                const int r = e / kHalf, c = e - r * kHalf;
                const int y = y0 + (r & G.bsy_mask), z = z0 + (r >> G.bsy_shift);
                const float2* src = aip + (int64_t(z) * G.ny + y) * G.nx + x0 + 2 * c;
                const float4 fa = *reinterpret_cast<const float4*>(src);
                const float4 fb = *reinterpret_cast<const float4*>(src + kPairs);
                dst[r * kPairs + ((r * kPairs) >> 3) + 2 * c] = make_float4(fa.x, fb.x, -fa.y, -fb.y);
                dst[r * kPairs + ((r * kPairs) >> 3) + 2 * c + 1] = make_float4(fa.z, fb.z, -fa.w, -fb.w);
            }
            continue;
        }
        for (int e = tid; e < bpairs; e += kBwdThreads) {
            const int r = e / kPairs, pp = e - r * kPairs;
            const int y = y0 + (r & G.bsy_mask), z = z0 + (r >> G.bsy_shift);
            const int xa = x0 + pp, xb = xa + kPairs;
            const float2* src = aip + (int64_t(min(z, G.nz - 1)) * G.ny + min(y, G.ny - 1)) * G.nx;
            const bool row_ok = y < G.ny && z < G.nz;
            const float2 fa = (row_ok && xa < G.nx) ? src[xa] : make_float2(0.f, 0.f);
            const float2 fb = (row_ok && xb < G.nx) ? src[xb] : make_float2(0.f, 0.f);
            dst[e + (e >> 3)] = make_float4(fa.x, fb.x, -fa.y, -fb.y);
        }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < kPer; ++h) {
        const int q = tid + h * kBwdThreads;
        if (q < nvalid)
            sorder[hist[bucket[h]] + atomicAdd(&cursor[bucket[h]], 1)] = static_cast<unsigned short>(q);
    }
    __syncthreads();
    // warps take 32-pair chunks of the sorted list (longest first) until none is left, so a
    // warp that drew short pairs goes on with the next chunk instead of idling
    const int nchunks = (nvalid + 31) / 32;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&chunk_next, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) break;
        const int rank = c * 32 + lane;
        if (rank >= nvalid) continue;
        const int lt = sorder[rank];
        const int64_t i = base + lt;
        const unsigned long long m = smask[lt];
        if (m == 0ull) {
            // a pair whose Gaussian reaches none of the brick's rows (the count-sorted list puts
            // them in the last chunks): its partial is zero, with no record or brick to load
            if (kDet) {
                float4* dst = reinterpret_cast<float4*>(part + int64_t(pair_gmj[i]) * GRAD_FLOATS);
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                dst[0] = z4;
                dst[1] = z4;
                dst[2] = z4;
            }
            continue;
        }
        const int b = pair_brick[i];
        int bx, by, bz;
        brick_xyz(b, G, bx, by, bz);
        const int x0 = bx * BX, y0 = by * G.bsy, z0 = bz * G.bsz;
        const int stage = sstage[lt];
        const Rec R = load_rec_bwd(rec4 + int64_t(sgid[lt]) * REC_F4);
        AdjAcc A;
        A.h = A.p1 = A.pq = A.ag = f2(0.f, 0.f);
        A.hy = A.hz = A.oy = A.oz = A.yy = A.zz = A.yz = 0.f;
        if (stage < kBwdStage)
            adjoint_rows<BX, true>(R, m, G, x0, y0, z0, &sfac[stage * kStageStride],
                                   aip, A);
        else
            adjoint_rows<BX, false>(R, m, G, x0, y0, z0, nullptr, aip, A);
        // moments about the mean: slot p of element e sits at u = uc_e + p along x
        const float uc0 = ux_base(R, x0);
        const float uc1 = (BX >= 8) ? ux_base(R, x0 + BX / 2) : uc0 + 2.0f;
        float m1x = fmaf(uc0, A.h.x, A.p1.x) + fmaf(uc1, A.h.y, A.p1.y);
        // sum h u^2 = uc^2 sum h + 2 uc sum h p + (2 pq - p1)
        float m2xx = fmaf(uc0, fmaf(uc0, A.h.x, 2.0f * A.p1.x), fmaf(2.0f, A.pq.x, -A.p1.x)) +
                     fmaf(uc1, fmaf(uc1, A.h.y, 2.0f * A.p1.y), fmaf(2.0f, A.pq.y, -A.p1.y));
        // (the y, z cross moments take slot o at uc_0 + o)
        float m2xy = fmaf(uc0, A.hy, A.oy);
        float m2xz = fmaf(uc0, A.hz, A.oz);
        float m1y = A.hy, m1z = A.hz;
        float m2yy = A.yy, m2zz = A.zz, m2yz = A.yz;
        const float dvp = A.ag.x + A.ag.y, dr = A.h.x + A.h.y;
        const float rr = R.r;
        const float dv = rr * dvp;
        m1x *= rr; m1y *= rr; m1z *= rr;
        m2xx *= rr; m2yy *= rr; m2zz *= rr; m2xy *= rr; m2xz *= rr; m2yz *= rr;
        if (kDet) {
            const int64_t j = pair_gmj[i];
            float4* dst = reinterpret_cast<float4*>(part + j * GRAD_FLOATS);
            dst[0] = make_float4(m1x, m1y, m1z, m2xx);
            dst[1] = make_float4(m2yy, m2zz, m2xy, m2xz);
            dst[2] = make_float4(m2yz, dv, dr, 0.f);
        } else {
            float* dst = gacc + int64_t(sgid[lt]) * GRAD_FLOATS;
            const float vals[11] = {m1x, m1y, m1z, m2xx, m2yy, m2zz, m2xy, m2xz, m2yz, dv, dr};
#pragma unroll
            for (int q = 0; q < 11; ++q) atomicAdd(dst + q, vals[q]);
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
    pdl_enter();
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
    G.fx = b.bx / 4; G.fy = b.by / 4; G.fz = b.bz / 4;
    G.bsy_shift = (b.by == 4) ? 2 : ((b.by == 8) ? 3 : 4);
    G.bsy_mask = b.by - 1;
    G.nbx = b.nbx; G.nby = b.nby;
    G.T = kHalfLog2e * cfg->trunc_sigma * cfg->trunc_sigma;
    G.Tcull = G.T * (1.0f + 1e-2f) + 1e-3f;
    G.sqrtTcull = sqrtf(G.Tcull);
    G.eps = cfg->eps;
    G.dnbx = make_fastdiv(static_cast<unsigned>(b.nbx));
    G.dnby = make_fastdiv(static_cast<unsigned>(b.nby));
    return G;
}

gs_status render_fwd_impl(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                          float* I, float* W, unsigned long long* stats, cudaStream_t st) {
    RenderGeo G = make_geo(grid, cfg);
    const int n_foot = G.fx * G.fy * G.fz;
    const int threads = 32 * ((n_foot + 1) / 2);  // a half-warp per footprint
    // records staged per round about in proportion to the footprints (the lists of smaller
    // bricks are shorter), so that smaller bricks keep more blocks resident
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    auto go = [&](auto kernel) {
        launch_k(kernel, dim3(bins->n_bricks), dim3(threads), 0, st, bins->brick_off, bins->pair_gid,
            rec4, G, I, W, stats);
    };
    if (n_foot >= 6)
        stats ? go(k_render_fwd<true, 8 * kFwdChunkPerFoot>) : go(k_render_fwd<false, 8 * kFwdChunkPerFoot>);
    else if (n_foot >= 3)
        stats ? go(k_render_fwd<true, 4 * kFwdChunkPerFoot>) : go(k_render_fwd<false, 4 * kFwdChunkPerFoot>);
    else
        stats ? go(k_render_fwd<true, 2 * kFwdChunkPerFoot>) : go(k_render_fwd<false, 2 * kFwdChunkPerFoot>);
    return last_launch_status();
}

gs_status bind_workspace(void* base, size_t bytes, int64_t n_gauss, int64_t capacity,
                         const gs_grid* grid, const gs_config* cfg, Workspace* ws);
bool bins_match(const gs_bins* b, const gs_grid* grid, const gs_config* cfg);

gs_status launch_bwd_prep(const float* I, const float* W, const float* dI, const RenderGeo& G,
                          const Workspace& ws, cudaStream_t st) {
    const int64_t nv = int64_t(G.nx) * G.ny * G.nz;
    const int64_t pb = (nv + 255) / 256;
    launch_k(k_bwd_prep, dim3(static_cast<unsigned>(pb < 65536 ? pb : 65536)), dim3(256), 0, st, I,
        W, dI, nv, G.eps, ws.aip);
    return last_launch_status();
}

template <int BX, bool kDet>
static gs_status launch_bwd_pairs(const gs_bins* bins, const RenderGeo& G, const Workspace& ws,
                                  cudaStream_t st) {
    if (bins->capacity == 0) return GS_OK;
    const unsigned gb = static_cast<unsigned>((bins->capacity + kBwdPairs - 1) / kBwdPairs);
    const float4* rec4 = reinterpret_cast<const float4*>(bins->rec);
    launch_k(k_render_bwd<BX, kDet>, dim3(gb), dim3(kBwdThreads), 0, st, bins->pair_gid,
        bins->pair_gmj, bins->pair_brick, bins->d_npairs, bins->capacity, rec4, G, ws.aip,
        kDet ? ws.part : nullptr, kDet ? nullptr : ws.gacc);
    return last_launch_status();
}

// Adjoint render kernel over ws.aip (already prepared): per-pair partials (deterministic) or
// atomically accumulated ws.gacc (fast; zeroed here).
gs_status launch_adjoint_pairs(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                               const Workspace& ws, cudaStream_t st) {
    RenderGeo G = make_geo(grid, cfg);
    const int64_t N = bins->n_gauss;
    if (!cfg->deterministic && N > 0 &&
        cudaMemsetAsync(ws.gacc, 0, sizeof(float) * GRAD_FLOATS * N, st) != cudaSuccess)
        return GS_ERR_CUDA;
    const bool det = cfg->deterministic != 0;
    switch (G.bsx) {
        case 4: return det ? launch_bwd_pairs<4, true>(bins, G, ws, st) : launch_bwd_pairs<4, false>(bins, G, ws, st);
        case 8: return det ? launch_bwd_pairs<8, true>(bins, G, ws, st) : launch_bwd_pairs<8, false>(bins, G, ws, st);
        case 16: return det ? launch_bwd_pairs<16, true>(bins, G, ws, st) : launch_bwd_pairs<16, false>(bins, G, ws, st);
    }
    return GS_ERR_INVALID_ARG;
}

// Render-space adjoint into ws.gacc [N, 12] (no parameter chain).
static gs_status render_bwd_geo(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                                const float* I, const float* W, const float* dI,
                                const Workspace& ws, cudaStream_t st) {
    RenderGeo G = make_geo(grid, cfg);
    gs_status s = launch_bwd_prep(I, W, dI, G, ws, st);
    if (s != GS_OK) return s;
    s = launch_adjoint_pairs(bins, grid, cfg, ws, st);
    if (s != GS_OK) return s;
    const int64_t N = bins->n_gauss;
    if (cfg->deterministic && N > 0) {
        launch_k(k_pair_reduce, dim3(static_cast<unsigned>((N + 255) / 256)), dim3(256), 0, st,
            ws.part, bins->gm_off, bins->d_npairs, bins->capacity, N, ws.gacc);
        s = last_launch_status();
    }
    return s;
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
    s = render_bwd_geo(bins, grid, cfg, I, W, dI, w, st);
    if (s != GS_OK) return s;
    if (bins->n_gauss == 0) return GS_OK;
    return launch_param_bwd(params, w.gacc, bins->n_gauss, grid, cfg, dparams, st);
}
