// gs_bin.cu -- Sec. 3.3 brick intersection and binning: per-Gaussian activation and bounds,
// per-brick Gaussian lists built by count / exclusive scan / stable radix scatter.
//
// Pipeline of gs_bin_bricks (all asynchronous on one stream):
//   k_preprocess   one thread per Gaussian: validity, FP32 brick range (fixed operation order,
//                  bit-exact against the oracle's binning specification), render record; it
//                  also clears the radix passes' two digit-count buffers.
//   scan           exclusive scan of per-Gaussian pair counts -> gm_off; its last thread stores
//                  the total as d_npairs and flags GS_STATUS_CAPACITY when it exceeds the
//                  bins' capacity.
//   k_emit         Gaussian-major pair emission (brick key, owner), staged per block in shared
//                  memory so the stores are coalesced.
//   radix passes   stable LSD radix sort of the brick keys, 8 bits per pass: per-tile digit
//                  counts (the first pass's added up by k_emit, each later pass's by the
//                  scatter before it), a digit-major scan, and a stable scatter whose in-tile
//                  ranks come from warp match masks. Stability keeps ascending Gaussian ids inside
//                  each brick, so the lists are deterministic.
//                  The last pass stores pair_brick (key), pair_gmj (Gaussian-major position)
//                  and pair_gid (owner) directly.
//   k_brick_off    brick_off from the boundaries of the sorted keys.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "gs_common.cuh"

namespace gs {

// ============================================================================ validation

gs_status validate_grid_cfg(const gs_grid* g, const gs_config* c) {
    if (!g || !c) return GS_ERR_INVALID_ARG;
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return GS_ERR_INVALID_ARG;
    if (int64_t(g->nx) * g->ny * g->nz > (int64_t(1) << 31) - 1) return GS_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) {
        if (!(g->h[k] > 0.0f) || !isfinite(g->h[k]) || !isfinite(g->origin[k]))
            return GS_ERR_INVALID_ARG;
        if (c->brick[k] <= 0 || c->brick[k] % 4 != 0) return GS_ERR_INVALID_ARG;
    }
    // rows of bx voxels along x (bx in {4, 8, 16}), at most 64 rows per brick
    if (c->brick[0] != 4 && c->brick[0] != 8 && c->brick[0] != 16) return GS_ERR_INVALID_ARG;
    if (c->brick[1] != 4 && c->brick[1] != 8 && c->brick[1] != 16) return GS_ERR_INVALID_ARG;
    if (c->brick[1] * c->brick[2] > 64) return GS_ERR_INVALID_ARG;
    if (c->brick[0] * c->brick[1] * c->brick[2] > 512) return GS_ERR_INVALID_ARG;
    if (!(c->trunc_sigma > 0.0f) || !isfinite(c->trunc_sigma)) return GS_ERR_INVALID_ARG;
    if (!(c->eps > 0.0f)) return GS_ERR_INVALID_ARG;
    if (c->signal_mode != 0 && c->signal_mode != 1) return GS_ERR_INVALID_ARG;
    if ((c->a_act != 0 && c->a_act != 1) || (c->t_act != 0 && c->t_act != 1))
        return GS_ERR_INVALID_ARG;
    BrickGeom b = brick_geom(g, c);
    if (int64_t(b.nbx) * b.nby * b.nbz > (int64_t(1) << 30)) return GS_ERR_INVALID_ARG;
    return GS_OK;
}

// ============================================================================ scan

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix and the
// block total. smem must hold 32 values. Ends with a barrier (smem reusable afterwards).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    T inc = warp_inclusive_scan(v, lane);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nwarps ? smem[lane] : T(0);
        s = warp_inclusive_scan(s, lane);
        smem[lane] = s;
    }
    __syncthreads();
    T prefix = (warp > 0 ? smem[warp - 1] : T(0)) + inc - v;
    *total = smem[nwarps - 1];
    __syncthreads();
    return prefix;
}

// Per-block sums (64-bit) of kScanTile consecutive values.
template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Tin* __restrict__ in, int64_t n,
                                                              long long* __restrict__ sums) {
    pdl_enter();
    __shared__ long long sm[32];
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += static_cast<long long>(in[base + i]);
    long long tot;
    block_exclusive_scan(s, sm, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of each block, offset by the block sums before it (nullptr: single block).
// kRaw: offs holds the raw block sums and each block adds up those before its own (few
// blocks); otherwise offs is already scanned.
template <typename Tin, typename Tout, bool kRaw>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin* __restrict__ in, Tout* out,
                                                            int64_t n, const long long* __restrict__ offs,
                                                            long long* total, CapCheck cc) {
    pdl_enter();
    __shared__ long long sm[32];
    long long boff = 0;
    if (kRaw) {
        long long o = 0;
        for (int k = threadIdx.x; k < static_cast<int>(blockIdx.x); k += kScanThreads) o += offs[k];
        block_exclusive_scan(o, sm, &boff);
    }
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    long long vals[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        vals[i] = (base + i < n) ? static_cast<long long>(in[base + i]) : 0;
        s += vals[i];
    }
    long long tot;
    long long run = block_exclusive_scan(s, sm, &tot);
    if (kRaw) run += boff;
    else if (offs) run += offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = static_cast<Tout>(run);
        run += vals[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
        if (total) *total = run;
        if (cc.npairs) {
            *cc.npairs = run;
            if (run > cc.capacity) atomicOr(cc.status, GS_STATUS_CAPACITY);
        }
    }
}

template <typename Tin, typename Tout>
static gs_status scan_rec(const Tin* in, Tout* out, int64_t n, long long* total, long long* tmp,
                          int64_t tmp_len, cudaStream_t st, CapCheck cc) {
    if (n <= 0) return GS_OK;
    if (n <= kScanTile) {
        launch_k(k_scan_down<Tin, Tout, false>, dim3(1), dim3(kScanThreads), 0, st, in, out, n,
            nullptr, total, cc);
        return last_launch_status();
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb + 1 > tmp_len) return GS_ERR_WORKSPACE;
    long long* sums = tmp;
    launch_k(k_scan_reduce<Tin>, dim3(static_cast<unsigned>(nb)), dim3(kScanThreads), 0, st, in, n,
        sums);
    gs_status s = last_launch_status();
    if (s != GS_OK) return s;
    if (nb <= kScanTile) {  // few blocks: each adds up the raw sums before its own
        launch_k(k_scan_down<Tin, Tout, true>, dim3(static_cast<unsigned>(nb)), dim3(kScanThreads),
            0, st, in, out, n, sums, total, cc);
        return last_launch_status();
    }
    // Scan the block sums in place (64-bit), recursively.
    s = scan_rec<long long, long long>(sums, sums, nb, nullptr, tmp + nb + 1, tmp_len - nb - 1, st,
                                       CapCheck{});
    if (s != GS_OK) return s;
    launch_k(k_scan_down<Tin, Tout, false>, dim3(static_cast<unsigned>(nb)), dim3(kScanThreads), 0,
        st, in, out, n, sums, total, cc);
    return last_launch_status();
}

gs_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, long long* total,
                             long long* tmp, int64_t tmp_len, cudaStream_t stream, CapCheck cc) {
    return scan_rec<int32_t, int32_t>(in, out, n, total, tmp, tmp_len, stream, cc);
}

// ============================================================================ preprocess

struct GridF {
    int n[3];
    float h[3];
    float o[3];
    float ih[3];  // 1 / h
    int b[3];
    int nb[3];
    FastDiv db[3];  // division by the brick size along each axis
};

// Error-free sum (Knuth): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Six blocks of 256 per SM (42 registers, a few values spilled to L1) measured faster than
// four (52 registers, no spills): the kernel is latency-bound on its division and square-root
// sequences, so the extra resident warps pay more than the spills cost.
__global__ void __launch_bounds__(256, 6) k_preprocess(const float* __restrict__ params, int64_t N, GridF G,
                                                    float trunc_sigma, int signal_mode, int a_act,
                                                    int t_act, float* __restrict__ rec,
                                                    int32_t* __restrict__ brange,
                                                    int32_t* __restrict__ gm_cnt,
                                                    int32_t* __restrict__ status,
                                                    int32_t* __restrict__ hist_zero,
                                                    int64_t hist_zero_len) {
    pdl_enter();
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g == 0) gm_cnt[N] = 0;  // sentinel: gm_off has N + 1 entries
    // the digit counts of the first two radix passes are accumulated by k_emit and the first
    // scatter: start them at zero
    for (int64_t i = g; i < hist_zero_len; i += int64_t(gridDim.x) * blockDim.x) hist_zero[i] = 0;
    if (g >= N) return;
    const float4* p4 = reinterpret_cast<const float4*>(params + g * 12);
    float4 a0 = p4[0], a1 = p4[1], a2 = p4[2];
    float p[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
    int32_t* br = brange + g * 8;
    float4* r4 = reinterpret_cast<float4*>(rec + g * REC_FLOATS);

    bool ok = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) ok = ok && isfinite(p[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) ok = ok && (fabsf(p[3 + k]) <= 30.0f);
    float nn = __fmul_rn(p[6], p[6]);
    nn = __fadd_rn(nn, __fmul_rn(p[7], p[7]));
    nn = __fadd_rn(nn, __fmul_rn(p[8], p[8]));
    nn = __fadd_rn(nn, __fmul_rn(p[9], p[9]));
    ok = ok && (nn > 0.0f);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!ok) {
#pragma unroll
        for (int k = 0; k < 8; ++k) br[k] = 0;
        gm_cnt[g] = 0;
#pragma unroll
        for (int k = 0; k < REC_F4; ++k) r4[k] = z4;
        atomicOr(status, GS_STATUS_NONFINITE);
        return;
    }

    // ---- binning specification (FP32, explicit rounding, fixed order) ----
    float s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = exp_cw(p[3 + k]);
    const float n = __fsqrt_rn(nn);
    const float w = __fdiv_rn(p[6], n), x = __fdiv_rn(p[7], n);
    const float y = __fdiv_rn(p[8], n), z = __fdiv_rn(p[9], n);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float R[3][3];
    R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
    const float ksig = __fmul_rn(trunc_sigma, 1.0001220703125f);
    int lo[3], hi[3];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float m0 = __fmul_rn(R[k][0], s[0]), m1 = __fmul_rn(R[k][1], s[1]);
        float m2 = __fmul_rn(R[k][2], s[2]);
        float sig = __fmul_rn(m0, m0);
        sig = __fadd_rn(sig, __fmul_rn(m1, m1));
        sig = __fadd_rn(sig, __fmul_rn(m2, m2));
        float e = __fmul_rn(ksig, __fsqrt_rn(sig));
        float lo_f = __fsub_rn(__fsub_rn(__fdiv_rn(__fsub_rn(__fsub_rn(p[k], e), G.o[k]), G.h[k]), 0.5f),
                               0.00390625f);
        float hi_f = __fadd_rn(__fsub_rn(__fdiv_rn(__fsub_rn(__fadd_rn(p[k], e), G.o[k]), G.h[k]), 0.5f),
                               0.00390625f);
        float nmax = static_cast<float>(G.n[k] - 1);
        if (!(hi_f >= 0.0f) || !(lo_f <= nmax)) {
            inside = false;
        } else {
            float lc = ceilf(lo_f), hc = floorf(hi_f);
            lc = fmaxf(lc, 0.0f);
            hc = fminf(hc, nmax);
            if (lc > hc) inside = false;
            lo[k] = static_cast<int>(lc);
            hi[k] = static_cast<int>(hc);
        }
    }
    int cnt = 0;
    if (inside) {
        int b0[3], b1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b0[k] = static_cast<int>(fast_div(static_cast<unsigned>(lo[k]), G.db[k]));
            b1[k] = static_cast<int>(fast_div(static_cast<unsigned>(hi[k]), G.db[k]));
            br[k] = b0[k];
            br[3 + k] = b1[k];
        }
        cnt = (b1[0] - b0[0] + 1) * (b1[1] - b0[1] + 1) * (b1[2] - b0[2] + 1);
        br[B_CNT] = cnt;
        br[B_VALID] = 1;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) br[k] = 0;
        br[B_VALID] = 1;
    }
    gm_cnt[g] = cnt;

    // ---- render record (accuracy only; contraction allowed) ----
    // M = sqrt(log2 e / 2) diag(1/s) R^T H: row k of M is R[:, k]^T H scaled by sqrt(k)/s_k.
    const float sk = 0.8493218002880191f;  // sqrt((1/2) log2 e)
    float Mx[3][3];                        // Mx[row][col]
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float f = sk / s[k];
#pragma unroll
        for (int j = 0; j < 3; ++j) Mx[k][j] = f * R[j][k] * G.h[j];
    }
    float col[3][3];  // col[j] = column j of M
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) col[j][k] = Mx[k][j];
    const float am0 = col[0][0] * col[0][0] + col[0][1] * col[0][1] + col[0][2] * col[0][2];
    const float inv_a = 1.0f / am0;
    float nrm[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        nrm[j] = sqrtf(col[j][0] * col[j][0] + col[j][1] * col[j][1] + col[j][2] * col[j][2]);
    // n1, n2: m1, m2 with their components along m0 removed
    // n1, n2: m1, m2 with their components along m0 removed; c_j = -(m_j . m0) / a
    float n1[3], n2[3];
    const float d1 = (col[1][0] * col[0][0] + col[1][1] * col[0][1] + col[1][2] * col[0][2]) * inv_a;
    const float d2 = (col[2][0] * col[0][0] + col[2][1] * col[0][1] + col[2][2] * col[0][2]) * inv_a;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        n1[k] = col[1][k] - d1 * col[0][k];
        n2[k] = col[2][k] - d2 * col[0][k];
    }
    const float Pyy = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
    const float Pzz = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
    const float P2yz = 2.0f * (n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
    // Mean in voxel-index space m = (mu - o) / h - 1/2 as a float head + tail, in double-float
    // arithmetic (Knuth's error-free two-sum; the quotient's remainder from one FMA), so that
    // m = mh + ml to about 2^-46 relative and d = (i - mh) - ml keeps one rounding at any
    // coordinate. (FP64 runs at 1/64 of the FP32 rate here.)
    float mh[3], ml[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float dh, dl;
        two_sum(p[k], -G.o[k], dh, dl);           // mu - o exactly
        const float qh = __fdiv_rn(dh, G.h[k]);   // correctly rounded: the remainder is exact
        const float rem = fmaf(-qh, G.h[k], dh);
        const float ql = __fmul_rn(__fadd_rn(rem, dl), G.ih[k]);
        float sh, sl;
        two_sum(qh, -0.5f, sh, sl);
        two_sum(sh, __fadd_rn(sl, ql), mh[k], ml[k]);
    }
    float A = a_act ? sigmoidf_(p[10]) : p[10];
    float T = t_act ? sigmoidf_(p[11]) : p[11];
    float v, r;
    if (signal_mode == 0) {
        v = A;
        r = T;
    } else {
        v = A * T;
        r = 1.0f;
    }
    r4[0] = make_float4(-mh[0], -ml[0], -mh[1], -mh[2]);
    r4[1] = make_float4(-ml[1], -ml[2], P2yz, -d2);
    r4[2] = make_float4(Pyy, -d1, Pzz, nrm[0]);
    // radius of a 4^3 footprint in whitened units: |M d|^2 <= sum_jk |m_j . m_k| (3/2)^2
    float gsum = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            gsum += fabsf(col[j][0] * col[k][0] + col[j][1] * col[k][1] + col[j][2] * col[k][2]);
    const float rho4 = 1.5f * sqrtf(gsum);
    // half-extents of the truncated ellipsoid's box in voxels, widened by 1 % and by a 4^3
    // footprint's half-width: a footprint whose centre is farther along an axis is missed
    float ext[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float sig = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) sig += (R[k][j] * s[j]) * (R[k][j] * s[j]);
        ext[k] = 1.01f * trunc_sigma * sqrtf(sig) * G.ih[k] + 1.5f + 1e-3f;
    }
    r4[3] = make_float4(ext[0], rho4, ext[1], ext[2]);
    // lower bound of q per squared voxel distance from the mean: (log2 e / 2) h_min^2 / s_max^2
    // bounds the smallest eigenvalue of the voxel-space form (less 1e-3 for rounding), so
    // a footprint whose voxel box lies farther than sqrt(Tcull / lam) from the mean is missed
    const float smax = fmaxf(s[0], fmaxf(s[1], s[2]));
    const float hmin = fminf(G.h[0], fminf(G.h[1], G.h[2]));
    const float lam = kHalfLog2e * (1.0f - 1e-3f) * (hmin / smax) * (hmin / smax);
    r4[4] = make_float4(v * r, r, v, lam);
}

// ============================================================================ capacity / emit

__global__ void k_capacity(const long long* __restrict__ total, int64_t capacity,
                           int64_t* __restrict__ npairs, int32_t* __restrict__ status) {
    pdl_enter();
    long long t = *total;
    *npairs = t;
    if (t > capacity) atomicOr(status, GS_STATUS_CAPACITY);
}

__device__ __forceinline__ int64_t valid_pairs(const int64_t* npairs, int64_t capacity) {
    int64_t P = *npairs;
    return (P > capacity || P < 0) ? 0 : P;
}

// One block per 256 consecutive Gaussians, whose pairs fill the contiguous Gaussian-major
// range [gm_off[g0], gm_off[g0 + 256]). When that range fits kEmitStage entries, each thread
// writes its pairs into shared memory and the block then stores the range with consecutive
// threads on consecutive addresses; otherwise threads write their pairs straight to global
// memory. Both paths write the same values. The block also adds its pairs to the first radix
// pass's digit counts (digit-major, hist[d * n_tiles + tile] over tiles of kSortTile
// Gaussian-major positions), so that pass needs no counting launch of its own: counted in
// shared memory when the range meets at most kEmitTiles tiles (then one global atomic per
// nonzero count), else one global atomic per pair.
constexpr int kEmitThreads = 256;
constexpr int kEmitStage = 4096;
constexpr int kEmitTiles = 4;

__global__ void __launch_bounds__(kEmitThreads) k_emit(const int32_t* __restrict__ brange,
                                                       const int32_t* __restrict__ gm_off, int64_t N,
                                                       int nbx, int nby,
                                                       const int64_t* __restrict__ npairs,
                                                       int64_t capacity, int32_t* __restrict__ keys,
                                                       int32_t* __restrict__ gm_gid,
                                                       int32_t* __restrict__ hist, int n_tiles) {
    pdl_enter();
    __shared__ int32_t skey[kEmitStage];
    __shared__ int32_t sgid[kEmitStage];
    __shared__ int32_t hcnt[kEmitTiles * kRadix];
    if (valid_pairs(npairs, capacity) == 0) return;
    const int64_t g0 = int64_t(blockIdx.x) * kEmitThreads;
    const int64_t g = g0 + threadIdx.x;
    const int64_t gl = min(g0 + kEmitThreads, N);
    const int base = gm_off[g0];
    const int total = gm_off[gl] - base;
    const bool staged = total <= kEmitStage;
    const int t0 = base / kSortTile;
    const bool local = total == 0 || (base + total - 1) / kSortTile - t0 < kEmitTiles;  // uniform
    for (int i = threadIdx.x; i < kEmitTiles * kRadix; i += kEmitThreads) hcnt[i] = 0;
    __syncthreads();
    int32_t* kdst = staged ? skey : keys + base;
    int32_t* gdst = staged ? sgid : gm_gid + base;
    if (g < N) {
        const int32_t* br = brange + g * 8;
        if (br[B_CNT] != 0) {
            int j = gm_off[g] - base;
            for (int bz = br[B_LOZ]; bz <= br[B_HIZ]; ++bz)
                for (int by = br[B_LOY]; by <= br[B_HIY]; ++by)
                    for (int bx = br[B_LOX]; bx <= br[B_HIX]; ++bx) {
                        const int key = (bz * nby + by) * nbx + bx;
                        kdst[j] = key;
                        gdst[j] = static_cast<int32_t>(g);
                        if (!staged) {  // (staged ranges are counted as they are stored)
                            const int t = (base + j) / kSortTile;
                            if (local)
                                atomicAdd(&hcnt[(t - t0) * kRadix + (key & (kRadix - 1))], 1);
                            else
                                atomicAdd(&hist[int64_t(key & (kRadix - 1)) * n_tiles + t], 1);
                        }
                        ++j;
                    }
        }
    }
    __syncthreads();
    if (staged) {
        for (int i = threadIdx.x; i < total; i += kEmitThreads) {
            const int key = skey[i];
            keys[base + i] = key;
            gm_gid[base + i] = sgid[i];
            atomicAdd(&hcnt[((base + i) / kSortTile - t0) * kRadix + (key & (kRadix - 1))], 1);
        }
        __syncthreads();
    }
    if (local) {
        for (int i = threadIdx.x; i < kEmitTiles * kRadix; i += kEmitThreads) {
            const int c = hcnt[i];
            if (c != 0) atomicAdd(&hist[int64_t(i % kRadix) * n_tiles + t0 + i / kRadix], c);
        }
    }
}

// ============================================================================ radix sort

// Stable scatter of one tile of kSortTile keys. Warp w owns the contiguous sub-tile
// [w * 256, (w + 1) * 256) and visits it in 8 rounds of 32 consecutive keys (kept in
// registers; with the digit counts accumulated by the launch before, 2,048-key tiles measured
// faster than 1,024, 1,536, 2,560 and 3,072 at the fitting size). Pass 1 counts each warp's
// digits. A block-wide prefix then gives, per digit,
// the tile-local start of its run and each warp's start inside it. Pass 2 places every key in
// shared memory at its warp's start + its rank among equal digits in lower lanes (warp match
// masks), so the tile sits in shared memory sorted by digit, ties in tile order. The tile is
// then written out in that order: digit d's run goes to [hist_off[d][tile], ...), so
// consecutive threads store consecutive addresses.
// kLast: the last pass stores the bins' per-pair arrays directly: brick (the key),
// Gaussian-major position (the value) and owner (gm_gid of the value). Every other pass adds
// each key to the next pass's digit counts at its output position's tile (one atomic per
// group of equal (tile, digit) in a warp), so no pass after the first needs a counting launch.
template <bool kFirst, bool kLast>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
    int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out,
    const int32_t* __restrict__ hist_off, const int64_t* __restrict__ npairs, int64_t capacity,
    int shift, int n_tiles, const int32_t* __restrict__ gm_gid, int32_t* __restrict__ pair_gid,
    int32_t* __restrict__ hist_next) {
    pdl_enter();
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kPerWarp = kSortTile / kWarps;
    constexpr int kRounds = kPerWarp / 32;
    static_assert(kSortThreads == kRadix, "one thread per digit in the block-wide prefix");
    __shared__ int wcnt[kWarps][kRadix];
    __shared__ int dstart[kRadix];   // tile-local start of each digit's run
    __shared__ int gstart[kRadix];   // global start of each digit's run for this tile
    __shared__ int wsum[kWarps];
    __shared__ int skey[kSortTile];
    __shared__ int sval[kSortTile];
    const int64_t P = valid_pairs(npairs, capacity);
    const int64_t tile0 = int64_t(blockIdx.x) * kSortTile;
    if (tile0 >= P) return;  // past the last pair: nothing to place
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d < kRadix; d += kSortThreads)
        for (int w = 0; w < kWarps; ++w) wcnt[w][d] = 0;
    __syncthreads();
    const int64_t sub0 = tile0 + int64_t(warp) * kPerWarp;
    const unsigned lt_mask = (1u << lane) - 1u;
    int kr[kRounds], vr[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = sub0 + r * 32 + lane;
        const bool valid = idx < P;
        kr[r] = valid ? keys_in[idx] : 0;
        vr[r] = valid ? (kFirst ? static_cast<int>(idx) : vals_in[idx]) : 0;
        const int d = (kr[r] >> shift) & (kRadix - 1);
        const unsigned tag = valid ? static_cast<unsigned>(d) : static_cast<unsigned>(kRadix + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: warps' starts inside digit d's run, and the run's length
    const int d = tid;
    int run = 0;
    for (int w = 0; w < kWarps; ++w) {
        const int c = wcnt[w][d];
        wcnt[w][d] = run;
        run += c;
    }
    // exclusive prefix of the run lengths over digits (block scan, digit order)
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const int start = before + incl - run;
    dstart[d] = start;
    gstart[d] = hist_off[int64_t(d) * n_tiles + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) wcnt[w][d] += start;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = sub0 + r * 32 + lane;
        const bool valid = idx < P;
        const int dk = (kr[r] >> shift) & (kRadix - 1);
        const unsigned tag = valid ? static_cast<unsigned>(dk) : static_cast<unsigned>(kRadix + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        if (valid) {
            const int lp = wcnt[warp][dk] + __popc(peers & lt_mask);
            skey[lp] = kr[r];
            sval[lp] = vr[r];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][dk] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    const int n_here = static_cast<int>(min(int64_t(kSortTile), P - tile0));
    for (int j = tid; j < n_here; j += kSortThreads) {
        const int key = skey[j];
        const int dk = (key >> shift) & (kRadix - 1);
        const int pos = gstart[dk] + (j - dstart[dk]);
        keys_out[pos] = key;
        vals_out[pos] = sval[j];
        if (kLast) {
            pair_gid[pos] = gm_gid[sval[j]];
        } else {
            const int tag = ((pos / kSortTile) << kRadixBits) | ((key >> (shift + kRadixBits)) & (kRadix - 1));
            const unsigned peers = __match_any_sync(__activemask(), tag);
            if (lane == __ffs(peers) - 1)
                atomicAdd(&hist_next[int64_t(tag & (kRadix - 1)) * n_tiles + (tag >> kRadixBits)],
                          __popc(peers));
        }
    }
}

// brick_off from the boundaries of the sorted keys (brick_off[b] = first pair of brick b, or
// the next non-empty brick's first pair; brick_off[nb] = P).
__global__ void __launch_bounds__(256) k_brick_off(const int32_t* __restrict__ keys,
                                                   const int64_t* __restrict__ npairs,
                                                   int64_t capacity, int nb,
                                                   int32_t* __restrict__ brick_off) {
    pdl_enter();
    const int64_t P = valid_pairs(npairs, capacity);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= P;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int cur = (i < P) ? keys[i] : nb;
        const int prev = (i > 0) ? keys[i - 1] : -1;
        for (int bb = prev + 1; bb <= cur; ++bb) brick_off[bb] = static_cast<int32_t>(i);
    }
}

}  // namespace gs

// ============================================================================ C ABI

using namespace gs;

namespace {

struct BinsLayout {
    size_t off_brick_off, off_pair_gid, off_pair_gmj, off_pair_brick, off_gm_off, off_rec, off_brange,
        off_npairs,
        off_status, bytes;
};

bool bins_layout(int64_t n_gauss, int64_t capacity, int32_t n_bricks, BinsLayout* L) {
    if (n_gauss < 0 || capacity < 0 || capacity > kMaxCapacity || n_bricks <= 0) return false;
    if (n_gauss > (int64_t(1) << 31) - 2) return false;
    const int64_t cap = capacity > 0 ? capacity : 1;
    const int64_t n = n_gauss > 0 ? n_gauss : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L->off_brick_off = take(sizeof(int32_t) * (int64_t(n_bricks) + 1));
    L->off_pair_gid = take(sizeof(int32_t) * cap);
    L->off_pair_gmj = take(sizeof(int32_t) * cap);
    L->off_pair_brick = take(sizeof(int32_t) * cap);
    L->off_gm_off = take(sizeof(int32_t) * (n + 1));
    L->off_rec = take(sizeof(float) * REC_FLOATS * n);
    L->off_brange = take(sizeof(int32_t) * 8 * n);
    L->off_npairs = take(sizeof(int64_t));
    L->off_status = take(sizeof(int32_t));
    L->bytes = off;
    return true;
}

int32_t n_bricks_of(const gs_grid* g, const gs_config* c) {
    BrickGeom b = brick_geom(g, c);
    return b.nbx * b.nby * b.nbz;
}

int64_t n_voxels_of(const gs_grid* g) { return int64_t(g->nx) * g->ny * g->nz; }

}  // namespace

extern "C" size_t gs_bins_bytes(int64_t n_gauss, int64_t capacity, const gs_grid* grid,
                                const gs_config* cfg) {
    if (validate_grid_cfg(grid, cfg) != GS_OK) return 0;
    BinsLayout L;
    if (!bins_layout(n_gauss, capacity, n_bricks_of(grid, cfg), &L)) return 0;
    return L.bytes;
}

extern "C" gs_status gs_bins_bind(void* arena, size_t arena_bytes, int64_t n_gauss,
                                  int64_t capacity, const gs_grid* grid, const gs_config* cfg,
                                  gs_bins* out) {
    if (!arena || !out) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return GS_ERR_INVALID_ARG;
    gs_status s = validate_grid_cfg(grid, cfg);
    if (s != GS_OK) return s;
    BinsLayout L;
    const int32_t nb = n_bricks_of(grid, cfg);
    if (!bins_layout(n_gauss, capacity, nb, &L)) return GS_ERR_INVALID_ARG;
    if (arena_bytes < L.bytes) return GS_ERR_WORKSPACE;
    char* a = static_cast<char*>(arena);
    BrickGeom b = brick_geom(grid, cfg);
    out->n_gauss = n_gauss;
    out->capacity = capacity;
    out->n_bricks = nb;
    out->nbx = b.nbx;
    out->nby = b.nby;
    out->nbz = b.nbz;
    out->brick_off = reinterpret_cast<int32_t*>(a + L.off_brick_off);
    out->pair_gid = reinterpret_cast<int32_t*>(a + L.off_pair_gid);
    out->pair_gmj = reinterpret_cast<int32_t*>(a + L.off_pair_gmj);
    out->pair_brick = reinterpret_cast<int32_t*>(a + L.off_pair_brick);
    out->gm_off = reinterpret_cast<int32_t*>(a + L.off_gm_off);
    out->rec = reinterpret_cast<float*>(a + L.off_rec);
    out->brange = reinterpret_cast<int32_t*>(a + L.off_brange);
    out->d_npairs = reinterpret_cast<int64_t*>(a + L.off_npairs);
    out->d_status = reinterpret_cast<int32_t*>(a + L.off_status);
    return GS_OK;
}

extern "C" size_t gs_workspace_bytes(int64_t n_gauss, int64_t capacity, const gs_grid* grid,
                                     const gs_config* cfg) {
    if (validate_grid_cfg(grid, cfg) != GS_OK) return 0;
    if (n_gauss < 0 || capacity < 0 || capacity > kMaxCapacity) return 0;
    Workspace ws;
    carve_workspace(nullptr, n_gauss, capacity, n_bricks_of(grid, cfg), n_voxels_of(grid),
                    cfg->deterministic != 0, &ws);
    return ws.bytes;
}

namespace gs {
// Shared by the other translation units: bind the workspace for a problem size.
gs_status bind_workspace(void* base, size_t bytes, int64_t n_gauss, int64_t capacity,
                         const gs_grid* grid, const gs_config* cfg, Workspace* ws) {
    if (!base) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(base) % 256 != 0) return GS_ERR_INVALID_ARG;
    carve_workspace(nullptr, n_gauss, capacity, n_bricks_of(grid, cfg), n_voxels_of(grid),
                    cfg->deterministic != 0, ws);
    if (bytes < ws->bytes) return GS_ERR_WORKSPACE;
    carve_workspace(base, n_gauss, capacity, n_bricks_of(grid, cfg), n_voxels_of(grid),
                    cfg->deterministic != 0, ws);
    return GS_OK;
}

bool bins_match(const gs_bins* b, const gs_grid* grid, const gs_config* cfg) {
    if (!b || !b->brick_off || !b->pair_gid || !b->pair_gmj || !b->pair_brick || !b->gm_off || !b->rec ||
        !b->brange || !b->d_npairs || !b->d_status)
        return false;
    BrickGeom g = brick_geom(grid, cfg);
    return b->nbx == g.nbx && b->nby == g.nby && b->nbz == g.nbz &&
           b->n_bricks == g.nbx * g.nby * g.nbz && b->capacity >= 0 &&
           b->capacity <= kMaxCapacity && b->n_gauss >= 0;
}

static int radix_passes(int32_t n_bricks) {
    int bits = 0;
    while ((int64_t(1) << bits) < n_bricks) ++bits;
    int passes = (bits + kRadixBits - 1) / kRadixBits;
    return passes < 1 ? 1 : passes;
}

gs_status bin_bricks_impl(const float* params, const gs_grid* grid, const gs_config* cfg,
                          gs_bins* bins, const Workspace& ws, cudaStream_t st) {
    const int64_t N = bins->n_gauss;
    const int64_t cap = bins->capacity;
    BrickGeom b = brick_geom(grid, cfg);
    GridF G;
    G.n[0] = grid->nx; G.n[1] = grid->ny; G.n[2] = grid->nz;
    for (int k = 0; k < 3; ++k) {
        G.h[k] = grid->h[k];
        G.o[k] = grid->origin[k];
        G.ih[k] = 1.0f / grid->h[k];
    }
    G.b[0] = b.bx; G.b[1] = b.by; G.b[2] = b.bz;
    G.nb[0] = b.nbx; G.nb[1] = b.nby; G.nb[2] = b.nbz;
    for (int k = 0; k < 3; ++k) G.db[k] = make_fastdiv(static_cast<unsigned>(G.b[k]));

    if (cudaMemsetAsync(bins->d_status, 0, sizeof(int32_t), st) != cudaSuccess) return GS_ERR_CUDA;
    long long* total = ws.scan_tmp + ws.scan_tmp_len - 1;
    if (N > 0) {
        const unsigned gb = static_cast<unsigned>((N + 255) / 256);
        launch_k(k_preprocess, dim3(gb), dim3(256), 0, st, params, N, G, cfg->trunc_sigma,
            cfg->signal_mode, cfg->a_act, cfg->t_act, bins->rec, bins->brange, ws.gm_cnt,
            bins->d_status, ws.hist, 2 * (int64_t(kRadix) * ws.n_tiles + 1));
        gs_status s = last_launch_status();
        if (s != GS_OK) return s;
        // gm_off = exclusive scan of counts (N + 1 entries; gm_cnt[N] = 0 sentinel); the scan's
        // last thread also stores the total as d_npairs and flags an overflow of the capacity.
        const CapCheck cc{cap, bins->d_npairs, bins->d_status};
        s = exclusive_scan_i32(ws.gm_cnt, bins->gm_off, N + 1, total, ws.scan_tmp,
                               ws.scan_tmp_len - 1, st, cc);
        if (s != GS_OK) return s;
    } else {
        if (cudaMemsetAsync(total, 0, sizeof(long long), st) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaMemsetAsync(bins->gm_off, 0, sizeof(int32_t), st) != cudaSuccess) return GS_ERR_CUDA;
        launch_k(k_capacity, dim3(1), dim3(1), 0, st, total, cap, bins->d_npairs, bins->d_status);
        const gs_status s = last_launch_status();
        if (s != GS_OK) return s;
    }
    gs_status s = GS_OK;
    if (N > 0) {
        launch_k(k_emit, dim3(static_cast<unsigned>((N + kEmitThreads - 1) / kEmitThreads)),
            dim3(kEmitThreads), 0, st, bins->brange, bins->gm_off, N, b.nbx, b.nby, bins->d_npairs,
            cap, ws.keys0, ws.gm_gid, ws.hist, ws.n_tiles);
        s = last_launch_status();
        if (s != GS_OK) return s;
    }
    if (cap == 0) {
        if (cudaMemsetAsync(bins->brick_off, 0, sizeof(int32_t) * (int64_t(bins->n_bricks) + 1), st) !=
            cudaSuccess)
            return GS_ERR_CUDA;
        return GS_OK;
    }

    // Stable LSD radix sort of brick keys; values are Gaussian-major positions.
    const int passes = radix_passes(bins->n_bricks);
    int32_t* kin = ws.keys0;
    int32_t* vin = ws.vals0;
    int32_t* kout = ws.keys1;
    int32_t* vout = ws.vals1;
    const int nt = ws.n_tiles;
    const int64_t hist_len = int64_t(kRadix) * nt;
    // digit counts: pass 0's from k_emit, pass p + 1's from pass p's scatter, in two buffers
    // that k_preprocess zeroed; a third pass reuses the first buffer, zeroed again here
    int32_t* hbuf[2] = {ws.hist, ws.hist1};
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        int32_t* hcur = hbuf[pass & 1];
        int32_t* hnext = hbuf[(pass + 1) & 1];
        if (pass >= 1 && pass + 1 < passes &&
            cudaMemsetAsync(hnext, 0, sizeof(int32_t) * hist_len, st) != cudaSuccess)
            return GS_ERR_CUDA;
        s = exclusive_scan_i32(hcur, hcur, hist_len, nullptr, ws.scan_tmp, ws.scan_tmp_len - 1, st);
        if (s != GS_OK) return s;
        // the last pass writes the bins' pair arrays (brick, Gaussian-major position, owner)
        const bool last = pass == passes - 1;
        int32_t* ko = last ? bins->pair_brick : kout;
        int32_t* vo = last ? bins->pair_gmj : vout;
        using ScatterFn = void (*)(const int32_t*, const int32_t*, int32_t*, int32_t*, const int32_t*,
                                   const int64_t*, int64_t, int, int, const int32_t*, int32_t*,
                                   int32_t*);
        ScatterFn kern = pass == 0 ? (last ? k_radix_scatter<true, true> : k_radix_scatter<true, false>)
                                   : (last ? k_radix_scatter<false, true> : k_radix_scatter<false, false>);
        launch_k(kern, dim3(nt), dim3(kSortThreads), 0, st, kin, vin, ko, vo, hcur,
            bins->d_npairs, cap, shift, nt, ws.gm_gid, bins->pair_gid, hnext);
        s = last_launch_status();
        if (s != GS_OK) return s;
        int32_t* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    launch_k(k_brick_off, dim3(1184), dim3(256), 0, st, bins->pair_brick, bins->d_npairs, cap,
        bins->n_bricks, bins->brick_off);
    return last_launch_status();
}

}  // namespace gs

extern "C" gs_status gs_bin_bricks(const float* params, const gs_grid* grid, const gs_config* cfg,
                                   gs_bins* bins, void* ws, size_t ws_bytes, gs_stream stream) {
    gs_status s = validate_grid_cfg(grid, cfg);
    if (s != GS_OK) return s;
    if (!bins_match(bins, grid, cfg)) return GS_ERR_INVALID_ARG;
    if (bins->n_gauss > 0 && !params) return GS_ERR_INVALID_ARG;
    if (params && reinterpret_cast<uintptr_t>(params) % 16 != 0) return GS_ERR_INVALID_ARG;
    Workspace w;
    s = bind_workspace(ws, ws_bytes, bins->n_gauss, bins->capacity, grid, cfg, &w);
    if (s != GS_OK) return s;
    return bin_bricks_impl(params, grid, cfg, bins, w, reinterpret_cast<cudaStream_t>(stream));
}
