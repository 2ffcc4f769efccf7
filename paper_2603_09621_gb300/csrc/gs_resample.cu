// gs_resample.cu -- trilinear resize with half-pixel centres (Sec. 4.1 makes the LR inputs
// by trilinear downsampling), its adjoint as a deterministic gather, and the adjoint fused
// with the adjoint render's per-voxel factors for the fitting step.
//
// Along one axis, destination sample j sits at the source continuous index
// c_j = (n_src / n_dst)(j + 1/2) - 1/2 (raised to 0 where negative) and reads source samples
// i0 = floor(c_j), i1 = min(i0 + 1, n_src - 1) with weights 1 - w, w = c_j - i0. c_j is
// formed with one rounding per FP32 operation (no contraction), so every kernel, and the
// oracle, take the same integer decisions.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"

namespace gs {

struct ResAxis {
    float scale;  // n_src / n_dst, FP32 division
    float inv;    // n_dst / n_src (only bounds the adjoint's search range)
    int n_src, n_dst;
};

struct ResGeo {
    ResAxis a[3];  // x, y, z
};

__device__ __forceinline__ void res_map(const ResAxis& A, int j, int& i0, int& i1, float& w) {
    float c = __fsub_rn(__fmul_rn(A.scale, __fadd_rn(float(j), 0.5f)), 0.5f);
    c = fmaxf(c, 0.0f);
    const float f = floorf(c);
    i0 = static_cast<int>(f);
    i1 = min(i0 + 1, A.n_src - 1);
    w = __fsub_rn(c, f);  // exact: 0 <= c - f < 1
}

// Weight with which destination sample j reads source sample i (both corners may coincide
// at the upper edge).
__device__ __forceinline__ float res_weight(const ResAxis& A, int j, int i) {
    int i0, i1;
    float w;
    res_map(A, j, i0, i1, w);
    return (i0 == i ? 1.0f - w : 0.0f) + (i1 == i ? w : 0.0f);
}

// Destination samples that may read source sample i: c_j in [i - 1, i + 1), widened by one.
__device__ __forceinline__ void res_range(const ResAxis& A, int i, int& jlo, int& jhi) {
    jlo = max(0, static_cast<int>(floorf((float(i) - 0.5f) * A.inv - 0.5f)) - 1);
    jhi = min(A.n_dst - 1, static_cast<int>(ceilf((float(i) + 1.5f) * A.inv - 0.5f)) + 1);
}

__global__ void __launch_bounds__(256) k_resample_fwd(const float* __restrict__ src, ResGeo G,
                                                      float* __restrict__ dst) {
    pdl_enter();
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    const int64_t n = int64_t(AX.n_dst) * AY.n_dst * AZ.n_dst;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t % AX.n_dst);
        const int y = static_cast<int>((t / AX.n_dst) % AY.n_dst);
        const int z = static_cast<int>(t / (int64_t(AX.n_dst) * AY.n_dst));
        int x0, x1, y0, y1, z0, z1;
        float wx, wy, wz;
        res_map(AX, x, x0, x1, wx);
        res_map(AY, y, y0, y1, wy);
        res_map(AZ, z, z0, z1, wz);
        const int64_t sx = AX.n_src, sxy = int64_t(AX.n_src) * AY.n_src;
        const float* p00 = src + z0 * sxy + y0 * sx;
        const float* p01 = src + z0 * sxy + y1 * sx;
        const float* p10 = src + z1 * sxy + y0 * sx;
        const float* p11 = src + z1 * sxy + y1 * sx;
        const float ux = 1.0f - wx, uy = 1.0f - wy, uz = 1.0f - wz;
        const float r00 = fmaf(wx, p00[x1], ux * p00[x0]);
        const float r01 = fmaf(wx, p01[x1], ux * p01[x0]);
        const float r10 = fmaf(wx, p10[x1], ux * p10[x0]);
        const float r11 = fmaf(wx, p11[x1], ux * p11[x0]);
        const float s0 = fmaf(wy, r01, uy * r00);
        const float s1 = fmaf(wy, r11, uy * r10);
        dst[t] = fmaf(wz, s1, uz * s0);
    }
}

// The destination samples that read source sample i form one run j0, j0 + 1, ... (i0(j) is
// non-decreasing in j). K slots cover it under the bounds of res_list_ok / res_two_taps.
// Slot k holds the weight of j0 + k (0 past the run); *n is the run length.
constexpr int kResList = 4;
template <int K = kResList>
__device__ __forceinline__ void res_list(const ResAxis& A, int i, int& j0, int& n, float (&w)[K]) {
    int lo, hi;
    res_range(A, i, lo, hi);
    int t = lo;
    for (; t < hi; ++t) {  // skip samples whose upper corner is still below i
        int a, b;
        float ww;
        res_map(A, t, a, b, ww);
        if (b >= i) break;
    }
    j0 = t;
    n = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = t + k;
        w[k] = (j < A.n_dst) ? res_weight(A, j, i) : 0.0f;
        n = (w[k] != 0.0f) ? k + 1 : n;
    }
}

// Run lengths with FP32 positions: c_j is within c 2^-23 of its exact value, so for source
// sizes up to 2^16 consecutive positions are spaced by the scale +- 2^-6.
//   kResList slots: scale >= 2/3 on every axis keeps the spacing above 0.65, so at most
//   four positions fall in one window [i - 1, i + 1).
//   2 slots: an exact copy (scale 1: c_j = j) or scale >= 1.05 (spacing above 1.03).
constexpr int kResMaxSrc = 1 << 16;
static bool res_list_ok(const ResGeo& G) {
    for (int a = 0; a < 3; ++a)
        if (!(G.a[a].inv <= 1.5f) || G.a[a].n_src > kResMaxSrc) return false;
    return true;
}

static bool res_two_taps(const ResGeo& G) {
    for (int a = 0; a < 3; ++a) {
        const ResAxis& A = G.a[a];
        if (A.n_src > kResMaxSrc) return false;
        if (A.n_dst != A.n_src && !(A.scale >= 1.05f)) return false;
    }
    return true;
}

// Adjoint value at source voxel (x, y, z): sum over the destination samples that read it, in
// ascending (z, y, x) order (any ratio).
__device__ __forceinline__ float res_gather(const float* __restrict__ ddst, const ResGeo& G, int x,
                                            int y, int z) {
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    int xlo, xhi, ylo, yhi, zlo, zhi;
    res_range(AX, x, xlo, xhi);
    res_range(AY, y, ylo, yhi);
    res_range(AZ, z, zlo, zhi);
    float acc = 0.0f;
    for (int jz = zlo; jz <= zhi; ++jz) {
        const float wz = res_weight(AZ, jz, z);
        if (wz == 0.0f) continue;
        for (int jy = ylo; jy <= yhi; ++jy) {
            const float wy = res_weight(AY, jy, y);
            if (wy == 0.0f) continue;
            const float wzy = wz * wy;
            const float* row = ddst + (int64_t(jz) * AY.n_dst + jy) * AX.n_dst;
            for (int jx = xlo; jx <= xhi; ++jx) {
                const float wx = res_weight(AX, jx, x);
                if (wx != 0.0f) acc = fmaf(wzy * wx, row[jx], acc);
            }
        }
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_resample_bwd(const float* __restrict__ ddst, ResGeo G,
                                                      float* __restrict__ dsrc) {
    pdl_enter();
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    const int64_t n = int64_t(AX.n_src) * AY.n_src * AZ.n_src;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t % AX.n_src);
        const int y = static_cast<int>((t / AX.n_src) % AY.n_src);
        const int z = static_cast<int>(t / (int64_t(AX.n_src) * AY.n_src));
        dsrc[t] = res_gather(ddst, G, x, y, z);
    }
}

// Table form of the adjoint gather (under res_list_ok / res_two_taps, with at most
// kResTabMax source samples over the three axes): each block tabulates the runs of every
// source x, y and z in shared memory once, then sweeps source rows (z, y) with one thread
// per voxel; a voxel reads its three runs from the tables and gathers in ascending (z, y, x)
// order.
constexpr int kResTabMax = 2048;

template <int K>
struct ResRun {
    int j0, n;
    float w[K];
};

template <bool kPrep, int K>
__global__ void __launch_bounds__(256) k_resample_adj_tab(const float* __restrict__ ddst, ResGeo G,
                                                          const float* __restrict__ Iv,
                                                          const float* __restrict__ Wv, float eps,
                                                          float* __restrict__ dsrc,
                                                          float2* __restrict__ aip) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char res_smem[];
    ResRun<K>* tab = reinterpret_cast<ResRun<K>*>(res_smem);
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    const int nx = AX.n_src, ny = AY.n_src, nz = AZ.n_src;
    ResRun<K>* xt = tab;
    ResRun<K>* yt = tab + nx;
    ResRun<K>* zt = tab + nx + ny;
    for (int e = threadIdx.x; e < nx + ny + nz; e += blockDim.x) {
        const int ax = e < nx ? 0 : (e < nx + ny ? 1 : 2);
        const int i = e - (ax > 0 ? nx : 0) - (ax > 1 ? ny : 0);
        ResAxis A;
        A.scale = ax == 0 ? AX.scale : (ax == 1 ? AY.scale : AZ.scale);
        A.inv = ax == 0 ? AX.inv : (ax == 1 ? AY.inv : AZ.inv);
        A.n_src = ax == 0 ? AX.n_src : (ax == 1 ? AY.n_src : AZ.n_src);
        A.n_dst = ax == 0 ? AX.n_dst : (ax == 1 ? AY.n_dst : AZ.n_dst);
        ResRun<K> rr;
        res_list<K>(A, i, rr.j0, rr.n, rr.w);
        tab[e] = rr;
    }
    __syncthreads();
    const int64_t rows = int64_t(nz) * ny;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int z = static_cast<int>(row / ny), y = static_cast<int>(row - int64_t(z) * ny);
        const ResRun<K> rz = zt[z], ry = yt[y];
        const int64_t row0 = row * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const ResRun<K> rx = xt[x];
            float acc = 0.0f;
#pragma unroll
            for (int a = 0; a < K; ++a) {
                if (a >= rz.n) break;
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    if (b >= ry.n) break;
                    const float wzy = rz.w[a] * ry.w[b];
                    const float* src =
                        ddst + (int64_t(rz.j0 + a) * AY.n_dst + (ry.j0 + b)) * AX.n_dst + rx.j0;
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        if (c >= rx.n) break;
                        if (rx.w[c] != 0.0f) acc = fmaf(wzy * rx.w[c], src[c], acc);
                    }
                }
            }
            if (kPrep) {
                const float w = Wv[row0 + x];
                const float al = acc / (w > eps ? w : eps);
                aip[row0 + x] = make_float2(al, (w > eps) ? al * Iv[row0 + x] : 0.0f);
            } else {
                dsrc[row0 + x] = acc;
            }
        }
    }
}

// Fitting step, any ratio: dL/dI at each HR voxel is the resize adjoint of dL/dLR; stored
// directly as the adjoint render's factors (alpha, alpha I'), alpha = dL/dI / max(W, eps),
// I' = I where W > eps, else 0.
__global__ void __launch_bounds__(256) k_resample_adj_prep(const float* __restrict__ dlr, ResGeo G,
                                                           const float* __restrict__ Iv,
                                                           const float* __restrict__ Wv, float eps,
                                                           float2* __restrict__ aip) {
    pdl_enter();
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    const int64_t n = int64_t(AX.n_src) * AY.n_src * AZ.n_src;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t % AX.n_src);
        const int y = static_cast<int>((t / AX.n_src) % AY.n_src);
        const int z = static_cast<int>(t / (int64_t(AX.n_src) * AY.n_src));
        const float gI = res_gather(dlr, G, x, y, z);
        const float w = Wv[t];
        const float al = gI / (w > eps ? w : eps);
        aip[t] = make_float2(al, (w > eps) ? al * Iv[t] : 0.0f);
    }
}

static bool dims_ok(int32_t nz, int32_t ny, int32_t nx) {
    return nz > 0 && ny > 0 && nx > 0 && nx < (1 << 23) && ny < (1 << 23) && nz < (1 << 23);
}

static ResGeo make_res(int32_t snz, int32_t sny, int32_t snx, int32_t dnz, int32_t dny, int32_t dnx) {
    ResGeo G;
    const int32_t s[3] = {snx, sny, snz}, d[3] = {dnx, dny, dnz};
    for (int a = 0; a < 3; ++a) {
        G.a[a].n_src = s[a];
        G.a[a].n_dst = d[a];
        G.a[a].scale = float(s[a]) / float(d[a]);
        G.a[a].inv = float(d[a]) / float(s[a]);
    }
    return G;
}

static unsigned res_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return static_cast<unsigned>(b < 152 * 64 ? b : 152 * 64);
}

gs_status resample_fwd_impl(const float* src, int32_t snz, int32_t sny, int32_t snx, float* dst,
                            int32_t dnz, int32_t dny, int32_t dnx, cudaStream_t st) {
    const ResGeo G = make_res(snz, sny, snx, dnz, dny, dnx);
    launch_k(k_resample_fwd, dim3(res_blocks(int64_t(dnz) * dny * dnx)), dim3(256), 0, st, src, G,
        dst);
    return last_launch_status();
}

// Separable form of the adjoint for one source plane z and a tile of kPlaneRows source rows:
// first U[y][jx] = sum over the z and y runs of w_z w_y dL/dLR[jz][jy][jx] for every LR column
// jx (shared memory), then each voxel sums its x run over U[y]. Fixed order: z, then y
// (inside U), then x.
template <bool kPrep, int K, int kPlaneRows>
__global__ void __launch_bounds__(256) k_resample_adj_plane(const float* __restrict__ ddst, ResGeo G,
                                                            const float* __restrict__ Iv,
                                                            const float* __restrict__ Wv, float eps,
                                                            float* __restrict__ dsrc,
                                                            float2* __restrict__ aip) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char res_smem[];
    const ResAxis &AX = G.a[0], &AY = G.a[1], &AZ = G.a[2];
    const int nx = AX.n_src, ny = AY.n_src;
    const int lnx = AX.n_dst, lny = AY.n_dst;
    ResRun<K>* xt = reinterpret_cast<ResRun<K>*>(res_smem);
    ResRun<K>* yt = xt + nx;                                // kPlaneRows entries
    float* U = reinterpret_cast<float*>(yt + kPlaneRows);  // [kPlaneRows][lnx]
    __shared__ ResRun<K> zr;
    const int z = blockIdx.x;
    const int y0 = blockIdx.y * kPlaneRows;
    const int rows = min(kPlaneRows, ny - y0);
    for (int e = threadIdx.x; e < nx + rows + 1; e += blockDim.x) {
        ResRun<K> rr;
        if (e < nx) {
            res_list<K>(AX, e, rr.j0, rr.n, rr.w);
            xt[e] = rr;
        } else if (e < nx + rows) {
            res_list<K>(AY, y0 + (e - nx), rr.j0, rr.n, rr.w);
            yt[e - nx] = rr;
        } else {
            res_list<K>(AZ, z, rr.j0, rr.n, rr.w);
            zr = rr;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * lnx; e += blockDim.x) {
        const int r = e / lnx, jx = e - r * lnx;
        const ResRun<K>& ry = yt[r];
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            if (a >= zr.n) break;
#pragma unroll
            for (int b = 0; b < K; ++b) {
                if (b >= ry.n) break;
                acc = fmaf(zr.w[a] * ry.w[b], ddst[(int64_t(zr.j0 + a) * lny + (ry.j0 + b)) * lnx + jx], acc);
            }
        }
        U[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * nx; e += blockDim.x) {
        const int r = e / nx, x = e - r * nx;
        const ResRun<K>& rx = xt[x];
        const float* u = U + r * lnx + rx.j0;
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (c >= rx.n) break;
            acc = fmaf(rx.w[c], u[c], acc);
        }
        const int64_t v = (int64_t(z) * ny + (y0 + r)) * nx + x;
        if (kPrep) {
            const float w = Wv[v];
            const float al = acc / (w > eps ? w : eps);
            aip[v] = make_float2(al, (w > eps) ? al * Iv[v] : 0.0f);
        } else {
            dsrc[v] = acc;
        }
    }
}

constexpr int kPlaneSmem = 48 * 1024;

template <bool kPrep, int K>
static bool launch_adj_plane_k(const float* dd, const ResGeo& G, const float* I, const float* W,
                               float eps, float* dsrc, float2* aip, cudaStream_t st) {
    const int nx = G.a[0].n_src, ny = G.a[1].n_src, nz = G.a[2].n_src, lnx = G.a[0].n_dst;
    const size_t base = sizeof(ResRun<K>) * size_t(nx);
    if (nz > 65535) return false;
    if (base + (sizeof(ResRun<K>) + sizeof(float) * lnx) * 32 <= size_t(kPlaneSmem)) {
        const size_t smem = base + (sizeof(ResRun<K>) + sizeof(float) * lnx) * 32;
        launch_k(k_resample_adj_plane<kPrep, K, 32>, dim3(dim3(nz, (ny + 31) / 32)), dim3(256),
            smem, st, dd, G, I, W, eps, dsrc, aip);
        return true;
    }
    if (base + (sizeof(ResRun<K>) + sizeof(float) * lnx) * 8 <= size_t(kPlaneSmem)) {
        const size_t smem = base + (sizeof(ResRun<K>) + sizeof(float) * lnx) * 8;
        launch_k(k_resample_adj_plane<kPrep, K, 8>, dim3(dim3(nz, (ny + 7) / 8)), dim3(256), smem,
            st, dd, G, I, W, eps, dsrc, aip);
        return true;
    }
    return false;
}

template <bool kPrep>
static bool launch_adj_plane(const float* dd, const ResGeo& G, const float* I, const float* W,
                             float eps, float* dsrc, float2* aip, cudaStream_t st) {
    if (!res_list_ok(G)) return false;
    if (res_two_taps(G)) return launch_adj_plane_k<kPrep, 2>(dd, G, I, W, eps, dsrc, aip, st);
    return launch_adj_plane_k<kPrep, kResList>(dd, G, I, W, eps, dsrc, aip, st);
}

template <bool kPrep>
static bool launch_adj_tab(const float* dd, const ResGeo& G, const float* I, const float* W,
                           float eps, float* dsrc, float2* aip, cudaStream_t st) {
    const int n_tab = G.a[0].n_src + G.a[1].n_src + G.a[2].n_src;
    if (!res_list_ok(G) || n_tab > kResTabMax) return false;
    const int64_t rows = int64_t(G.a[2].n_src) * G.a[1].n_src;
    const unsigned nb = static_cast<unsigned>(rows < 152 * 8 ? rows : 152 * 8);
    if (res_two_taps(G))
        launch_k(k_resample_adj_tab<kPrep, 2>, dim3(nb), dim3(256), sizeof(ResRun<2>) * n_tab, st,
            dd, G, I, W, eps, dsrc, aip);
    else
        launch_k(k_resample_adj_tab<kPrep, kResList>, dim3(nb), dim3(256),
            sizeof(ResRun<kResList>) * n_tab, st, dd, G, I, W, eps, dsrc, aip);
    return true;
}

gs_status resample_adj_prep_impl(const float* dlr, int32_t lnz, int32_t lny, int32_t lnx,
                                 const float* I, const float* W, int32_t nz, int32_t ny, int32_t nx,
                                 float eps, float2* aip, cudaStream_t st) {
    const ResGeo G = make_res(nz, ny, nx, lnz, lny, lnx);
    if (!launch_adj_plane<true>(dlr, G, I, W, eps, nullptr, aip, st) &&
        !launch_adj_tab<true>(dlr, G, I, W, eps, nullptr, aip, st))
        launch_k(k_resample_adj_prep, dim3(res_blocks(int64_t(nz) * ny * nx)), dim3(256), 0, st,
            dlr, G, I, W, eps, aip);
    return last_launch_status();
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_resample_fwd(const float* src, int32_t snz, int32_t sny, int32_t snx,
                                     float* dst, int32_t dnz, int32_t dny, int32_t dnx,
                                     gs_stream stream) {
    if (!src || !dst || !dims_ok(snz, sny, snx) || !dims_ok(dnz, dny, dnx)) return GS_ERR_INVALID_ARG;
    return resample_fwd_impl(src, snz, sny, snx, dst, dnz, dny, dnx,
                             reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_resample_bwd(const float* ddst, int32_t dnz, int32_t dny, int32_t dnx,
                                     float* dsrc, int32_t snz, int32_t sny, int32_t snx,
                                     gs_stream stream) {
    if (!ddst || !dsrc || !dims_ok(snz, sny, snx) || !dims_ok(dnz, dny, dnx)) return GS_ERR_INVALID_ARG;
    const ResGeo G = make_res(snz, sny, snx, dnz, dny, dnx);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!launch_adj_plane<false>(ddst, G, nullptr, nullptr, 0.f, dsrc, nullptr, st) &&
        !launch_adj_tab<false>(ddst, G, nullptr, nullptr, 0.f, dsrc, nullptr, st))
        launch_k(k_resample_bwd, dim3(res_blocks(int64_t(snz) * sny * snx)), dim3(256), 0, st, ddst,
            G, dsrc);
    return last_launch_status();
}
