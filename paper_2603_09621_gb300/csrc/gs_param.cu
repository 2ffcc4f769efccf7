// gs_param.cu -- per-Gaussian elementwise kernels: Eq. 2 signal proxy, the chain from the
// render-space adjoint to the raw parameters (Sec. 3.1 parameterisation), bias-corrected Adam,
// and the lattice initialisation from the LR volume (Fig. 1 caption).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gs_common.cuh"

namespace gs {

// ------------------------------------------------------------------------ Eq. 2
__global__ void k_signal_proxy(const float* __restrict__ T1, const float* __restrict__ T2,
                               int64_t n, float TR, float TE, float* __restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = -expm1f(-TR / T1[i]) * expf(-TE / T2[i]);
}

// ------------------------------------------------------------------------ chain
// Render-space gradient (m1 = sum G d, m2 = sum G d d^T in voxel index space, dv, dr; G is
// dL/dw times w of each contributing pair) -> dL/d(raw params):
//   dL/dmu = Sigma^{-1} H m1                      (world units, H = diag(h))
//   dL/dSigma^{-1} = -1/2 H M2 H                  (full symmetric matrix)
//   Sigma^{-1} = R D R^T, D = diag(s^-2):  dL/dlog_s_m = -2 D_mm (R^T G R)_mm,
//                                          dL/dR = 2 G R D,
//   R(q_n) for the unit quaternion q_n = q / |q|, then dq = (dq_n - q_n (q_n . dq_n)) / |q|,
//   (v, r) -> (A, T) by the signal mode, then the identity / sigmoid activations.
struct ChainGeo {
    float h[3];
    int signal_mode, a_act, t_act;
};

__global__ void __launch_bounds__(256) k_param_bwd(const float* __restrict__ params,
                                                   const float* __restrict__ gacc, int64_t N,
                                                   ChainGeo C, float* __restrict__ dparams) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const float4* p4 = reinterpret_cast<const float4*>(params + g * 12);
    const float4 a0 = p4[0], a1 = p4[1], a2 = p4[2];
    const float p[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
    float4* d4 = reinterpret_cast<float4*>(dparams + g * 12);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) ok = ok && isfinite(p[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) ok = ok && (fabsf(p[3 + k]) <= 30.0f);
    const float nn = p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9];
    ok = ok && (nn > 0.0f);
    if (!ok) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        d4[0] = z; d4[1] = z; d4[2] = z;
        return;
    }
    const float4* g4 = reinterpret_cast<const float4*>(gacc + g * GRAD_FLOATS);
    const float4 b0 = g4[0], b1 = g4[1], b2 = g4[2];
    const float m1[3] = {b0.x * C.h[0], b0.y * C.h[1], b0.z * C.h[2]};  // H m1
    // M2 (index space) -> G = -1/2 H M2 H
    float Gm[3][3];
    Gm[0][0] = -0.5f * C.h[0] * C.h[0] * b0.w;
    Gm[1][1] = -0.5f * C.h[1] * C.h[1] * b1.x;
    Gm[2][2] = -0.5f * C.h[2] * C.h[2] * b1.y;
    Gm[0][1] = Gm[1][0] = -0.5f * C.h[0] * C.h[1] * b1.z;
    Gm[0][2] = Gm[2][0] = -0.5f * C.h[0] * C.h[2] * b1.w;
    Gm[1][2] = Gm[2][1] = -0.5f * C.h[1] * C.h[2] * b2.x;
    const float dv = b2.y, dr = b2.z;

    float s[3], D[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s[k] = exp_cw(p[3 + k]);
        D[k] = 1.0f / (s[k] * s[k]);
    }
    const float n = sqrtf(nn);
    const float w = p[6] / n, x = p[7] / n, y = p[8] / n, z = p[9] / n;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (y * y + z * z);
    R[0][1] = 2.f * (x * y - w * z);
    R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);
    R[1][1] = 1.f - 2.f * (x * x + z * z);
    R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);
    R[2][1] = 2.f * (y * z + w * x);
    R[2][2] = 1.f - 2.f * (x * x + y * y);
    // Sigma^{-1} and dmu
    float Ci[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Ci[a][b] = R[a][0] * R[b][0] * D[0] + R[a][1] * R[b][1] * D[1] + R[a][2] * R[b][2] * D[2];
    float out[12];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = Ci[a][0] * m1[0] + Ci[a][1] * m1[1] + Ci[a][2] * m1[2];
    // G R (3x3)
    float GR[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < 3; ++m)
            GR[a][m] = Gm[a][0] * R[0][m] + Gm[a][1] * R[1][m] + Gm[a][2] * R[2][m];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float rtgr = R[0][m] * GR[0][m] + R[1][m] * GR[1][m] + R[2][m] * GR[2][m];
        out[3 + m] = -2.0f * D[m] * rtgr;
    }
    float dR[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < 3; ++m) dR[a][m] = 2.0f * GR[a][m] * D[m];
    float dq[4];
    dq[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] +
                   x * dR[2][1]);
    dq[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                   z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    dq[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                   w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    dq[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] -
                   2.f * z * dR[1][1] + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float qn[4] = {w, x, y, z};
    const float dot = qn[0] * dq[0] + qn[1] * dq[1] + qn[2] * dq[2] + qn[3] * dq[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) out[6 + k] = (dq[k] - qn[k] * dot) / n;
    const float A = C.a_act ? sigmoidf_(p[10]) : p[10];
    const float T = C.t_act ? sigmoidf_(p[11]) : p[11];
    float dA, dT;
    if (C.signal_mode == 0) {
        dA = dv;
        dT = dr;
    } else {
        dA = dv * T;
        dT = dv * A;
    }
    out[10] = C.a_act ? dA * A * (1.0f - A) : dA;
    out[11] = C.t_act ? dT * T * (1.0f - T) : dT;
    d4[0] = make_float4(out[0], out[1], out[2], out[3]);
    d4[1] = make_float4(out[4], out[5], out[6], out[7]);
    d4[2] = make_float4(out[8], out[9], out[10], out[11]);
}

gs_status launch_param_bwd(const float* params, const float* gacc, int64_t n, const gs_grid* grid,
                           const gs_config* cfg, float* dparams, cudaStream_t st) {
    ChainGeo C;
    for (int k = 0; k < 3; ++k) C.h[k] = grid->h[k];
    C.signal_mode = cfg->signal_mode;
    C.a_act = cfg->a_act;
    C.t_act = cfg->t_act;
    k_param_bwd<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(params, gacc, n, C, dparams);
    return last_launch_status();
}

// ------------------------------------------------------------------------ Adam
struct AdamLr {
    float lr[5];
    float beta1, beta2;          // decay rates
    float omb1, omb2;            // 1 - beta, formed in double on the host
    float log_b1, log_b2;        // log(beta), formed in double on the host
    float eps;
};

__device__ __forceinline__ int lr_group(int col) {
    return col < 3 ? 0 : (col < 6 ? 1 : (col < 10 ? 2 : (col == 10 ? 3 : 4)));
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ params, const float* __restrict__ grad,
                                              float* __restrict__ m, float* __restrict__ v, int64_t n,
                                              AdamLr hp, const int32_t* __restrict__ d_step) {
    const int t = *d_step + 1;
    // bias corrections 1 - beta^t = -expm1(t log beta), accurate for small t (1 - beta ~ 1e-3)
    const float bc1 = -expm1f(float(t) * hp.log_b1);
    const float bc2 = -expm1f(float(t) * hp.log_b2);
    const float rs_bc2 = 1.0f / sqrtf(bc2);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float gr = grad[i];
        const float mi = hp.beta1 * m[i] + hp.omb1 * gr;
        const float vi = hp.beta2 * v[i] + hp.omb2 * gr * gr;
        m[i] = mi;
        v[i] = vi;
        const float lr = hp.lr[lr_group(static_cast<int>(i % 12))];
        const float denom = sqrtf(vi) * rs_bc2 + hp.eps;
        params[i] -= (lr / bc1) * mi / denom;
    }
}

__global__ void k_step_inc(int32_t* d_step) { *d_step += 1; }

// ------------------------------------------------------------------------ init
struct InitGeo {
    int nx, ny, nzl;         // LR volume dims
    double o[3], hl[3];      // origin, LR spacing
    double ext[3];           // HR extent L = n h
    int nl[3];               // lattice counts
    float log_s[3];
    float t_raw;
};

__global__ void __launch_bounds__(256) k_init_lattice(const float* __restrict__ lr, InitGeo G,
                                                      float* __restrict__ params) {
    const int64_t n = int64_t(G.nl[0]) * G.nl[1] * G.nl[2];
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int i = static_cast<int>(g % G.nl[0]);
    const int j = static_cast<int>((g / G.nl[0]) % G.nl[1]);
    const int k = static_cast<int>(g / (int64_t(G.nl[0]) * G.nl[1]));
    const int idx[3] = {i, j, k};
    const int dims[3] = {G.nx, G.ny, G.nzl};
    // Lattice centres and LR continuous indices in FP64 (a handful of operations per point).
    float c[3], f[3];
    int i0[3], i1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double cd = G.o[a] + (double(idx[a]) + 0.5) * (G.ext[a] / double(G.nl[a]));
        double u = (cd - G.o[a]) / G.hl[a] - 0.5;
        u = fmin(fmax(u, 0.0), double(dims[a] - 1));
        i0[a] = static_cast<int>(floor(u));
        i1[a] = min(i0[a] + 1, dims[a] - 1);
        f[a] = static_cast<float>(u - double(i0[a]));
        c[a] = static_cast<float>(cd);
    }
    float acc = 0.f;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const float wgt = (cx ? f[0] : 1.f - f[0]) * (cy ? f[1] : 1.f - f[1]) *
                                  (cz ? f[2] : 1.f - f[2]);
                const int xi = cx ? i1[0] : i0[0], yi = cy ? i1[1] : i0[1], zi = cz ? i1[2] : i0[2];
                acc += wgt * lr[(int64_t(zi) * G.ny + yi) * G.nx + xi];
            }
    float4* o4 = reinterpret_cast<float4*>(params + g * 12);
    o4[0] = make_float4(c[0], c[1], c[2], G.log_s[0]);
    o4[1] = make_float4(G.log_s[1], G.log_s[2], 1.0f, 0.0f);
    o4[2] = make_float4(0.0f, 0.0f, acc, G.t_raw);
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_signal_proxy(const float* T1, const float* T2, int64_t n, float TR, float TE,
                                     float* T_out, gs_stream stream) {
    if (n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!T1 || !T2 || !T_out) return GS_ERR_INVALID_ARG;
    const int64_t blocks64 = (n + 255) / 256;
    const unsigned blocks = static_cast<unsigned>(blocks64 < 65536 ? blocks64 : 65536);
    k_signal_proxy<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(T1, T2, n, TR, TE, T_out);
    return last_launch_status();
}

extern "C" gs_status gs_adam_step(float* params, const float* grad, float* m, float* v,
                                  int64_t n_gauss, const gs_adam* hp, int32_t* d_step,
                                  gs_stream stream) {
    if (n_gauss < 0 || !hp || !d_step) return GS_ERR_INVALID_ARG;
    if (n_gauss > 0 && (!params || !grad || !m || !v)) return GS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n_gauss > 0) {
        AdamLr a;
        a.lr[0] = hp->lr_mu;
        a.lr[1] = hp->lr_scale;
        a.lr[2] = hp->lr_rot;
        a.lr[3] = hp->lr_a;
        a.lr[4] = hp->lr_t;
        if (!(hp->beta1 >= 0.0 && hp->beta1 < 1.0 && hp->beta2 >= 0.0 && hp->beta2 < 1.0 &&
              hp->eps > 0.0))
            return GS_ERR_INVALID_ARG;
        a.beta1 = static_cast<float>(hp->beta1);
        a.beta2 = static_cast<float>(hp->beta2);
        a.omb1 = static_cast<float>(1.0 - hp->beta1);
        a.omb2 = static_cast<float>(1.0 - hp->beta2);
        a.log_b1 = static_cast<float>(log(hp->beta1 > 0.0 ? hp->beta1 : 1e-300));
        a.log_b2 = static_cast<float>(log(hp->beta2 > 0.0 ? hp->beta2 : 1e-300));
        a.eps = static_cast<float>(hp->eps);
        const int64_t n = n_gauss * 12;
        const int64_t blocks64 = (n + 255) / 256;
        const unsigned blocks = static_cast<unsigned>(blocks64 < 65536 ? blocks64 : 65536);
        k_adam<<<blocks, 256, 0, st>>>(params, grad, m, v, n, a, d_step);
        gs_status s = last_launch_status();
        if (s != GS_OK) return s;
    }
    k_step_inc<<<1, 1, 0, st>>>(d_step);
    return last_launch_status();
}

extern "C" gs_status gs_init_lattice(const float* lr, const gs_grid* g, int32_t s, int32_t nlx,
                                     int32_t nly, int32_t nlz, int32_t t_act, float t_init,
                                     float* params, gs_stream stream) {
    if (!lr || !g || !params || s <= 0 || nlx <= 0 || nly <= 0 || nlz <= 0) return GS_ERR_INVALID_ARG;
    if (g->nx <= 0 || g->ny <= 0 || g->nz / s <= 0) return GS_ERR_INVALID_ARG;
    if (t_act && !(t_init > 0.0f && t_init < 1.0f)) return GS_ERR_INVALID_ARG;
    InitGeo G;
    G.nx = g->nx;
    G.ny = g->ny;
    G.nzl = g->nz / s;
    const int n[3] = {g->nx, g->ny, g->nz};
    const int nl[3] = {nlx, nly, nlz};
    for (int a = 0; a < 3; ++a) {
        G.o[a] = g->origin[a];
        G.hl[a] = double(g->h[a]) * (a == 2 ? double(s) : 1.0);
        G.ext[a] = double(n[a]) * double(g->h[a]);
        G.nl[a] = nl[a];
        G.log_s[a] = static_cast<float>(log(0.5 * G.ext[a] / double(nl[a])));
    }
    G.t_raw = t_act ? static_cast<float>(log(double(t_init) / (1.0 - double(t_init)))) : t_init;
    const int64_t N = int64_t(nlx) * nly * nlz;
    k_init_lattice<<<static_cast<unsigned>((N + 255) / 256), 256, 0,
                     reinterpret_cast<cudaStream_t>(stream)>>>(lr, G, params);
    return last_launch_status();
}
