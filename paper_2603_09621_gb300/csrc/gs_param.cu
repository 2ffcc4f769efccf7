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
    pdl_enter();
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

// dL/d(raw params) of one Gaussian from its render-space gradient g[11] (see above).
// Returns false (and zeros) for an invalid Gaussian.
__device__ __forceinline__ void chain_one(const float* p, const float* gv, const ChainGeo& C,
                                          float* out) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) ok = ok && isfinite(p[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) ok = ok && (fabsf(p[3 + k]) <= 30.0f);
    const float nn = p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9];
    ok = ok && (nn > 0.0f);
    if (!ok) {
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = 0.0f;
        return;
    }
    const float m1[3] = {gv[G_M1X] * C.h[0], gv[G_M1Y] * C.h[1], gv[G_M1Z] * C.h[2]};  // H m1
    // M2 (index space) -> G = -1/2 H M2 H
    float Gm[3][3];
    Gm[0][0] = -0.5f * C.h[0] * C.h[0] * gv[G_M2XX];
    Gm[1][1] = -0.5f * C.h[1] * C.h[1] * gv[G_M2YY];
    Gm[2][2] = -0.5f * C.h[2] * C.h[2] * gv[G_M2ZZ];
    Gm[0][1] = Gm[1][0] = -0.5f * C.h[0] * C.h[1] * gv[G_M2XY];
    Gm[0][2] = Gm[2][0] = -0.5f * C.h[0] * C.h[2] * gv[G_M2XZ];
    Gm[1][2] = Gm[2][1] = -0.5f * C.h[1] * C.h[2] * gv[G_M2YZ];
    const float dv = gv[G_DV], dr = gv[G_DR];

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
}

__device__ __forceinline__ void load12(const float* src, float* d) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4 a = s4[0], b = s4[1], c = s4[2];
    d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
    d[8] = c.x; d[9] = c.y; d[10] = c.z; d[11] = c.w;
}

__device__ __forceinline__ void store12(float* dst, const float* d) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    d4[0] = make_float4(d[0], d[1], d[2], d[3]);
    d4[1] = make_float4(d[4], d[5], d[6], d[7]);
    d4[2] = make_float4(d[8], d[9], d[10], d[11]);
}

__global__ void __launch_bounds__(256) k_param_bwd(const float* __restrict__ params,
                                                   const float* __restrict__ gacc, int64_t N,
                                                   ChainGeo C, float* __restrict__ dparams) {
    pdl_enter();
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float p[12], gv[12], out[12];
    load12(params + g * 12, p);
    load12(gacc + g * GRAD_FLOATS, gv);
    chain_one(p, gv, C, out);
    store12(dparams + g * 12, out);
}

gs_status launch_param_bwd(const float* params, const float* gacc, int64_t n, const gs_grid* grid,
                           const gs_config* cfg, float* dparams, cudaStream_t st) {
    ChainGeo C;
    for (int k = 0; k < 3; ++k) C.h[k] = grid->h[k];
    C.signal_mode = cfg->signal_mode;
    C.a_act = cfg->a_act;
    C.t_act = cfg->t_act;
    launch_k(k_param_bwd, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, st, params,
        gacc, n, C, dparams);
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

struct AdamCoef {
    float bc1, rs_bc2;
};

__device__ __forceinline__ AdamCoef adam_coef(const AdamLr& hp, const int32_t* d_step) {
    const int t = *d_step + 1;
    // bias corrections 1 - beta^t = -expm1(t log beta), accurate for small t (1 - beta ~ 1e-3)
    AdamCoef c;
    c.bc1 = -expm1f(float(t) * hp.log_b1);
    c.rs_bc2 = 1.0f / sqrtf(-expm1f(float(t) * hp.log_b2));
    return c;
}

__device__ __forceinline__ float adam_one(float& p, float gr, float& m, float& v, float lr,
                                          const AdamLr& hp, const AdamCoef& c) {
    const float mi = hp.beta1 * m + hp.omb1 * gr;
    const float vi = hp.beta2 * v + hp.omb2 * gr * gr;
    m = mi;
    v = vi;
    const float denom = sqrtf(vi) * c.rs_bc2 + hp.eps;
    p -= (lr / c.bc1) * mi / denom;
    return p;
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ params, const float* __restrict__ grad,
                                              float* __restrict__ m, float* __restrict__ v, int64_t n,
                                              AdamLr hp, const int32_t* __restrict__ d_step,
                                              const int32_t* __restrict__ d_skip) {
    pdl_enter();
    if (d_skip && *d_skip != 0) return;  // the step was declared a no-op (see gs_fit_apply)
    const AdamCoef c = adam_coef(hp, d_step);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        float p = params[i], mi = m[i], vi = v[i];
        adam_one(p, grad[i], mi, vi, hp.lr[lr_group(static_cast<int>(i % 12))], hp, c);
        params[i] = p;
        m[i] = mi;
        v[i] = vi;
    }
}

// Fitting step tail, one thread per Gaussian: sum the per-brick partials in Gaussian-major
// order (deterministic mode) or take the atomically accumulated gradient, chain it to the
// raw parameters (written to grad), and (kAdam) apply Adam to params, m, v.
template <bool kDet, bool kAdam>
__global__ void __launch_bounds__(256, 4) k_chain_adam(
    float* __restrict__ params, float* __restrict__ grad, float* __restrict__ m,
    float* __restrict__ v, const float* __restrict__ part, const float* __restrict__ gacc,
    const int32_t* __restrict__ gm_off, const int64_t* __restrict__ npairs, int64_t capacity,
    int64_t N, ChainGeo C, AdamLr hp, const int32_t* __restrict__ d_step) {
    pdl_enter();
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float gv[12];
    const int64_t P = *npairs;
    if (P < 0 || P > capacity) {
        // The binning overflowed: this step rendered nothing, so it leaves the parameters and
        // moments as they are (the caller grows the bins and repeats the step).
#pragma unroll
        for (int k = 0; k < 12; ++k) gv[k] = 0.f;
        store12(grad + g * 12, gv);
        return;
    }
    if (kDet) {
#pragma unroll
        for (int k = 0; k < 12; ++k) gv[k] = 0.f;
        const int a = gm_off[g], e = gm_off[g + 1];
        for (int j = a; j < e; ++j) {
            float t[12];
            load12(part + int64_t(j) * GRAD_FLOATS, t);
#pragma unroll
            for (int k = 0; k < 11; ++k) gv[k] += t[k];
        }
    } else {
        load12(gacc + g * GRAD_FLOATS, gv);
    }
    float p[12], out[12], mm[12], vv[12];
    load12(params + g * 12, p);
    chain_one(p, gv, C, out);
    store12(grad + g * 12, out);
    if (!kAdam) return;
    load12(m + g * 12, mm);
    load12(v + g * 12, vv);
    const AdamCoef c = adam_coef(hp, d_step);
#pragma unroll
    for (int k = 0; k < 12; ++k) adam_one(p[k], out[k], mm[k], vv[k], hp.lr[lr_group(k)], hp, c);
    store12(params + g * 12, p);
    store12(m + g * 12, mm);
    store12(v + g * 12, vv);
}

// Counts a step, unless npairs is given and the step's binning overflowed the pair capacity
// (then the fitting step was a no-op), or d_skip is given and nonzero.
__global__ void k_step_inc(int32_t* d_step, const int64_t* __restrict__ npairs, int64_t capacity,
                           const int32_t* __restrict__ d_skip) {
    pdl_enter();
    if (d_skip && *d_skip != 0) return;
    if (npairs) {
        const int64_t P = *npairs;
        if (P < 0 || P > capacity) return;
    }
    *d_step += 1;
}

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
    pdl_enter();
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

namespace gs {
static AdamLr make_adam_lr(const gs_adam* hp) {
    AdamLr a;
    a.lr[0] = hp->lr_mu;
    a.lr[1] = hp->lr_scale;
    a.lr[2] = hp->lr_rot;
    a.lr[3] = hp->lr_a;
    a.lr[4] = hp->lr_t;
    a.beta1 = static_cast<float>(hp->beta1);
    a.beta2 = static_cast<float>(hp->beta2);
    a.omb1 = static_cast<float>(1.0 - hp->beta1);
    a.omb2 = static_cast<float>(1.0 - hp->beta2);
    a.log_b1 = static_cast<float>(log(hp->beta1 > 0.0 ? hp->beta1 : 1e-300));
    a.log_b2 = static_cast<float>(log(hp->beta2 > 0.0 ? hp->beta2 : 1e-300));
    a.eps = static_cast<float>(hp->eps);
    return a;
}

static bool adam_ok(const gs_adam* hp) {
    return hp->beta1 >= 0.0 && hp->beta1 < 1.0 && hp->beta2 >= 0.0 && hp->beta2 < 1.0 &&
           hp->eps > 0.0;
}

gs_status launch_chain_adam(float* params, float* grad, float* m, float* v, const float* part,
                            const float* gacc, const gs_bins* bins, int64_t n,
                            const gs_grid* grid, const gs_config* cfg, const gs_adam* hp,
                            int32_t* d_step, cudaStream_t st) {
    if (!adam_ok(hp)) return GS_ERR_INVALID_ARG;
    ChainGeo C;
    for (int k = 0; k < 3; ++k) C.h[k] = grid->h[k];
    C.signal_mode = cfg->signal_mode;
    C.a_act = cfg->a_act;
    C.t_act = cfg->t_act;
    const AdamLr a = make_adam_lr(hp);
    const unsigned gb = static_cast<unsigned>((n + 255) / 256);
    if (cfg->deterministic)
        launch_k(k_chain_adam<true, true>, dim3(gb), dim3(256), 0, st, params, grad, m, v, part,
            gacc, bins->gm_off, bins->d_npairs, bins->capacity, n, C, a, d_step);
    else
        launch_k(k_chain_adam<false, true>, dim3(gb), dim3(256), 0, st, params, grad, m, v, part,
            gacc, bins->gm_off, bins->d_npairs, bins->capacity, n, C, a, d_step);
    gs_status s = last_launch_status();
    if (s != GS_OK) return s;
    launch_k(k_step_inc, dim3(1), dim3(1), 0, st, d_step, bins->d_npairs, bins->capacity,
        static_cast<const int32_t*>(nullptr));
    return last_launch_status();
}

// The same tail without Adam: the raw-parameter gradient of the step into grad (zero when
// the step's binning overflowed).
gs_status launch_chain_grad(const float* params, float* grad, const float* part,
                            const float* gacc, const gs_bins* bins, int64_t n,
                            const gs_grid* grid, const gs_config* cfg, cudaStream_t st) {
    ChainGeo C;
    for (int k = 0; k < 3; ++k) C.h[k] = grid->h[k];
    C.signal_mode = cfg->signal_mode;
    C.a_act = cfg->a_act;
    C.t_act = cfg->t_act;
    const AdamLr a = {};
    const unsigned gb = static_cast<unsigned>((n + 255) / 256);
    float* p = const_cast<float*>(params);  // read only without Adam
    if (cfg->deterministic)
        launch_k(k_chain_adam<true, false>, dim3(gb), dim3(256), 0, st, p, grad,
            static_cast<float*>(nullptr), static_cast<float*>(nullptr), part, gacc, bins->gm_off,
            bins->d_npairs, bins->capacity, n, C, a, static_cast<const int32_t*>(nullptr));
    else
        launch_k(k_chain_adam<false, false>, dim3(gb), dim3(256), 0, st, p, grad,
            static_cast<float*>(nullptr), static_cast<float*>(nullptr), part, gacc, bins->gm_off,
            bins->d_npairs, bins->capacity, n, C, a, static_cast<const int32_t*>(nullptr));
    return last_launch_status();
}

// Adam over n values of params with grad, moments m, v and the step counter d_step; nothing
// changes when d_skip is given and nonzero.
gs_status launch_adam(float* params, const float* grad, float* m, float* v, int64_t n_gauss,
                      const gs_adam* hp, int32_t* d_step, const int32_t* d_skip,
                      cudaStream_t st) {
    if (n_gauss > 0) {
        if (!adam_ok(hp)) return GS_ERR_INVALID_ARG;
        const AdamLr a = make_adam_lr(hp);
        const int64_t n = n_gauss * 12;
        const int64_t blocks64 = (n + 255) / 256;
        const unsigned blocks = static_cast<unsigned>(blocks64 < 65536 ? blocks64 : 65536);
        launch_k(k_adam, dim3(blocks), dim3(256), 0, st, params, grad, m, v, n, a, d_step, d_skip);
        gs_status s = last_launch_status();
        if (s != GS_OK) return s;
    }
    launch_k(k_step_inc, dim3(1), dim3(1), 0, st, d_step, static_cast<const int64_t*>(nullptr),
        int64_t(0), d_skip);
    return last_launch_status();
}
}  // namespace gs

extern "C" gs_status gs_signal_proxy(const float* T1, const float* T2, int64_t n, float TR, float TE,
                                     float* T_out, gs_stream stream) {
    if (n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!T1 || !T2 || !T_out) return GS_ERR_INVALID_ARG;
    const int64_t blocks64 = (n + 255) / 256;
    const unsigned blocks = static_cast<unsigned>(blocks64 < 65536 ? blocks64 : 65536);
    launch_k(k_signal_proxy, dim3(blocks), dim3(256), 0, reinterpret_cast<cudaStream_t>(stream), T1,
        T2, n, TR, TE, T_out);
    return last_launch_status();
}

extern "C" gs_status gs_adam_step(float* params, const float* grad, float* m, float* v,
                                  int64_t n_gauss, const gs_adam* hp, int32_t* d_step,
                                  gs_stream stream) {
    if (n_gauss < 0 || !hp || !d_step) return GS_ERR_INVALID_ARG;
    if (n_gauss > 0 && (!params || !grad || !m || !v)) return GS_ERR_INVALID_ARG;
    return launch_adam(params, grad, m, v, n_gauss, hp, d_step, nullptr,
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gs_status gs_init_lattice_lr(const float* lr, int32_t lnz, int32_t lny, int32_t lnx,
                                        const gs_grid* g, int32_t nlx, int32_t nly, int32_t nlz,
                                        int32_t t_act, float t_init, float* params,
                                        gs_stream stream) {
    if (!lr || !g || !params || nlx <= 0 || nly <= 0 || nlz <= 0) return GS_ERR_INVALID_ARG;
    if (lnx <= 0 || lny <= 0 || lnz <= 0 || g->nx <= 0 || g->ny <= 0 || g->nz <= 0)
        return GS_ERR_INVALID_ARG;
    if (t_act && !(t_init > 0.0f && t_init < 1.0f)) return GS_ERR_INVALID_ARG;
    InitGeo G;
    G.nx = lnx;
    G.ny = lny;
    G.nzl = lnz;
    const int n[3] = {g->nx, g->ny, g->nz};
    const int ln[3] = {lnx, lny, lnz};
    const int nl[3] = {nlx, nly, nlz};
    for (int a = 0; a < 3; ++a) {
        G.o[a] = g->origin[a];
        G.ext[a] = double(n[a]) * double(g->h[a]);
        G.hl[a] = G.ext[a] / double(ln[a]);
        G.nl[a] = nl[a];
        G.log_s[a] = static_cast<float>(log(0.5 * G.ext[a] / double(nl[a])));
    }
    G.t_raw = t_act ? static_cast<float>(log(double(t_init) / (1.0 - double(t_init)))) : t_init;
    const int64_t N = int64_t(nlx) * nly * nlz;
    launch_k(k_init_lattice, dim3(static_cast<unsigned>((N + 255) / 256)), dim3(256), 0,
        reinterpret_cast<cudaStream_t>(stream), lr, G, params);
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
    launch_k(k_init_lattice, dim3(static_cast<unsigned>((N + 255) / 256)), dim3(256), 0,
        reinterpret_cast<cudaStream_t>(stream), lr, G, params);
    return last_launch_status();
}
