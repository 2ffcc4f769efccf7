/*
 * gs_oracle.c -- plain FP64 CPU oracle for physics-grounded Gaussian volume rendering.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference leg may load this library. The product path (the CUDA library
 * in the package) never calls, links or imports anything here, and this file shares no
 * code, header, constant table or helper with it.
 *
 * What it computes (paper: "Physics-Driven 3D Gaussian Rendering for Zero-Shot MRI
 * Super-Resolution"):
 *   - Sec. 3.1 / Eq. 2: relaxation proxy T = (1 - exp(-TR/T1)) * exp(-TE/T2).
 *   - Sec. 3.2 / Eq. 3-4: I(p) = sum_i A_i w_i(p) / sum_i w_i(p),
 *       w_i(p) = exp(-1/2 (p-mu_i)^T Sigma_i^{-1} (p-mu_i)) * r_i.
 *   - Sec. 3.3: Gaussians are truncated at their 3-sigma Mahalanobis ellipsoid; a pair
 *     (i, p) contributes only when d^2 = (p-mu)^T Sigma^{-1} (p-mu) <= sigma_t^2 (inclusive).
 *   - Sec. 3.3 / Eq. 5-6: gradients of a loss through the normalised aggregation,
 *     dL/dtheta_i = sum_p dL/dI(p) (A_i - I(p))/W(p) dw_i/dtheta_i and
 *     dL/dA_i = sum_p dL/dI(p) w_i(p)/W(p); the relaxation factor gets the analogous term
 *     (w is linear in r). The chain continues to the raw parameters (log-scale, quaternion).
 *
 * Readings where the paper is silent (each is listed with its reason in the design notes):
 *   - r_i = T_i (signal mode 0); signal mode 1 uses v_i = A_i T_i and r_i = 1.
 *   - I = S / max(W, eps); for W < eps, dI/dw_i = v_i / eps.
 *   - Sigma = R diag(s^2) R^T with s = exp(log_s) and R from the normalised quaternion
 *     (w, x, y, z); A and T use an identity or a sigmoid activation.
 *   - Voxel (i, j, k) of a grid with spacing h and origin o has centre o + (i+1/2, j+1/2, k+1/2) h.
 *   - Gaussians whose raw parameters are non-finite, whose quaternion is zero or whose
 *     log-scale lies outside [-30, 30] are invalid and contribute nothing.
 *
 * Everything is a direct loop over voxels and Gaussians in FP64, in ascending Gaussian order.
 * The only shortcut is an exact bounding box per Gaussian: d^2 >= |p-mu|^2 / s_max^2, so a
 * voxel farther than sigma_t * s_max (padded) from mu cannot contribute; skipping it adds
 * exactly nothing. `prune = 0` turns the shortcut off (tests check both give equal results).
 *
 * og_bins_fp32 is the one FP32 routine: the brick-binning decision (an integer result decided
 * by floating point) is taken in the GPU kernel's precision with a fully specified operation
 * order (no contraction, Cody-Waite exponential), so brick lists can be compared bit-exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_NPARAM 12

/* ---------------------------------------------------------------- Eq. 2 */

/* Eq. 2: relaxation proxy of a tissue with relaxation times T1, T2 at repetition time TR and
 * echo time TE (all in the same time unit). */
double og_signal_proxy1(double T1, double T2, double TR, double TE) {
    return (1.0 - exp(-TR / T1)) * exp(-TE / T2);
}

void og_signal_proxy(const double* T1, const double* T2, int64_t n, double TR, double TE,
                     double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = og_signal_proxy1(T1[i], T2[i], TR, TE);
}

/* ------------------------------------------------------ per-Gaussian state */

typedef struct {
    int valid;
    double mu[3];
    double s[3];       /* scales (standard deviations along the principal axes) */
    double qn[4];      /* normalised quaternion (w, x, y, z) */
    double qnorm;      /* |q| before normalisation */
    double R[3][3];    /* rotation matrix */
    double C[3][3];    /* Sigma^{-1} = R diag(1/s^2) R^T */
    double A, T;       /* activated amplitude and relaxation proxy */
    double v, r;       /* signal and relaxation factor entering Eq. 3-4 */
    int lo[3], hi[3];  /* voxel index box that may contain d^2 <= sigma_t^2 (+ ambiguity band) */
} og_gauss;

static double og_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static int og_finite(double x) { return isfinite(x) ? 1 : 0; }

/* Rotation matrix of the unit quaternion (w, x, y, z) (Hamilton convention). */
static void og_quat_to_R(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void og_activate(const double* p, const int32_t dims[3], const double h[3],
                        const double origin[3], double sigma_t, double amb_tol,
                        int signal_mode, int a_act, int t_act, int prune, og_gauss* g) {
    memset(g, 0, sizeof(*g));
    for (int k = 0; k < OG_NPARAM; ++k)
        if (!og_finite((double)p[k])) return;
    double qn2 = 0.0;
    for (int k = 0; k < 4; ++k) qn2 += (double)p[6 + k] * (double)p[6 + k];
    if (!(qn2 > 0.0)) return;
    for (int k = 0; k < 3; ++k)
        if (fabs((double)p[3 + k]) > 30.0) return;
    g->valid = 1;
    for (int k = 0; k < 3; ++k) {
        g->mu[k] = (double)p[k];
        g->s[k] = exp((double)p[3 + k]);
    }
    g->qnorm = sqrt(qn2);
    for (int k = 0; k < 4; ++k) g->qn[k] = (double)p[6 + k] / g->qnorm;
    og_quat_to_R(g->qn, g->R);
    /* C = R diag(1/s^2) R^T */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += g->R[a][m] * g->R[b][m] / (g->s[m] * g->s[m]);
            g->C[a][b] = acc;
        }
    g->A = a_act ? og_sigmoid((double)p[10]) : (double)p[10];
    g->T = t_act ? og_sigmoid((double)p[11]) : (double)p[11];
    if (signal_mode == 0) {
        g->v = g->A;
        g->r = g->T;
    } else {
        g->v = g->A * g->T;
        g->r = 1.0;
    }
    /* Exact bounding box: d^2 >= |p-mu|^2 / s_max^2. Pairs of the ambiguity band have
     * d^2 <= sigma_t^2 + amb_tol sum_ab |C_ab d_a d_b| and sum_ab |C_ab d_a d_b| <=
     * 3 |p-mu|^2 / s_min^2 (|C_ab| <= 1 / s_min^2), so they lie within
     * |p-mu|^2 <= sigma_t^2 s_max^2 / (1 - 3 amb_tol s_max^2 / s_min^2); the radius is padded
     * by a further 1 % in d^2 and one voxel is added. A Gaussian so anisotropic that the
     * denominator is not clearly positive is not pruned. */
    double smax = g->s[0], smin = g->s[0];
    for (int k = 1; k < 3; ++k) {
        if (g->s[k] > smax) smax = g->s[k];
        if (g->s[k] < smin) smin = g->s[k];
    }
    double shrink = 1.0;
    if (amb_tol > 0.0) shrink = 1.0 - 3.0 * amb_tol * (smax * smax) / (smin * smin);
    int no_prune = !prune || shrink < 0.05;
    double rad = sqrt(sigma_t * sigma_t * (amb_tol > 0.0 ? 1.01 : 1.0) / shrink) * smax *
                     (1.0 + 1e-6) + 1e-9;
    for (int k = 0; k < 3; ++k) {
        if (no_prune) {
            g->lo[k] = 0;
            g->hi[k] = dims[k] - 1;
            continue;
        }
        double lo = ceil((g->mu[k] - rad - origin[k]) / h[k] - 0.5) - 1.0;
        double hi = floor((g->mu[k] + rad - origin[k]) / h[k] - 0.5) + 1.0;
        if (lo < 0.0) lo = 0.0;
        if (hi > (double)(dims[k] - 1)) hi = (double)(dims[k] - 1);
        if (lo > hi) {
            g->lo[k] = 1;
            g->hi[k] = 0;
        } else {
            g->lo[k] = (int)lo;
            g->hi[k] = (int)hi;
        }
    }
}

static og_gauss* og_activate_all(const double* params, int64_t N, const int32_t dims[3],
                                 const double h[3], const double origin[3], double sigma_t,
                                 double amb_tol, int signal_mode, int a_act, int t_act,
                                 int prune) {
    og_gauss* G = (og_gauss*)malloc(sizeof(og_gauss) * (size_t)(N > 0 ? N : 1));
    if (!G) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        og_activate(params + i * OG_NPARAM, dims, h, origin, sigma_t, amb_tol, signal_mode,
                    a_act, t_act, prune, &G[i]);
    return G;
}

static double og_d2(const og_gauss* g, const double d[3]) {
    double acc = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += d[a] * g->C[a][b] * d[b];
    return acc;
}

/* Sum of the absolute terms of the quadratic form: the scale of its rounding error. */
static double og_d2_abs(const og_gauss* g, const double d[3]) {
    double acc = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += fabs(d[a] * g->C[a][b] * d[b]);
    return acc;
}

/* ------------------------------------------------------------- Eq. 3-4 */

/* Ambiguous pairs recorded per voxel (the rest are only counted). */
#define OG_AMB_SLOTS 8

/*
 * Forward render of the voxels in crop = [x0,x1) x [y0,y1) x [z0,z1) (NULL: whole grid).
 * Outputs are crop-shaped, z-major, x fastest:
 *   S = sum_i v_i w_i, W = sum_i w_i, I = S / max(W, eps),
 *   amb = number of pairs with |d^2 - sigma_t^2| <= amb_tol * sum_ab |C_ab d_a d_b| (a
 *         rounded evaluation of d^2 may fall on either side of the truncation boundary),
 *   npair (optional) = number of contributing pairs (d^2 <= sigma_t^2) per voxel.
 * Optional outputs for validating a result that took its own decisions on ambiguous pairs:
 *   S_sure, W_sure = the sums over contributing pairs that are not ambiguous;
 *   for the first OG_AMB_SLOTS ambiguous pairs of a voxel (ascending Gaussian order), slot k
 *   of voxel j (index j * OG_AMB_SLOTS + k): amb_id = the Gaussian, amb_vw = v_i w_i and
 *   amb_w = w_i with w_i = exp(-d^2/2) r_i whichever side of the boundary d^2 lies,
 *   amb_rel = (d^2 - sigma_t^2) / sum_ab |C_ab d_a d_b| (<= 0: the pair contributes to S, W);
 *   cond_w = sum_i w_i sum_ab |C_ab d_a d_b| over contributing pairs (the rounding scale of
 *   the voxel's quadratic forms, weighted as W);
 *   cond_i = sum_i w_i |v_i - I| sum_ab |C_ab d_a d_b| over contributing pairs (the same scale
 *   weighted as the sensitivity of I to each weight, dI/dw_i = (v_i - I) / W).
 * Returns the number of invalid Gaussians.
 */
int64_t og_render(const double* params, int64_t N, const int32_t dims[3], const double h[3],
                  const double origin[3], const int32_t* crop, double sigma_t, double eps,
                  int signal_mode, int a_act, int t_act, double amb_tol, int prune, double* I,
                  double* W, double* S, int32_t* amb, int32_t* npair, double* S_sure,
                  double* W_sure, int32_t* amb_id, double* amb_vw, double* amb_w,
                  double* amb_rel, double* cond_w, double* cond_i) {
    int32_t c[6] = {0, dims[0], 0, dims[1], 0, dims[2]};
    if (crop) memcpy(c, crop, sizeof(c));
    const int64_t cx = c[1] - c[0], cy = c[3] - c[2], cz = c[5] - c[4];
    og_gauss* G = og_activate_all(params, N, dims, h, origin, sigma_t, amb_tol, signal_mode,
                                  a_act, t_act, prune);
    if (!G) return -1;
    int64_t n_invalid = 0;
    for (int64_t i = 0; i < N; ++i) n_invalid += G[i].valid ? 0 : 1;
    const double s2 = sigma_t * sigma_t;
    const int want_abs = amb_tol > 0.0 || cond_w != NULL;

    /* One z-slice per task: each voxel is owned by one thread and sums Gaussians in
     * ascending order, so the result does not depend on the thread count. */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t zz = 0; zz < cz; ++zz) {
        const int z = (int)(zz + c[4]);
        const int64_t zoff = zz * cy * cx;
        double* Sz = S + zoff;
        double* Wz = W + zoff;
        int32_t* Az = amb + zoff;
        int32_t* Nz = npair ? npair + zoff : NULL;
        for (int64_t k = 0; k < cy * cx; ++k) {
            Sz[k] = 0.0;
            Wz[k] = 0.0;
            Az[k] = 0;
            if (Nz) Nz[k] = 0;
            if (S_sure) S_sure[zoff + k] = 0.0;
            if (W_sure) W_sure[zoff + k] = 0.0;
            if (cond_w) cond_w[zoff + k] = 0.0;
        }
        const double pz = origin[2] + (z + 0.5) * h[2];
        for (int64_t i = 0; i < N; ++i) {
            const og_gauss* g = &G[i];
            if (!g->valid || z < g->lo[2] || z > g->hi[2]) continue;
            int ylo = g->lo[1] > c[2] ? g->lo[1] : c[2];
            int yhi = g->hi[1] < c[3] - 1 ? g->hi[1] : c[3] - 1;
            int xlo = g->lo[0] > c[0] ? g->lo[0] : c[0];
            int xhi = g->hi[0] < c[1] - 1 ? g->hi[0] : c[1] - 1;
            for (int y = ylo; y <= yhi; ++y) {
                const double py = origin[1] + (y + 0.5) * h[1];
                for (int x = xlo; x <= xhi; ++x) {
                    const double px = origin[0] + (x + 0.5) * h[0];
                    double d[3] = {px - g->mu[0], py - g->mu[1], pz - g->mu[2]};
                    double d2 = og_d2(g, d);
                    double dabs = want_abs ? og_d2_abs(g, d) : 0.0;
                    int64_t idx = (int64_t)(y - c[2]) * cx + (x - c[0]);
                    int is_amb = amb_tol > 0.0 && fabs(d2 - s2) <= amb_tol * dabs;
                    if (is_amb) {
                        int k = Az[idx];
                        if (amb_id && k < OG_AMB_SLOTS) {
                            int64_t sl = (zoff + idx) * OG_AMB_SLOTS + k;
                            double wk = exp(-0.5 * d2) * g->r;
                            amb_id[sl] = (int32_t)i;
                            amb_vw[sl] = g->v * wk;
                            amb_w[sl] = wk;
                            amb_rel[sl] = (d2 - s2) / dabs;
                        }
                        Az[idx] += 1;
                    }
                    if (d2 <= s2) {
                        double w = exp(-0.5 * d2) * g->r;
                        Sz[idx] += g->v * w;
                        Wz[idx] += w;
                        if (Nz) Nz[idx] += 1;
                        if (!is_amb && S_sure) S_sure[zoff + idx] += g->v * w;
                        if (!is_amb && W_sure) W_sure[zoff + idx] += w;
                        if (cond_w) cond_w[zoff + idx] += w * dabs;
                    }
                }
            }
        }
        for (int64_t k = 0; k < cy * cx; ++k) I[zoff + k] = Sz[k] / (Wz[k] > eps ? Wz[k] : eps);
        if (!cond_i) continue;
        /* second pass over the slice, now that I is known */
        for (int64_t k = 0; k < cy * cx; ++k) cond_i[zoff + k] = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            const og_gauss* g = &G[i];
            if (!g->valid || z < g->lo[2] || z > g->hi[2]) continue;
            int ylo = g->lo[1] > c[2] ? g->lo[1] : c[2];
            int yhi = g->hi[1] < c[3] - 1 ? g->hi[1] : c[3] - 1;
            int xlo = g->lo[0] > c[0] ? g->lo[0] : c[0];
            int xhi = g->hi[0] < c[1] - 1 ? g->hi[0] : c[1] - 1;
            for (int y = ylo; y <= yhi; ++y) {
                const double py = origin[1] + (y + 0.5) * h[1];
                for (int x = xlo; x <= xhi; ++x) {
                    const double px = origin[0] + (x + 0.5) * h[0];
                    double d[3] = {px - g->mu[0], py - g->mu[1], pz - g->mu[2]};
                    double d2 = og_d2(g, d);
                    if (!(d2 <= s2)) continue;
                    int64_t idx = (int64_t)(y - c[2]) * cx + (x - c[0]);
                    double w = exp(-0.5 * d2) * g->r;
                    cond_i[zoff + idx] += w * fabs(g->v - I[zoff + idx]) * og_d2_abs(g, d);
                }
            }
        }
    }
    free(G);
    return n_invalid;
}

/* ------------------------------------------------------------- Eq. 5-6 */

/*
 * Chain from the render-space gradient of one Gaussian -- dL/dmu, dL/dC (the full symmetric
 * 3 x 3 matrix of entry derivatives), dL/dv, dL/dr -- to its 12 raw parameters:
 * C = R D R^T with D = diag(s^-2), s = exp(log_s), R from the normalised quaternion;
 * (v, r) from (A, T) by the signal mode; A, T from (a, t) by their activations.
 * The map is linear in the render-space gradient.
 */
static void og_chain(const og_gauss* g, int signal_mode, int a_act, int t_act,
                     const double dmu[3], double dC[3][3], double dv, double dr, double* dp) {
    /* dL/dD_mm = (R^T G R)_mm, dL/dR = 2 G R D (G = dL/dC). */
    double RtGR[3];
    for (int m = 0; m < 3; ++m) {
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc += g->R[a][m] * dC[a][b] * g->R[b][m];
        RtGR[m] = acc;
    }
    for (int m = 0; m < 3; ++m) {
        /* D_mm = exp(-2 log_s_m)  =>  dD_mm/dlog_s_m = -2 D_mm */
        double Dmm = 1.0 / (g->s[m] * g->s[m]);
        dp[3 + m] = RtGR[m] * (-2.0 * Dmm);
    }
    double dR[3][3];
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < 3; ++m) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b) acc += dC[a][b] * g->R[b][m];
            dR[a][m] = 2.0 * acc / (g->s[m] * g->s[m]);
        }
    /* dR/dq for R(w, x, y, z) as in og_quat_to_R. */
    double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
    double dqn[4];
    dqn[0] = 2.0 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] +
                    x * dR[2][1]);
    dqn[1] = 2.0 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.0 * x * dR[1][1] -
                    w * dR[1][2] + z * dR[2][0] + w * dR[2][1] - 2.0 * x * dR[2][2]);
    dqn[2] = 2.0 * (-2.0 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] +
                    z * dR[1][2] - w * dR[2][0] + z * dR[2][1] - 2.0 * y * dR[2][2]);
    dqn[3] = 2.0 * (-2.0 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] -
                    2.0 * z * dR[1][1] + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    /* q_n = q / |q|  =>  dq = (dq_n - q_n (q_n . dq_n)) / |q| */
    double dot = 0.0;
    for (int k = 0; k < 4; ++k) dot += g->qn[k] * dqn[k];
    for (int k = 0; k < 4; ++k) dp[6 + k] = (dqn[k] - g->qn[k] * dot) / g->qnorm;
    for (int a = 0; a < 3; ++a) dp[a] = dmu[a];
    /* (v, r) -> (A, T) -> raw (a, t) */
    double dA, dT;
    if (signal_mode == 0) {
        dA = dv;
        dT = dr;
    } else {
        dA = dv * g->T;
        dT = dv * g->A;
    }
    dp[10] = a_act ? dA * g->A * (1.0 - g->A) : dA;
    dp[11] = t_act ? dT * g->T * (1.0 - g->T) : dT;
}

/*
 * Gradient of L with respect to the raw parameters, given dI = dL/dI on the crop
 * (crop-shaped; voxels outside the crop have dL/dI = 0). The forward pass over the crop is
 * recomputed here in FP64. Outputs:
 *   dparams [N,12]: dL/d(mu, log_s, q, a, t) of the raw parameters,
 *   dgeo [N,11] (optional): dL/d(mu(3), c_xx, c_yy, c_zz, c_xy, c_xz, c_yz, v, r), where c_ab
 *     is the single variable that sets both symmetric entries C_ab = C_ba of the inverse
 *     covariance (so an off-diagonal derivative is the sum of the two entry derivatives).
 *   dlo, dhi [N,12] (optional, need amb_tol > 0): bounds of every gradient a renderer can
 *     produce that decides each ambiguous pair (band of og_render) either way. At a voxel with
 *     n <= OG_AMB_SLOTS ambiguous pairs every include/exclude subset of them gives its own
 *     S, W, I and so its own contribution to each Gaussian at that voxel (zero for an
 *     ambiguous Gaussian left out); dlo and dhi add, per voxel, the smallest and the largest
 *     of those contributions (componentwise) to dparams in place of the FP64 decision's.
 *     Voxels are independent, so the sum of per-voxel ranges contains every combination.
 *   n_unenum (optional): voxels with dI != 0 and more than OG_AMB_SLOTS ambiguous pairs
 *     (their ranges are not formed; dparams uses the FP64 decisions there).
 */
int64_t og_render_grad(const double* params, int64_t N, const int32_t dims[3], const double h[3],
                       const double origin[3], const int32_t* crop, double sigma_t, double eps,
                       int signal_mode, int a_act, int t_act, double amb_tol, int prune,
                       const double* dI, double* dparams, double* dgeo, double* dlo,
                       double* dhi, int64_t* n_unenum) {
    int32_t c[6] = {0, dims[0], 0, dims[1], 0, dims[2]};
    if (crop) memcpy(c, crop, sizeof(c));
    const int64_t cx = c[1] - c[0], cy = c[3] - c[2], cz = c[5] - c[4];
    const int64_t nv = cx * cy * cz;
    const size_t nv1 = (size_t)(nv > 0 ? nv : 1);
    const int box = (dlo != NULL || dhi != NULL) && amb_tol > 0.0;
    const double tol_r = box ? amb_tol : 0.0;
    double* I = (double*)malloc(sizeof(double) * nv1);
    double* W = (double*)malloc(sizeof(double) * nv1);
    double* S = (double*)malloc(sizeof(double) * nv1);
    int32_t* amb = (int32_t*)malloc(sizeof(int32_t) * nv1);
    double *Ss = NULL, *Ws = NULL, *avw = NULL, *aw = NULL, *arel = NULL;
    int32_t* aid = NULL;
    if (box) {
        Ss = (double*)malloc(sizeof(double) * nv1);
        Ws = (double*)malloc(sizeof(double) * nv1);
        aid = (int32_t*)malloc(sizeof(int32_t) * nv1 * OG_AMB_SLOTS);
        avw = (double*)malloc(sizeof(double) * nv1 * OG_AMB_SLOTS);
        aw = (double*)malloc(sizeof(double) * nv1 * OG_AMB_SLOTS);
        arel = (double*)malloc(sizeof(double) * nv1 * OG_AMB_SLOTS);
        if (!Ss || !Ws || !aid || !avw || !aw || !arel) return -1;
    }
    if (!I || !W || !S || !amb) return -1;
    int64_t n_invalid = og_render(params, N, dims, h, origin, crop, sigma_t, eps, signal_mode,
                                  a_act, t_act, tol_r, prune, I, W, S, amb, NULL, Ss, Ws, aid,
                                  avw, aw, arel, NULL, NULL);
    og_gauss* G = og_activate_all(params, N, dims, h, origin, sigma_t, tol_r, signal_mode, a_act,
                                  t_act, prune);
    const double s2 = sigma_t * sigma_t;
    if (n_unenum) {
        int64_t cnt = 0;
        if (box)
            for (int64_t k = 0; k < nv; ++k) cnt += (amb[k] > OG_AMB_SLOTS && dI[k] != 0.0) ? 1 : 0;
        *n_unenum = cnt;
    }

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        const og_gauss* g = &G[i];
        double* dp = dparams + i * OG_NPARAM;
        for (int k = 0; k < OG_NPARAM; ++k) dp[k] = 0.0;
        if (dgeo)
            for (int k = 0; k < 11; ++k) dgeo[i * 11 + k] = 0.0;
        double lo_d[OG_NPARAM], hi_d[OG_NPARAM];
        for (int k = 0; k < OG_NPARAM; ++k) lo_d[k] = hi_d[k] = 0.0;
        if (!g->valid) {
            if (dlo) memset(dlo + i * OG_NPARAM, 0, sizeof(double) * OG_NPARAM);
            if (dhi) memset(dhi + i * OG_NPARAM, 0, sizeof(double) * OG_NPARAM);
            continue;
        }
        double dmu[3] = {0, 0, 0};
        double dC[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double dv = 0.0, dr = 0.0;
        int zlo = g->lo[2] > c[4] ? g->lo[2] : c[4];
        int zhi = g->hi[2] < c[5] - 1 ? g->hi[2] : c[5] - 1;
        int ylo = g->lo[1] > c[2] ? g->lo[1] : c[2];
        int yhi = g->hi[1] < c[3] - 1 ? g->hi[1] : c[3] - 1;
        int xlo = g->lo[0] > c[0] ? g->lo[0] : c[0];
        int xhi = g->hi[0] < c[1] - 1 ? g->hi[0] : c[1] - 1;
        for (int z = zlo; z <= zhi; ++z) {
            const double pz = origin[2] + (z + 0.5) * h[2];
            for (int y = ylo; y <= yhi; ++y) {
                const double py = origin[1] + (y + 0.5) * h[1];
                for (int x = xlo; x <= xhi; ++x) {
                    const double px = origin[0] + (x + 0.5) * h[0];
                    double d[3] = {px - g->mu[0], py - g->mu[1], pz - g->mu[2]};
                    double d2 = og_d2(g, d);
                    const int in = d2 <= s2;
                    const int is_amb = box && fabs(d2 - s2) <= amb_tol * og_d2_abs(g, d);
                    if (!in && !is_amb) continue;
                    int64_t idx = ((int64_t)(z - c[4]) * cy + (y - c[2])) * cx + (x - c[0]);
                    double gI = dI[idx];
                    if (gI == 0.0) continue;
                    double gk = exp(-0.5 * d2);   /* Gaussian kernel */
                    double w = gk * g->r;         /* Eq. 4 */
                    double Cd[3];
                    for (int a = 0; a < 3; ++a) {
                        Cd[a] = 0.0;
                        for (int b = 0; b < 3; ++b) Cd[a] += g->C[a][b] * d[b];
                    }
                    double coef = 0.0;
                    if (in) {
                        double Wp = W[idx];
                        /* dI/dw_i: (v_i - I)/W for W >= eps (Eq. 5), v_i/eps below the floor. */
                        double dIdw = (Wp > eps) ? (g->v - I[idx]) / Wp : g->v / eps;
                        double dIdv = w / (Wp > eps ? Wp : eps); /* Eq. 6 */
                        coef = gI * dIdw;
                        dv += gI * dIdv;
                        dr += coef * gk;
                        /* dw/dmu = w C d ; dw/dC_ab = -1/2 w d_a d_b */
                        for (int a = 0; a < 3; ++a) {
                            dmu[a] += coef * w * Cd[a];
                            for (int b = 0; b < 3; ++b) dC[a][b] += coef * w * (-0.5) * d[a] * d[b];
                        }
                    }
                    const int n = box ? amb[idx] : 0;
                    if (n == 0 || n > OG_AMB_SLOTS) continue;
                    /* Voxel with ambiguous pairs: this Gaussian's contribution under every
                     * include/exclude subset of them. It is coef_s JU + dvc_s JV with the
                     * chained unit vectors below. */
                    double uC[3][3], umu[3], zmu[3] = {0, 0, 0};
                    double zC[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                    for (int a = 0; a < 3; ++a) {
                        umu[a] = w * Cd[a];
                        for (int b = 0; b < 3; ++b) uC[a][b] = -0.5 * w * d[a] * d[b];
                    }
                    double JU[OG_NPARAM], JV[OG_NPARAM];
                    og_chain(g, signal_mode, a_act, t_act, umu, uC, 0.0, gk, JU);
                    og_chain(g, signal_mode, a_act, t_act, zmu, zC, 1.0, 0.0, JV);
                    const int64_t sl = idx * OG_AMB_SLOTS;
                    int j = -1;
                    if (is_amb)
                        for (int k = 0; k < n; ++k)
                            if (aid[sl + k] == (int32_t)i) j = k;
                    double vstar[OG_NPARAM];
                    {
                        double Wp = W[idx];
                        double dvc = in ? gI * w / (Wp > eps ? Wp : eps) : 0.0;
                        for (int k = 0; k < OG_NPARAM; ++k) vstar[k] = coef * JU[k] + dvc * JV[k];
                    }
                    double mn[OG_NPARAM], mx[OG_NPARAM];
                    for (int k = 0; k < OG_NPARAM; ++k) {
                        mn[k] = INFINITY;
                        mx[k] = -INFINITY;
                    }
                    for (int sig = 0; sig < (1 << n); ++sig) {
                        double val[OG_NPARAM];
                        if (j >= 0 && !((sig >> j) & 1)) {
                            for (int k = 0; k < OG_NPARAM; ++k) val[k] = 0.0;
                        } else {
                            double Wsig = Ws[idx], Ssig = Ss[idx];
                            for (int k = 0; k < n; ++k)
                                if ((sig >> k) & 1) {
                                    Wsig += aw[sl + k];
                                    Ssig += avw[sl + k];
                                }
                            double Wf = Wsig > eps ? Wsig : eps;
                            double Isig = Ssig / Wf;
                            double dIdw = (Wsig > eps) ? (g->v - Isig) / Wsig : g->v / eps;
                            double cs = gI * dIdw, dvc = gI * w / Wf;
                            for (int k = 0; k < OG_NPARAM; ++k) val[k] = cs * JU[k] + dvc * JV[k];
                        }
                        for (int k = 0; k < OG_NPARAM; ++k) {
                            if (val[k] < mn[k]) mn[k] = val[k];
                            if (val[k] > mx[k]) mx[k] = val[k];
                        }
                    }
                    for (int k = 0; k < OG_NPARAM; ++k) {
                        lo_d[k] += mn[k] - vstar[k];
                        hi_d[k] += mx[k] - vstar[k];
                    }
                }
            }
        }
        if (dgeo) {
            double* o = dgeo + i * 11;
            o[0] = dmu[0];
            o[1] = dmu[1];
            o[2] = dmu[2];
            o[3] = dC[0][0];
            o[4] = dC[1][1];
            o[5] = dC[2][2];
            o[6] = dC[0][1] + dC[1][0];
            o[7] = dC[0][2] + dC[2][0];
            o[8] = dC[1][2] + dC[2][1];
            o[9] = dv;
            o[10] = dr;
        }
        og_chain(g, signal_mode, a_act, t_act, dmu, dC, dv, dr, dp);
        if (dlo)
            for (int k = 0; k < OG_NPARAM; ++k) dlo[i * OG_NPARAM + k] = dp[k] + lo_d[k];
        if (dhi)
            for (int k = 0; k < OG_NPARAM; ++k) dhi[i * OG_NPARAM + k] = dp[k] + hi_d[k];
    }
    free(G);
    free(I);
    free(W);
    free(S);
    free(amb);
    free(Ss);
    free(Ws);
    free(aid);
    free(avw);
    free(aw);
    free(arel);
    return n_invalid;
}

/* ------------------------------------------------- FP32 brick-binning spec */

/*
 * Exponential in FP32 by Cody-Waite argument reduction and a degree-7 Taylor polynomial
 * (W. J. Cody and W. Waite, "Software Manual for the Elementary Functions", 1980):
 * exp(x) = 2^k exp(r), k = floor(x log2(e) + 1/2), r = x - k ln2 with ln2 split into a
 * 15-bit head (so k * head is exact) and a tail. Valid for |x| <= 30. Every operation is
 * one IEEE round-to-nearest operation, in the order written (compiled without contraction).
 */
static float og_exp_cw(float x) {
    const float L2E = 1.44269502f;            /* log2(e) rounded to float */
    const float LN2_HI = 0.693145751953125f;  /* ln 2, leading 15 bits */
    const float LN2_LO = 1.42860677e-6f;      /* ln 2 - LN2_HI */
    float kf = floorf(x * L2E + 0.5f);
    float r = (x - kf * LN2_HI) - kf * LN2_LO;
    float p = 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int k = (int)kf;
    uint32_t bits = (uint32_t)(k + 127) << 23;
    float two_k;
    memcpy(&two_k, &bits, sizeof(two_k));
    return p * two_k;
}

float og_exp_cw_public(float x) { return og_exp_cw(x); }

/*
 * Brick range of each Gaussian, decided in FP32 with the operation order below (the GPU
 * binning kernel follows the same specification, so brick lists compare bit-exactly):
 *   s_k = exp_cw(log_s_k);  n = sqrt(((q0 q0 + q1 q1) + q2 q2) + q3 q3);  qn = q / n
 *   products xx, yy, zz, xy, xz, yz, wx, wy, wz; rotation entries as in og_quat_to_R with
 *   the inner sums formed first and the factor 2 applied last; M_kj = R_kj s_j;
 *   Sigma_kk = (M_k0^2 + M_k1^2) + M_k2^2;  e_k = (sigma_t (1 + 2^-13)) sqrt(Sigma_kk)
 *   lo_f = (((mu_k - e_k) - o_k) / h_k - 1/2) - 2^-8,  hi_f = (((mu_k + e_k) - o_k) / h_k - 1/2) + 2^-8
 *   voxel range [ceil(lo_f), floor(hi_f)] clamped to [0, n_k - 1]; brick range = voxel / b_k.
 * out[g*7 + 0..5] = brick lo (x, y, z), brick hi (x, y, z); out[g*7+6] = 1 if the Gaussian
 * meets the grid, else 0 (then the range is empty). Invalid Gaussians (see header) are empty.
 */
void og_bins_fp32(const float* params, int64_t N, const int32_t dims[3], const float h[3],
                  const float origin[3], const int32_t brick[3], float sigma_t, int32_t* out) {
    const float ksig = sigma_t * 1.0001220703125f; /* sigma_t (1 + 2^-13) */
    for (int64_t g = 0; g < N; ++g) {
        const float* p = params + g * OG_NPARAM;
        int32_t* o = out + g * 7;
        for (int k = 0; k < 7; ++k) o[k] = 0;
        int ok = 1;
        for (int k = 0; k < OG_NPARAM; ++k)
            if (!isfinite(p[k])) ok = 0;
        for (int k = 0; k < 3; ++k)
            if (!(fabsf(p[3 + k]) <= 30.0f)) ok = 0;
        if (!ok) continue;
        float s[3];
        for (int k = 0; k < 3; ++k) s[k] = og_exp_cw(p[3 + k]);
        float nn = p[6] * p[6];
        nn = nn + p[7] * p[7];
        nn = nn + p[8] * p[8];
        nn = nn + p[9] * p[9];
        if (!(nn > 0.0f)) continue;
        float n = sqrtf(nn);
        float w = p[6] / n, x = p[7] / n, y = p[8] / n, z = p[9] / n;
        float xx = x * x, yy = y * y, zz = z * z;
        float xy = x * y, xz = x * z, yz = y * z;
        float wx = w * x, wy = w * y, wz = w * z;
        float R[3][3];
        R[0][0] = 1.0f - 2.0f * (yy + zz);
        R[0][1] = 2.0f * (xy - wz);
        R[0][2] = 2.0f * (xz + wy);
        R[1][0] = 2.0f * (xy + wz);
        R[1][1] = 1.0f - 2.0f * (xx + zz);
        R[1][2] = 2.0f * (yz - wx);
        R[2][0] = 2.0f * (xz - wy);
        R[2][1] = 2.0f * (yz + wx);
        R[2][2] = 1.0f - 2.0f * (xx + yy);
        int32_t lo[3], hi[3];
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
            float m0 = R[k][0] * s[0], m1 = R[k][1] * s[1], m2 = R[k][2] * s[2];
            float sig = m0 * m0;
            sig = sig + m1 * m1;
            sig = sig + m2 * m2;
            float e = ksig * sqrtf(sig);
            float lo_f = (((p[k] - e) - origin[k]) / h[k] - 0.5f) - 0.00390625f;
            float hi_f = (((p[k] + e) - origin[k]) / h[k] - 0.5f) + 0.00390625f;
            float nmax = (float)(dims[k] - 1);
            if (!(hi_f >= 0.0f) || !(lo_f <= nmax)) {
                inside = 0;
                break;
            }
            float lc = ceilf(lo_f), hc = floorf(hi_f);
            if (lc < 0.0f) lc = 0.0f;
            if (hc > nmax) hc = nmax;
            if (lc > hc) {
                inside = 0;
                break;
            }
            lo[k] = (int32_t)lc;
            hi[k] = (int32_t)hc;
        }
        if (!inside) continue;
        for (int k = 0; k < 3; ++k) {
            o[k] = lo[k] / brick[k];
            o[3 + k] = hi[k] / brick[k];
        }
        o[6] = 1;
    }
}

/* --------------------------------------------------------- thread control */

int og_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void og_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
