/*
 * gs_api.h -- C ABI of the GB300 (sm_103a) Gaussian volume rasteriser for zero-shot MRI
 * super-resolution ("Physics-Driven 3D Gaussian Rendering for Zero-Shot MRI
 * Super-Resolution", Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" are CUDA device memory owned by the caller; "host" pointers
 *     are ordinary host memory. The library allocates no memory: scratch comes from a
 *     caller-provided workspace whose size gs_workspace_bytes() reports.
 *   - Every compute call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless its comment says "synchronous". Argument errors are detected on
 *     the host before any launch and returned at once; CUDA launch errors map to
 *     GS_ERR_CUDA. Conditions found on the device (pair capacity exceeded, invalid Gaussians)
 *     are written to the device status word of the bins (see gs_status_read).
 *   - Raw Gaussian parameters are float32 [N, 12] row-major (48 bytes per Gaussian), Sec. 3.1
 *     (position 3, covariance 7 = log-scale 3 + quaternion 4, amplitude 1, relaxation 1):
 *        [mu_x, mu_y, mu_z, log_s_x, log_s_y, log_s_z, q_w, q_x, q_y, q_z, a, t]
 *     Sigma = R(q/|q|) diag(exp(2 log_s)) R^T; A = act_a(a); T = act_t(t) (identity or
 *     sigmoid). Signal mode 0 renders v = A with relaxation factor r = T (Eq. 3-4); mode 1
 *     renders v = A T with r = 1. Gaussians with a non-finite value, a zero quaternion or a
 *     log-scale outside [-30, 30] are invalid: they contribute nothing and raise
 *     GS_STATUS_NONFINITE in the device status word.
 *   - Volumes are float32 [nz, ny, nx] (x fastest). Voxel (i, j, k) has centre
 *     origin + (i + 1/2, j + 1/2, k + 1/2) * h (world units, mm).
 *   - The forward render is I(p) = sum_i v_i w_i(p) / max(sum_i w_i(p), eps) with
 *     w_i(p) = r_i exp(-d^2/2), d^2 = (p - mu_i)^T Sigma_i^{-1} (p - mu_i), and a pair
 *     contributes only when d^2 <= trunc_sigma^2 (Eq. 3-4; the 3-sigma truncation of
 *     Sec. 3.3). Per voxel the sum runs over Gaussians in ascending id order, so results are
 *     deterministic and independent of the brick shape.
 */
#ifndef GS_API_H
#define GS_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the CUDA runtime's stream handle type). */
typedef struct CUstream_st* gs_stream;

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1, /* a null pointer, a bad size or an unsupported option */
    GS_ERR_CAPACITY = -2,    /* the pair list needs more than the bins' capacity */
    GS_ERR_WORKSPACE = -3,   /* workspace smaller than gs_workspace_bytes() */
    GS_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    GS_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    GS_ERR_NONFINITE = -6    /* invalid Gaussians (NaN/Inf, zero quaternion, |log_s| > 30) */
} gs_status;

/* Bits of the device status word written by the kernels. */
#define GS_STATUS_CAPACITY 1
#define GS_STATUS_NONFINITE 2

/* Voxel grid: nx, ny, nz voxels; spacing h (x, y, z) and origin in world units. */
typedef struct {
    int32_t nx, ny, nz;
    float h[3];
    float origin[3];
} gs_grid;

/* Rendering options.
 *   brick: brick shape in voxels (x, y, z): x and y in {4, 8, 16}, z a multiple of 4,
 *          y * z <= 64 and x * y * z <= 512. Sec. 3.3 uses 8 x 8 x 4; the default is 8 x 8 x 8.
 *          Output does not depend on it.
 *   trunc_sigma: Mahalanobis truncation radius (3.0: the 3-sigma ellipsoids of Sec. 3.3).
 *   eps: floor of the weight sum in the normalisation of Eq. 3 (the paper gives none).
 *   deterministic: 1 = the backward pass reduces per-Gaussian gradients in a fixed order
 *                  (bit-reproducible, no floating-point atomics); 0 = one float atomic
 *                  per (brick, Gaussian, value).
 *   signal_mode: 0 (v = A, r = T) or 1 (v = A T, r = 1).
 *   a_act, t_act: 0 = identity, 1 = sigmoid for A and T. */
typedef struct {
    int32_t brick[3];
    float trunc_sigma;
    float eps;
    int32_t deterministic;
    int32_t signal_mode;
    int32_t a_act;
    int32_t t_act;
} gs_config;

/* Brick bins of one Gaussian cloud on one grid (Sec. 3.3: "for each brick b we identify
 * intersecting Gaussians G_b"). All arrays are device memory carved from one caller-owned
 * arena by gs_bins_bind(). Brick b = (bx, by, bz) has linear index (bz * nby + by) * nbx + bx.
 *   brick_off [n_bricks + 1]: pairs of brick b are [brick_off[b], brick_off[b+1]).
 *   pair_gid  [capacity]: Gaussian id of each pair, brick-major, ascending inside a brick.
 *   pair_gmj  [capacity]: position of each brick-major pair in the Gaussian-major order.
 *   pair_brick [capacity]: linear brick index of each brick-major pair.
 *   gm_off    [n_gauss + 1]: Gaussian-major pair offsets (bricks of one Gaussian ascend).
 *   rec       [n_gauss, 20] float: per-Gaussian render record (internal layout).
 *   brange    [n_gauss, 8] int32: brick range lo (x, y, z), hi (x, y, z), pair count, valid.
 *   d_npairs  device int64: pairs needed by the last gs_bin_bricks call.
 *   d_status  device int32: GS_STATUS_* bits of the last gs_bin_bricks call. */
typedef struct {
    int64_t n_gauss;
    int64_t capacity;
    int32_t n_bricks;
    int32_t nbx, nby, nbz;
    int32_t* brick_off;
    int32_t* pair_gid;
    int32_t* pair_gmj;
    int32_t* pair_brick;
    int32_t* gm_off;
    float* rec;
    int32_t* brange;
    int64_t* d_npairs;
    int32_t* d_status;
} gs_bins;

/* Adam hyper-parameters (bias-corrected Adam, Kingma & Ba 2015; the paper names no
 * optimiser). Learning rates per parameter group: means, log-scales, quaternion, a, t. */
typedef struct {
    float lr_mu, lr_scale, lr_rot, lr_a, lr_t;
    double beta1, beta2, eps; /* double, so 1 - beta is exact for decimal inputs like 0.999 */
} gs_adam;

/* Size in bytes of the device arena that gs_bins_bind() carves; 0 on invalid arguments.
 * capacity is the maximum number of (brick, Gaussian) pairs, at most 2^31 - 4096. */
size_t gs_bins_bytes(int64_t n_gauss, int64_t capacity, const gs_grid* grid,
                     const gs_config* cfg);

/* Fill `out` with pointers into `arena` (device, at least gs_bins_bytes() bytes, 256-byte
 * aligned). Host-only; nothing is launched. */
gs_status gs_bins_bind(void* arena, size_t arena_bytes, int64_t n_gauss, int64_t capacity,
                       const gs_grid* grid, const gs_config* cfg, gs_bins* out);

/* Scratch bytes needed by gs_bin_bricks, gs_render_bwd, gs_l1_loss and gs_fit_step for this
 * problem size (one workspace serves all of them; calls sharing it must not overlap). */
size_t gs_workspace_bytes(int64_t n_gauss, int64_t capacity, const gs_grid* grid,
                          const gs_config* cfg);

/* Sec. 3.1 / Eq. 2: T = (1 - exp(-TR/T1)) exp(-TE/T2) elementwise.
 * T1, T2, T_out: device float [n]. TR, TE in the same unit as T1, T2. */
gs_status gs_signal_proxy(const float* T1, const float* T2, int64_t n, float TR, float TE,
                          float* T_out, gs_stream stream);

/* Sec. 3.3 brick intersection and binning: activate every Gaussian, bound its truncated
 * ellipsoid by its axis-aligned box (half-extent trunc_sigma sqrt(Sigma_kk), padded by
 * 2^-13 relative and 2^-8 voxel), and list it in every brick the box meets (count, exclusive
 * scan, stable radix scatter: deterministic, bit-exact). The brick-range arithmetic is a
 * fixed FP32 operation sequence (documented in the oracle's binning specification).
 * params: device float [n_gauss, 12]. bins: bound to this n_gauss, grid and cfg.
 * ws: device workspace of ws_bytes >= gs_workspace_bytes().
 * If the pairs exceed bins->capacity, *d_npairs holds the count needed, the status word
 * gets GS_STATUS_CAPACITY, and the brick lists are left empty (no later kernel reads past
 * the capacity). */
gs_status gs_bin_bricks(const float* params, const gs_grid* grid, const gs_config* cfg,
                        gs_bins* bins, void* ws, size_t ws_bytes, gs_stream stream);

/* Eq. 3-4 forward render (Sec. 3.3: one CTA per brick, the brick's Gaussians staged through
 * shared memory). Writes I = S / max(W, eps) and W = sum_i w_i for every voxel.
 * I, W: device float [nz, ny, nx]. d_stats: device uint64 [2] or NULL; when given, adds the
 * number of pairs with d^2 <= trunc_sigma^2 (stats[0]) and of pairs evaluated (stats[1]). */
gs_status gs_render_fwd(const gs_bins* bins, const gs_grid* grid, const gs_config* cfg,
                        float* I, float* W, unsigned long long* d_stats, gs_stream stream);

/* Eq. 5-6 adjoint of the forward render and the chain to the raw parameters.
 * params: device float [n_gauss, 12] (the ones binned); I, W: the forward outputs;
 * dI: device float [nz, ny, nx], dL/dI; dparams: device float [n_gauss, 12], overwritten
 * with dL/d(raw params). ws: workspace (>= gs_workspace_bytes()). */
gs_status gs_render_bwd(const float* params, const gs_bins* bins, const gs_grid* grid,
                        const gs_config* cfg, const float* I, const float* W, const float* dI,
                        float* dparams, void* ws, size_t ws_bytes, gs_stream stream);

/* Slice-profile forward model (not in the paper; the fitting workload's reading): box
 * average of s consecutive slices along z. hr: device [nz, ny, nx]; lr: device
 * [nz / s, ny, nx] (integer division; trailing slices are dropped). */
gs_status gs_downsample_fwd(const float* hr, int32_t nz, int32_t ny, int32_t nx, int32_t s,
                            float* lr, gs_stream stream);

/* Adjoint of gs_downsample_fwd: dhr[z] = dlr[z / s] / s for z < s (nz / s), else 0.
 * dlr: device [nz / s, ny, nx]; dhr: device [nz, ny, nx]. */
gs_status gs_downsample_bwd(const float* dlr, int32_t nz, int32_t ny, int32_t nx, int32_t s,
                            float* dhr, gs_stream stream);

/* Trilinear resize with half-pixel centres (Sec. 4.1 makes the LR inputs by trilinear
 * downsampling; the convention is this library's reading): along each axis, destination
 * sample j reads the source at continuous index c_j = (n_src / n_dst)(j + 1/2) - 1/2 (raised
 * to 0 where negative), i.e. samples floor(c_j) and min(floor(c_j) + 1, n_src - 1) with
 * linear weights; c_j is formed in FP32, one rounding per operation. Any sizes (down- or
 * upsampling, per axis). src: device [snz, sny, snx]; dst: device [dnz, dny, dnx].
 * Every size must be in [1, 2^23). */
gs_status gs_resample_fwd(const float* src, int32_t snz, int32_t sny, int32_t snx, float* dst,
                          int32_t dnz, int32_t dny, int32_t dnx, gs_stream stream);

/* Adjoint (transpose) of gs_resample_fwd: dsrc [snz, sny, snx] = R^T ddst [dnz, dny, dnx],
 * each source voxel gathering the destination samples that read it in a fixed order
 * (deterministic, no atomics). dsrc is overwritten. */
gs_status gs_resample_bwd(const float* ddst, int32_t dnz, int32_t dny, int32_t dnx, float* dsrc,
                          int32_t snz, int32_t sny, int32_t snx, gs_stream stream);

/* Mean absolute error over n values, reduced in a fixed order (deterministic).
 * pred, target: device float [n]; d_loss: device float scalar; dpred: device float [n] or
 * NULL, receives sign(pred - target) / n (sign(0) = 0). ws: workspace. */
gs_status gs_l1_loss(const float* pred, const float* target, int64_t n, float* d_loss,
                     float* dpred, void* ws, size_t ws_bytes, gs_stream stream);

/* Largest n accepted by gs_l1_loss_static (4096 partial sums of 8192 values each). */
#define GS_L1_STATIC_MAX_N 33554432LL

/* Mean absolute error like gs_l1_loss, for callers that cannot allocate device memory (the
 * paper has no counterpart; it is a property of this library's interface). A process that
 * reserved its whole device budget at start-up, or a host program that embeds this library
 * without a GPU allocator, cannot provide gs_l1_loss's workspace; this entry point keeps the
 * per-block partial sums in a 16 KB array compiled into the library instead (every GPU that
 * loads the library holds it until the process exits) and calls no allocation routine.
 * pred, target: device float [n]; d_loss: device float scalar; dpred: device float [n] or
 * NULL (sign(pred - target) / n). n must be in [1, GS_L1_STATIC_MAX_N]; larger n returns
 * GS_ERR_INVALID_ARG before any launch. The first call on a device looks up the array's
 * device address (with that device current); make that first call before any stream
 * capture. The address found then belongs to the context current at that first call; after
 * that context is destroyed (cudaDeviceReset, or a context rebuilt after an error) the
 * process must not call this entry point again. All calls in one process share the one array
 * (each process has its own copy) and it keeps the last call's partial sums; every call
 * overwrites the entries it reads, so nothing needs clearing, but calls of one process that
 * overlap on the GPU (from concurrent streams or threads on the same device) race on it:
 * issue them in order on one stream. */
gs_status gs_l1_loss_static(const float* pred, const float* target, int64_t n, float* d_loss,
                            float* dpred, gs_stream stream);

/* One bias-corrected Adam update of params [n_gauss, 12] from grad, with moments m, v
 * (device float [n_gauss, 12], zero before the first step). d_step: device int32, the
 * number of steps taken so far; incremented on the device (graph-capturable). */
gs_status gs_adam_step(float* params, const float* grad, float* m, float* v, int64_t n_gauss,
                       const gs_adam* hp, int32_t* d_step, gs_stream stream);

/* gs_init_lattice for an LR volume made by gs_resample_fwd from the HR grid: lr is device
 * [lnz, lny, lnx] on the grid with the HR origin and field of view, spacing L_a / ln_a. */
gs_status gs_init_lattice_lr(const float* lr, int32_t lnz, int32_t lny, int32_t lnx,
                             const gs_grid* hr_grid, int32_t nlx, int32_t nly, int32_t nlz,
                             int32_t t_act, float t_init, float* params, gs_stream stream);

/* Initial cloud from the LR volume (Fig. 1 caption: Gaussians are initialised from the
 * coordinates of the LR volume; details are this library's reading): an axis lattice of
 * nl = (nlx, nly, nlz) points with centres origin + (i + 1/2) L / nl, amplitude = trilinear
 * sample of lr (edge-clamped) at the centre, T = t_init (through t_act), log-scale =
 * log(L_a / (2 nl_a)), identity rotation. lr: device [hr_nz / s, ny, nx] on the grid with
 * spacing (h_x, h_y, s h_z); params: device float [nlx nly nlz, 12] (x fastest). */
gs_status gs_init_lattice(const float* lr, const gs_grid* hr_grid, int32_t s, int32_t nlx,
                          int32_t nly, int32_t nlz, int32_t t_act, float t_init, float* params,
                          gs_stream stream);

/* LR forward models of the fitting step: the z box slice profile of factor s
 * (gs_downsample_fwd), or the trilinear resize to (lr_nz, lr_ny, lr_nx) (gs_resample_fwd). */
#define GS_LR_ZBOX 0
#define GS_LR_TRILINEAR 1

/* One zero-shot fitting iteration (all device work, no host synchronisation; the step can
 * be captured in a CUDA graph): bin, forward render, LR forward model (lr_model), L1 loss
 * against lr_target, its adjoint, adjoint render, Adam. Every pointer is device memory:
 *   params, grad, m, v [n_gauss, 12]; I, W [nz, ny, nx]; lr_pred and lr_target of the LR
 *   shape: [nz / s, ny, nx] for GS_LR_ZBOX, [lr_nz, lr_ny, lr_nx] for GS_LR_TRILINEAR (after
 *   the step lr_pred holds dL/dLR); d_loss float scalar (the loss of this
 *   step's forward pass); d_step int32 (Adam step counter); bins bound for n_gauss; ws
 *   workspace. On return grad holds dL/d(params) of this step.
 *   If this step's binning overflows the bins' capacity, the step is a no-op: params, m, v
 *   and d_step keep their values (grad is zeroed) and the status word carries
 *   GS_STATUS_CAPACITY, so a caller can grow the bins and repeat the step with the same
 *   result as if the capacity had sufficed.
 * phase_events: NULL, or GS_FIT_PHASES cudaEvent_t handles (host) recorded on `stream` at
 *   the start and after each phase: [0] start, [1] binning, [2] forward render, [3] slice
 *   profile + L1 + adjoint profile (with the adjoint's per-voxel factors), [4] adjoint render
 *   kernel, [5] gradient reduction + parameter chain + Adam, [6] end (same as [5]).
 *   n_phase_events is 0 or GS_FIT_PHASES. */
#define GS_FIT_PHASES 7
typedef struct {
    gs_grid grid;
    gs_config cfg;
    gs_adam adam;
    int64_t n_gauss;
    int32_t s;
    float* params;
    float* grad;
    float* m;
    float* v;
    int32_t* d_step;
    gs_bins bins;
    float* I;
    float* W;
    float* lr_pred;
    const float* lr_target;
    float* d_loss;
    void* ws;
    size_t ws_bytes;
    void* const* phase_events;
    int32_t n_phase_events;
    int32_t lr_model;                 /* GS_LR_ZBOX (uses s) or GS_LR_TRILINEAR */
    int32_t lr_nx, lr_ny, lr_nz;      /* LR shape of GS_LR_TRILINEAR, each in [1, 2^23) */
} gs_fit_state;

gs_status gs_fit_step(gs_fit_state* st, gs_stream stream);

/* gs_fit_step split in two around its gradient, for one volume fitted by several processes,
 * each owning a z-slab of it (the paper fits one scan on one device; the loss of Sec. 3.3 is
 * a mean over LR voxels and its gradient (Eq. 5-6) a sum over voxels, so the slabs' gradients
 * add up to the whole volume's, and one sum-reduction of grad between the two calls gives
 * every process the same update).
 * gs_fit_grad: bin, render, LR forward model, L1, adjoints and the chain to the raw
 *   parameters, as gs_fit_step, without Adam: on return grad holds dL/d(params) of this
 *   state's volume (zero if the step's binning overflowed the bins' capacity; the status word
 *   then carries GS_STATUS_CAPACITY and *bins.d_npairs exceeds bins.capacity). The L1
 *   mean is taken over n_lr_total LR values when n_lr_total > 0 (the whole volume's count, so
 *   that d_loss and grad are this slab's share of the whole volume's loss and gradient), over
 *   this state's own LR values when it is 0; n_lr_total < 0 is invalid. The step counter is
 *   not changed. Phase events as gs_fit_step ([5] follows the chain).
 * gs_fit_apply: one bias-corrected Adam update of params, m, v from grad with st->adam, and
 *   the step counter incremented, unless d_skip (device int32, or NULL) holds a nonzero value:
 *   then nothing changes (pass the OR over all processes of "my binning overflowed" so that an
 *   overflow anywhere makes the step a no-op everywhere, as in gs_fit_step).
 * With one process, gs_fit_grad(st, 0) followed by gs_fit_apply(st, overflowed) gives
 * gs_fit_step's result bit for bit. */
/* gs_fit_step with the step's inputs and its loss in host memory (the same step, for callers
 * whose data lives on the host): copies h_params (host float [n_gauss, 12], or NULL to keep
 * st->params) and h_lr_target (host float of the LR shape, or NULL to keep st->lr_target) to
 * the state's device buffers, runs gs_fit_step, and copies the step's loss to *h_loss (host
 * float, or NULL), asynchronously with respect to the host (one cudaMemcpyAsync per buffer;
 * page-locked host memory makes the copies asynchronous). The LR target is copied on a side
 * stream that the library creates once per device (with two events) at the first such call
 * on it, overlapped with the step's binning and forward render; the step waits for it before
 * its LR model, and the copy itself waits for the work issued on `stream` before the call.
 * st->lr_target must be writable device memory when h_lr_target is given. The caller
 * synchronises `stream` before reading *h_loss. */
gs_status gs_fit_step_host(gs_fit_state* st, const float* h_params, const float* h_lr_target,
                           float* h_loss, gs_stream stream);

gs_status gs_fit_grad(gs_fit_state* st, int64_t n_lr_total, gs_stream stream);
gs_status gs_fit_apply(gs_fit_state* st, const int32_t* d_skip, gs_stream stream);

/* Synchronous: waits for `stream`, then copies the device status word to *h_status and
 * returns GS_ERR_CAPACITY or GS_ERR_NONFINITE if the matching bit is set, else GS_OK. */
gs_status gs_status_read(const int32_t* d_status, int32_t* h_status, gs_stream stream);

/* Static string naming a status code. */
const char* gs_status_string(gs_status s);

/* Number of kernels this library has launched in the calling process (host counter). */
unsigned long long gs_launch_count(void);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_API_H */
