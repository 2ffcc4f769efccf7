// gs_common.cuh -- internal definitions shared by the CUDA translation units of libgsmri.
// Not part of the public ABI (include/gs_api.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_api.h"

namespace gs {

// ------------------------------------------------------------------ render record
// Per-Gaussian record (20 floats = 5 float4, 80 bytes) written by the preprocess kernel and
// staged into shared memory by the render kernels. Coordinates are voxel-index space: voxel
// (i, j, k) sits at (i, j, k). The mean mu' = (mu - o) / h - 1/2 is a float head plus a
// float tail (double-float arithmetic), stored negated, so d = (i + (-head)) + (-tail) =
// (i - head) - tail is accurate to one rounding of d even at large coordinates, and the
// (y, z) components of a row's offset are one packed pair of additions.
// The exponent q = (log2 e / 2) d^T Sigma'^{-1} d (Sigma' the covariance in voxel units, the
// Gaussian kernel is 2^-q) is stored by completing the square along x:
//     q(dx, dy, dz) = S(dy, dz) + (sa (dx - dx*(dy, dz)))^2,
//     S(dy, dz) = Pyy dy^2 + P2yz dy dz + Pzz dz^2   (the minimum of q along the x-row),
//     dx*(dy, dz) = c1 dy + c2 dz                      (where that minimum is reached);
// (P2yz, c2) and (Pyy, c1) sit side by side, so (Pyy dy + P2yz dz, c1 dy + c2 dz) is one
// packed multiply and one packed FMA.
// With M = sqrt(log2 e / 2) diag(1/s) R^T H (columns m0, m1, m2, the whitened steps of one
// voxel along x, y, z): sa = |m0| (the whitened length of one voxel step along x),
// c_j = -(m_j . m0) / |m0|^2, and S is the Gram form of m1, m2 with their components along m0
// removed. Every term of this form has the size of q itself
// for voxels inside the ellipsoid, so FP32 keeps its accuracy for strongly anisotropic
// Gaussians, and the value at a voxel depends only on the voxel and the Gaussian.
// rho4 bounds |M (p - c)| over a 4 x 4 x 4 voxel footprint around its centre c:
// |M d|^2 <= sum_jk |m_j . m_k| |d_j| |d_k| <= (3/2)^2 sum_jk |m_j . m_k| (culling).
// ext_k = 1.01 trunc_sigma sigma_k + 3/2 + 10^-3 (sigma_k the standard deviation along axis k
// in voxels) bounds the offset of a 4^3 footprint's centre from the mean when the truncated
// ellipsoid reaches one of its voxels (culling).
enum RecField : int {
    R_NMHX = 0, R_NMLX = 1,                 // -(mu' head, tail) along x
    R_NMHY = 2, R_NMHZ = 3,                 // -mu' head along y, z
    R_NMLY = 4, R_NMLZ = 5,                 // -mu' tail along y, z
    R_P2YZ = 6, R_C2 = 7,                   // dz coefficients of the row terms (S, dx*)
    R_PYY = 8, R_C1 = 9,                    // their dy coefficients
    R_PZZ = 10, R_SA = 11,                  // dz^2 coefficient of S; sa = |m0|
    R_EXTX = 12,                            // box half-extent along x (see below)
    R_RHO4 = 13,                            // footprint radius (see above)
    R_EXTY = 14, R_EXTZ = 15,               // box half-extents along y, z
    R_VR = 16,                              // v * r
    R_R = 17,                               // r
    R_V = 18,                               // v
    REC_FLOATS = 20
};
constexpr int REC_F4 = REC_FLOATS / 4;

// Render-space gradient accumulated per Gaussian by the adjoint kernel (12 floats):
// m1 = sum G d (3), m2 = sum G d d^T (xx, yy, zz, xy, xz, yz), dv, dr, pad, where
// G = dL/dw * w for every contributing pair (see gs_render.cu).
enum GradField : int {
    G_M1X = 0, G_M1Y = 1, G_M1Z = 2,
    G_M2XX = 3, G_M2YY = 4, G_M2ZZ = 5, G_M2XY = 6, G_M2XZ = 7, G_M2YZ = 8,
    G_DV = 9, G_DR = 10, G_PAD = 11,
    GRAD_FLOATS = 12
};

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = 0.7213475204444817f;  // (1/2) log2(e)

// Brick-range brange layout [N, 8].
enum BrangeField : int { B_LOX = 0, B_LOY, B_LOZ, B_HIX, B_HIY, B_HIZ, B_CNT, B_VALID };

// ------------------------------------------------------------------ sort constants
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024 values per block

constexpr int kL1Blocks = 1024;  // fixed block count of the L1 reduction (deterministic)

constexpr int64_t kMaxCapacity = (int64_t(1) << 31) - 4096;

// ------------------------------------------------------------------ workspace layout
struct Workspace {
    int32_t* keys0;
    int32_t* vals0;
    int32_t* keys1;
    int32_t* vals1;
    int32_t* gm_gid;
    int32_t* gm_cnt;
    int32_t* hist;           // digit counts / offsets of the radix passes: two buffers
    int32_t* hist1;          // of hist_len + 1, contiguous (hist1 = hist + hist_len + 1)
    long long* scan_tmp;     // block sums of the multi-level scan
    float* part;             // [capacity, 12] per-pair partial gradients (deterministic mode)
    float* gacc;             // [n_gauss, 12] render-space gradient per Gaussian
    float2* aip;             // [n_voxels] (alpha, alpha I'), alpha = dL/dI / max(W, eps)
    float* l1_part;          // [kL1Blocks]
    int64_t scan_tmp_len;
    int32_t n_tiles;
    size_t bytes;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int64_t scan_tmp_len_for(int64_t n) {
    // Space for every level of the recursive block-sum scan of n values.
    int64_t total = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n + 1;
    }
    return total + 8;
}

// Carve (or size, if base == nullptr) the workspace. Returns false on overflow.
inline bool carve_workspace(void* base, int64_t n_gauss, int64_t capacity, int32_t n_bricks,
                            int64_t n_voxels, bool deterministic, Workspace* ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return base ? static_cast<char*>(base) + o : nullptr;
    };
    const int64_t cap = capacity > 0 ? capacity : 1;
    const int64_t n = n_gauss > 0 ? n_gauss : 1;
    ws->n_tiles = static_cast<int32_t>((cap + kSortTile - 1) / kSortTile);
    int64_t hist_len = int64_t(kRadix) * ws->n_tiles;
    int64_t max_scan = hist_len;
    if (n + 1 > max_scan) max_scan = n + 1;
    if (int64_t(n_bricks) + 1 > max_scan) max_scan = int64_t(n_bricks) + 1;
    ws->scan_tmp_len = scan_tmp_len_for(max_scan);
    ws->keys0 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
    ws->vals0 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
    ws->keys1 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
    ws->vals1 = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
    ws->gm_gid = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
    ws->gm_cnt = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 1)));
    ws->hist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2 * (hist_len + 1)));
    ws->hist1 = ws->hist ? ws->hist + hist_len + 1 : nullptr;
    ws->scan_tmp = reinterpret_cast<long long*>(take(sizeof(long long) * ws->scan_tmp_len));
    ws->part = reinterpret_cast<float*>(
        take(deterministic ? sizeof(float) * GRAD_FLOATS * cap : 256));
    ws->gacc = reinterpret_cast<float*>(take(sizeof(float) * GRAD_FLOATS * n));
    ws->aip = reinterpret_cast<float2*>(take(sizeof(float2) * (n_voxels > 0 ? n_voxels : 1)));
    ws->l1_part = reinterpret_cast<float*>(take(sizeof(float) * kL1Blocks));
    ws->bytes = off;
    return true;
}

// Division by an invariant positive integer d (T. Granlund and P. L. Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, the unsigned case): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, every 32-bit unsigned n has
// n / d = (t + ((n - t) >> s1)) >> s2, t = mulhi(m, n), s1 = min(l, 1), s2 = max(l - 1, 0):
// one high multiply, a subtraction and three shifts in place of a division sequence.
struct FastDiv {
    unsigned m;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = static_cast<unsigned>(((1ull << 32) * ((1ull << l) - d)) / d + 1ull);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l - 1 > 0 ? l - 1 : 0;
    return f;
}

// ------------------------------------------------------------------ helpers
struct BrickGeom {
    int nbx, nby, nbz;
    int bx, by, bz;
};

inline BrickGeom brick_geom(const gs_grid* g, const gs_config* c) {
    BrickGeom b;
    b.bx = c->brick[0];
    b.by = c->brick[1];
    b.bz = c->brick[2];
    b.nbx = (g->nx + b.bx - 1) / b.bx;
    b.nby = (g->ny + b.by - 1) / b.by;
    b.nbz = (g->nz + b.bz - 1) / b.bz;
    return b;
}

// Validation shared by the entry points. Returns GS_OK or GS_ERR_INVALID_ARG.
gs_status validate_grid_cfg(const gs_grid* g, const gs_config* c);

// Launch counter (every kernel launch site is followed by last_launch_status()).
void note_launch();

// ------------------------------------------------------------------ launch chaining
// Programmatic dependent launch (sm_90 and later): every kernel is launched with programmatic
// stream serialisation, so its launch overlaps the end of its predecessor on the stream, and
// its first statement (pdl_enter) waits until the predecessor has completed and its memory is
// visible; nothing is read or written before the wait. Kernels do not trigger their
// successors early (the trigger is implicit as their blocks exit): an early trigger measured
// slower in graph replays of the fitting step.
template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     A&&... args) {
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = 1;
    (void)cudaLaunchKernelEx(&c, k, static_cast<A&&>(args)...);  // errors: cudaGetLastError
}

// Launch error check -> gs_status; counts the launch it follows.
inline gs_status last_launch_status() {
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// Optional check of a scan's grand total against a pair capacity: with npairs set, the total
// is stored there and GS_STATUS_CAPACITY is or-ed into *status when it exceeds capacity.
struct CapCheck {
    int64_t capacity = 0;
    int64_t* npairs = nullptr;
    int32_t* status = nullptr;
};

// Device-wide exclusive scan of int32 values (n <= kMaxCapacity + 1); 64-bit accumulation.
// out may alias in. If total != nullptr, the grand total is written there (device int64).
gs_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, long long* total,
                             long long* tmp, int64_t tmp_len, cudaStream_t stream,
                             CapCheck cc = CapCheck{});

// Parameter chain + render-space gradient -> raw-parameter gradient (gs_param.cu).
gs_status launch_param_bwd(const float* params, const float* gacc, int64_t n,
                           const gs_grid* grid, const gs_config* cfg, float* dparams,
                           cudaStream_t stream);

// L1 loss with optional sign gradient into dpred (gs_volume.cu).
gs_status resample_fwd_impl(const float* src, int32_t snz, int32_t sny, int32_t snx, float* dst,
                            int32_t dnz, int32_t dny, int32_t dnx, cudaStream_t st);
gs_status resample_adj_prep_impl(const float* dlr, int32_t lnz, int32_t lny, int32_t lnx,
                                 const float* I, const float* W, int32_t nz, int32_t ny, int32_t nx,
                                 float eps, float2* aip, cudaStream_t st);
gs_status launch_l1(const float* pred, const float* target, int64_t n, float* d_loss,
                    float* dpred, float* partials, cudaStream_t stream, int64_t n_norm = 0);
// Fitting-step tails (gs_param.cu): chain without Adam; Adam with an optional device skip flag.
gs_status launch_chain_grad(const float* params, float* grad, const float* part,
                            const float* gacc, const gs_bins* bins, int64_t n,
                            const gs_grid* grid, const gs_config* cfg, cudaStream_t st);
gs_status launch_adam(float* params, const float* grad, float* m, float* v, int64_t n_gauss,
                      const gs_adam* hp, int32_t* d_step, const int32_t* d_skip,
                      cudaStream_t st);

}  // namespace gs

// ------------------------------------------------------------------ device math
#ifdef __CUDACC__
namespace gs {

// FP32 exponential of the binning specification: Cody-Waite argument reduction with a
// 15-bit head of ln 2 and a degree-7 Taylor polynomial in Horner form (W. J. Cody and
// W. Waite, "Software Manual for the Elementary Functions", 1980). Every operation is one
// explicitly rounded IEEE operation in a fixed order (no contraction), so the result is the
// same on any IEEE-754 implementation that follows the same sequence. |x| <= 30.
__device__ __forceinline__ float exp_cw(float x) {
    const float L2E = 1.44269502f;
    const float LN2_HI = 0.693145751953125f;
    const float LN2_LO = 1.42860677e-6f;
    float kf = floorf(__fadd_rn(__fmul_rn(x, L2E), 0.5f));
    float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, LN2_HI)), __fmul_rn(kf, LN2_LO));
    float p = 1.0f / 5040.0f;
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 720.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 120.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 24.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f / 6.0f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    int k = static_cast<int>(kf);
    float two_k = __int_as_float((k + 127) << 23);
    return __fmul_rn(p, two_k);
}

// First statement of every kernel: wait for the preceding kernel on the stream (see
// launch_k; a no-op for a launch without a programmatic dependency).
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// 2^x on the special-function unit (ex2.approx, flush-to-zero).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Approximate square root (sqrt.approx, flush-to-zero); for bounds that carry a margin.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ unsigned fast_div(unsigned n, FastDiv f) {
    const unsigned t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}


}  // namespace gs
#endif
