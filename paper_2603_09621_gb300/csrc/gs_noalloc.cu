// gs_noalloc.cu -- L1 loss for callers that cannot allocate device memory.
//
// gs_l1_loss needs a caller-provided workspace for its per-block partial sums. Some callers
// cannot obtain one: a process that reserved its whole device memory budget at start-up and
// may not allocate afterwards, or a host program that embeds this library without any GPU
// allocator of its own. gs_l1_loss_static gives them the same loss with the partial sums in a
// fixed array compiled into this library instead.
//
// The array below is file-scope device memory: every GPU that loads the library holds it
// until the process exits. Its host-side name is only a stand-in for the symbol, so host code
// obtains the device address once per device with cudaGetSymbolAddress (with that device
// current) and passes the pointer to the kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int kStaticBlocks = 4096;        // partial sums held in the static array
constexpr int kStaticChunk = 8192;         // elements reduced by one block
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

static_assert(int64_t(kStaticBlocks) * kStaticChunk == GS_L1_STATIC_MAX_N,
              "the header's maximum must match the static scratch");

__device__ __align__(256) float g_l1_scratch[kStaticBlocks];

std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Each block sums |pred - target| over one chunk in a fixed order and writes one partial;
// optionally writes sign(pred - target) / n.
__global__ void __launch_bounds__(kStaticThreads) k_l1_static_partial(
    const float* __restrict__ pred, const float* __restrict__ target, int64_t n, float inv_n,
    float* __restrict__ dpred, float* __restrict__ partials) {
    pdl_enter();
    __shared__ float sm[kStaticThreads];
    const int64_t base = int64_t(blockIdx.x) * kStaticChunk;
    float acc = 0.f;
    for (int k = threadIdx.x; k < kStaticChunk; k += kStaticThreads) {
        const int64_t i = base + k;
        if (i < n) {
            const float d = pred[i] - target[i];
            acc += fabsf(d);
            if (dpred) dpred[i] = (d > 0.f) ? inv_n : ((d < 0.f) ? -inv_n : 0.f);
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kStaticThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

// One block adds the used partials [0, nblocks) in a fixed order.
__global__ void __launch_bounds__(1024) k_l1_static_final(const float* __restrict__ partials,
                                                          int nblocks, float inv_n,
                                                          float* __restrict__ loss) {
    pdl_enter();
    __shared__ float sm[1024];
    float acc = 0.f;
    for (int i = threadIdx.x; i < nblocks; i += 1024) acc += partials[i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sm[0] * inv_n;
}

// Device address of the static scratch on the current device, looked up once per device and
// kept for the life of the process: it is valid for the context that was current at the first
// call (a context destroyed and rebuilt later reloads the module at another address).
gs_status scratch_for_current_device(float** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_l1_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_l1_loss_static(const float* pred, const float* target, int64_t n,
                                       float* d_loss, float* dpred, gs_stream stream) {
    using namespace gs;
    if (!pred || !target || !d_loss || n <= 0) return GS_ERR_INVALID_ARG;
    if (n > GS_L1_STATIC_MAX_N) return GS_ERR_INVALID_ARG;
    float* scratch = nullptr;
    gs_status s = scratch_for_current_device(&scratch);
    if (s != GS_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nblocks = static_cast<int>((n + kStaticChunk - 1) / kStaticChunk);
    const float inv_n = 1.0f / float(n);
    launch_k(k_l1_static_partial, dim3(nblocks), dim3(kStaticThreads), 0, st, pred, target, n,
        inv_n, dpred, scratch);
    s = last_launch_status();
    if (s != GS_OK) return s;
    launch_k(k_l1_static_final, dim3(1), dim3(1024), 0, st, scratch, nblocks, inv_n, d_loss);
    return last_launch_status();
}
