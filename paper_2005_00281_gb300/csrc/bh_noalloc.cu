// bh_residual_misfit_noalloc: the data residual and misfit of
// bh_residual_misfit for callers that cannot allocate device memory.
//
// Why: bh_residual_misfit needs a bh_model, and building one calls
// cudaMalloc.  Some callers may not allocate at all: processes whose device
// memory is fixed up front by another allocator (a framework's pool, or a
// budget set at start-up), and serving paths that forbid allocation after
// warm-up because an allocation can synchronise the device.
// This entry point takes only the caller's buffers and keeps its FP64
// partial sums in a file-scope __device__ array instead.
//
// The scratch array is shared by every call in the process and keeps the
// previous call's contents; every slot a call reads is written earlier in
// the same call, so nothing has to be cleared.  Two calls whose kernels run
// at the same time on the GPU (different streams, no ordering between them)
// race on that array and may return wrong J values.
#include "bh.h"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

void bh_internal_set_thread_error(const std::string& msg);

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr size_t kPerBlock = (size_t)kThreads * kPerThread;  // 4096 samples per block
constexpr int kMaxBlocks = BH_NOALLOC_MAX_SAMPLES / (int)kPerBlock;
static_assert((size_t)kMaxBlocks * kPerBlock == BH_NOALLOC_MAX_SAMPLES, "limit");

// kMaxBlocks FP64 partial sums, then the final J (64 KB + 8 B; every GPU that
// loads the library holds it until the process exits)
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 1];

// pass 1: residual and per-block sum of squares, fixed order inside a block
// resid may alias mod (each element is read, then written, by one thread),
// so neither carries __restrict__
__global__ void __launch_bounds__(kThreads) k_misfit_partial(size_t n, const float* mod,
                                                             const float* __restrict__ obs,
                                                             float* resid, double* scratch)
{
    __shared__ double sh[kThreads];
    const size_t base = (size_t)blockIdx.x * kPerBlock;
    double s = 0.0;
    for (int q = 0; q < kPerThread; ++q) {
        size_t k = base + (size_t)q * kThreads + threadIdx.x;
        if (k < n) {
            float d = mod[k] - obs[k];
            resid[k] = d;
            s += (double)d * (double)d;
        }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[blockIdx.x] = sh[0];
}

// pass 2: J = 1/2 sum of the partials, fixed order
__global__ void __launch_bounds__(1024) k_misfit_total(int nblocks, double* scratch)
{
    __shared__ double sh[1024];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[kMaxBlocks] = 0.5 * sh[0];
}

// Device address of the scratch array, looked up once per device with that
// device current.  The host-side name g_noalloc_scratch is not a device
// address and must never be passed to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

bh_status scratch_for_current_device(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        bh_internal_set_thread_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return BH_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        bh_internal_set_thread_error("device ordinal out of range");
        return BH_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            bh_internal_set_thread_error(std::string("cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
            return BH_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return BH_OK;
}

}  // namespace

extern "C" bh_status bh_residual_misfit_noalloc(const float* seis_mod, const float* seis_obs,
                                                float* resid, size_t n, double* J, void* stream)
{
    if (!seis_mod || !seis_obs || !resid || !J) {
        bh_internal_set_thread_error("bh_residual_misfit_noalloc: NULL argument");
        return BH_ERR_INVALID_ARG;
    }
    if (n > (size_t)BH_NOALLOC_MAX_SAMPLES) {
        bh_internal_set_thread_error(
            "bh_residual_misfit_noalloc: " + std::to_string(n) +
            " samples exceed the limit of " + std::to_string(BH_NOALLOC_MAX_SAMPLES) +
            " (BH_NOALLOC_MAX_SAMPLES); use bh_residual_misfit");
        return BH_ERR_INVALID_ARG;
    }
    if (n == 0) {
        *J = 0.0;
        return BH_OK;
    }
    double* scratch = nullptr;
    bh_status st = scratch_for_current_device(&scratch);
    if (st != BH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + kPerBlock - 1) / kPerBlock);
    k_misfit_partial<<<nb, kThreads, 0, s>>>(n, seis_mod, seis_obs, resid, scratch);
    k_misfit_total<<<1, 1024, 0, s>>>(nb, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(J, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        bh_internal_set_thread_error(std::string("bh_residual_misfit_noalloc: ") +
                                     cudaGetErrorString(e));
        return BH_ERR_CUDA;
    }
    return BH_OK;
}
