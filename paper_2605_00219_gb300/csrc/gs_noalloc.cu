// gs_noalloc.cu -- L1 loss and gradient that needs no device allocation.
//
// Some callers cannot allocate device memory at all: a host framework that
// owns every byte of the GPU through its own pool and forbids libraries from
// calling cudaMalloc, a real-time renderer whose frame loop must never block
// on the allocator, or code that runs while allocation is disallowed.  Such a
// caller can still compute the L1 loss of its rendered images and the
// gradient dL/dC with gs_loss_l1_noalloc(), which needs no plan and no
// workspace: its only scratch (one partial sum per thread block and a
// completion counter) lives in the static device array below, which the
// library image carries and every GPU that loads the library keeps until the
// process exits.
//
// The array is shared by all calls on a device and keeps whatever the last
// call left in it; the counter is cleared before every launch.  Calls whose
// executions overlap on the GPU (different streams, no ordering between
// them) race on the array and must not be issued.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr int64_t kNaMaxBlocks = GS_L1_NOALLOC_MAX_VALUES / (kNaThreads * kNaItems);
constexpr int kNaMaxDevices = 64;
static_assert(kNaMaxBlocks * kNaThreads * kNaItems == GS_L1_NOALLOC_MAX_VALUES, "whole blocks");

// [0] completion counter, [1..63] unused (keeps the partials 256-byte
// aligned), [64 ..] one float partial sum per thread block.
static __device__ __align__(256) uint32_t g_l1_noalloc_scratch[64 + kNaMaxBlocks];

std::mutex g_setup_mutex;
uint32_t* g_scratch_addr[kNaMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// cached.  It is the address in the device's primary context; a device reset
// or another current context would make it stale, which the header rules
// out for callers.
gs_status scratch_on_current_device(uint32_t** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_l1_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return GS_OK;
}

__global__ void __launch_bounds__(kNaThreads) k_loss_l1_noalloc(const float* __restrict__ image,
                                                                const float* __restrict__ target,
                                                                float* __restrict__ dl, int64_t n, float inv_n,
                                                                uint32_t* __restrict__ scratch,
                                                                float* __restrict__ loss_out)
{
    __shared__ float ws[kNaThreads / 32];
    __shared__ bool is_last;
    uint32_t* counter = scratch;
    float* part = reinterpret_cast<float*>(scratch + 64);
    const int64_t base = (int64_t)blockIdx.x * kNaThreads * kNaItems;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kNaItems; i++) {
        const int64_t idx = base + i * kNaThreads + threadIdx.x;
        if (idx < n) {
            const float d = image[idx] - target[idx];
            dl[idx] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
            s += fabsf(d);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < kNaThreads / 32; i++) t += ws[i];
        part[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        float t = 0.f, comp = 0.f;  // Kahan-compensated FP32 sum, fixed order
        for (unsigned i = 0; i < gridDim.x; i++) {
            const float y = ((volatile float*)part)[i] - comp;
            const float u = t + y;
            comp = (u - t) - y;
            t = u;
        }
        *loss_out = t * inv_n;
        *counter = 0u;
    }
}

}  // namespace

extern "C" gs_status gs_loss_l1_noalloc(const float* image, const float* target, float* dL_dimage, float* loss,
                                        int64_t n_values, void* stream)
{
    if (!image || !target || !dL_dimage || !loss) return GS_ERR_INVALID_ARG;
    if (n_values <= 0 || n_values > GS_L1_NOALLOC_MAX_VALUES) return GS_ERR_INVALID_ARG;
    uint32_t* scratch = nullptr;
    const gs_status e = scratch_on_current_device(&scratch);
    if (e != GS_OK) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(scratch, 0, sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    const int64_t blocks = (n_values + kNaThreads * kNaItems - 1) / (kNaThreads * kNaItems);
    k_loss_l1_noalloc<<<(unsigned)blocks, kNaThreads, 0, st>>>(image, target, dL_dimage, n_values,
                                                               1.0f / (float)n_values, scratch, loss);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}
