// Pipe-throughput microbenchmarks used as roofline denominators for the entry generation:
// float32 FMA, packed float32x2 FMA, and the MUFU ex2 / sqrt approximations, each timed with
// CUDA events on the caller's stream at whatever clock the GPU runs.
#include <cuda_runtime.h>

#include "lgp_internal.cuh"

namespace lgp {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

// results land here only if a chain happens to hit an exact sentinel (keeps the loops live)
__device__ float g_peak_sink[16384];

__global__ void peak_ffma_kernel(int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.0f) g_peak_sink[blockIdx.x & 16383] = s;
}

__global__ void peak_ffma2_kernel(int iters, float b, float c) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == 12345.0f) g_peak_sink[blockIdx.x & 16383] = s;
}

__global__ void peak_ex2_kernel(int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = -(threadIdx.x * 1e-4f + k * 0.01f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = -ex2_approx(a[k]);  // stays in [-1, -0.5]
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.0f) g_peak_sink[blockIdx.x & 16383] = s;
}

__global__ void peak_sqrt_kernel(int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 2.0f + threadIdx.x * 1e-4f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = sqrt_approx(a[k]);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.0f) g_peak_sink[blockIdx.x & 16383] = s;
}

}  // namespace
}  // namespace lgp

using namespace lgp;

// which: 0 FFMA (results/s), 1 FFMA2 (float32 FMAs/s, two per instruction lane), 2 MUFU ex2, 3 MUFU sqrt.
extern "C" lgp_status lgp_measure_pipe_peak(int32_t which, double *ops_per_s, lgp_stream stream) {
    if (!ops_per_s || which < 0 || which > 3) return LGP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return LGP_ERR_CUDA;
    const int blocks = sms * 8;
    const int iters = 4096;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return LGP_ERR_CUDA;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, st);
        switch (which) {
            case 0: peak_ffma_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f); break;
            case 1: peak_ffma2_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f); break;
            case 2: peak_ex2_kernel<<<blocks, kPeakThreads, 0, st>>>(iters); break;
            default: peak_sqrt_kernel<<<blocks, kPeakThreads, 0, st>>>(iters); break;
        }
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return LGP_ERR_CUDA;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;  // first launch warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double per_thread = (double)iters * kChains * (which == 1 ? 2.0 : 1.0);
    *ops_per_s = per_thread * blocks * kPeakThreads / (best * 1e-3);
    return cudaGetLastError() == cudaSuccess ? LGP_OK : LGP_ERR_CUDA;
}
