// lgp_kernel_matvec_noalloc: the tensor-core product K_y V for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc:
//   - programs whose device memory is owned by another allocator (a framework's
//     caching pool, a fixed arena sized at start-up), which must not see a library
//     take memory behind their back;
//   - services that run under a fixed device-memory budget, where an allocation
//     that fails in the middle of a request cannot be retried;
//   - latency-critical loops, where cudaMalloc/cudaFree can synchronise the device.
// For them this entry point takes no context and allocates nothing. Its scratch
// (prescaled X, the split copies of V, the split-column partial sums and two status
// words) is one file-scope __device__ array, held by every GPU that loads the
// library until the process exits. lgp_kernel_matvec_noalloc_status reads the
// status words back.
//
// Limits: N <= 8192, t in {16, 32}, D <= 8.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "lgp_internal.cuh"

using namespace lgp;

namespace {

constexpr int64_t kNoallocMaxN = 8192;   // largest N accepted
constexpr int64_t kNoallocNp = 8192;     // rows after padding to a multiple of 256
constexpr int kNoallocMaxT = 32;
constexpr int kNoallocMaxSplits = 16;    // the product's grid splits the columns at most 16 ways at Np = 8192

constexpr size_t kXsBytes = (size_t)kNoallocNp * 8 * sizeof(float);
constexpr size_t kVsplitBytes = (size_t)2 * kNoallocNp * kNoallocMaxT * 2 + 2 * 64 * 4 + (size_t)8 * kNoallocNp * 4;
constexpr size_t kPartialBytes = (size_t)kNoallocMaxSplits * kNoallocNp * kNoallocMaxT * sizeof(float);
constexpr size_t kFlagBytes = 256;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffXs = 0;
constexpr size_t kOffVsplit = align256(kOffXs + kXsBytes);
constexpr size_t kOffPartial = align256(kOffVsplit + kVsplitBytes);
constexpr size_t kOffFlags = align256(kOffPartial + kPartialBytes);
constexpr size_t kScratchBytes = align256(kOffFlags + kFlagBytes);  // about 17.3 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device (the array's name is
// only a host-side stand-in; kernels must be given this address).
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

cudaError_t scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool is_device_array(const void *p) {
    if (!p || ((uintptr_t)p) % 4 != 0) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == dev;
}

}  // namespace

extern "C" lgp_status lgp_kernel_matvec_noalloc(const lgp_hyper *hyp, const float *X, const float *V, float *out,
                                                int64_t N, int32_t t, int32_t prec, lgp_stream stream) {
    if (!hyp || N < 1) return LGP_ERR_INVALID_ARG;
    if (N > kNoallocMaxN || !(t == 16 || t == 32)) return LGP_ERR_UNSUPPORTED;
    if (!(prec == LGP_PREC_AUTO || prec == LGP_PREC_SPLIT_F16 || prec == LGP_PREC_SPLIT_BF16))
        return LGP_ERR_UNSUPPORTED;
    if (!kind_supported(hyp->kind)) return LGP_ERR_INVALID_ARG;
    if (hyp->D < 1 || hyp->D > kMaxD) return LGP_ERR_UNSUPPORTED;
    if (!hyp->log_lengthscale || !std::isfinite(hyp->log_outputscale) || !std::isfinite(hyp->log_noise))
        return LGP_ERR_INVALID_ARG;
    if (!is_device_array(X) || !is_device_array(V) || !is_device_array(out)) return LGP_ERR_INVALID_ARG;
    if (out == V || (const float *)out == X) return LGP_ERR_INVALID_ARG;
    if (!tc_supported(t)) return LGP_ERR_UNSUPPORTED;

    KernelParams kp = {};
    kp.kind = hyp->kind;
    kp.D = hyp->D;
    kp.dpad = dpad_of(hyp->D);
    const double c = prescale_of(hyp->kind);
    for (int d = 0; d < hyp->D; ++d) {
        const double ll = hyp->log_lengthscale[d];
        if (!std::isfinite(ll)) return LGP_ERR_INVALID_ARG;
        kp.scale[d] = (float)(c * std::exp(-ll));
        if (!(kp.scale[d] > 0.0f) || !std::isfinite(kp.scale[d])) return LGP_ERR_UNSUPPORTED;
    }
    kp.s2 = (float)std::exp((double)hyp->log_outputscale);
    kp.log2_s2 = (float)((double)hyp->log_outputscale / std::log(2.0));
    kp.noise = (float)std::exp((double)hyp->log_noise);
    if (!(kp.s2 > 0.0f) || !std::isfinite(kp.s2) || !std::isfinite(kp.noise)) return LGP_ERR_UNSUPPORTED;

    int sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return LGP_ERR_CUDA;
    const int64_t Np = (N + 255) / 256 * 256;
    const int64_t partial_floats = mv_tc_partial_floats(Np, t, sms);
    if (partial_floats * (int64_t)sizeof(float) > (int64_t)kPartialBytes) return LGP_ERR_UNSUPPORTED;

    unsigned char *base = nullptr;
    if (scratch_for_current_device(&base) != cudaSuccess) return LGP_ERR_CUDA;
    float *xs = (float *)(base + kOffXs);
    void *vsplit = base + kOffVsplit;
    float *partial = (float *)(base + kOffPartial);
    int *flags = (int *)(base + kOffFlags);
    cudaStream_t st = (cudaStream_t)stream;

    // The array keeps the previous call's contents. Every region the product reads is rewritten
    // first (the product clears its own column maxima); the two status words (flags[0]: NaN or
    // Inf in X, flags[1]: a bounded wait ran out) are only ever OR-ed into, so they accumulate
    // over calls until lgp_kernel_matvec_noalloc_status reads and clears them.
    launch_prep_x(X, N, kp.D, kp.dpad, kp.scale, xs, Np, flags, st);
    if (cudaGetLastError() != cudaSuccess) return LGP_ERR_CUDA;
    const int fmt = prec == LGP_PREC_SPLIT_BF16 ? 0 : 1;
    if (launch_mv_tc(kp, xs, N, Np, V, t, out, t, t, fmt, vsplit, partial, (int64_t)(kPartialBytes / sizeof(float)),
                     nullptr, flags + 1, 4000000000LL, sms, st) != cudaSuccess)
        return LGP_ERR_CUDA;
    return LGP_OK;
}

extern "C" lgp_status lgp_kernel_matvec_noalloc_status(lgp_stream stream) {
    unsigned char *base = nullptr;
    if (scratch_for_current_device(&base) != cudaSuccess) return LGP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int words[2] = {0, 0};
    if (cudaStreamSynchronize(st) != cudaSuccess) return LGP_ERR_CUDA;
    if (cudaMemcpy(words, base + kOffFlags, sizeof words, cudaMemcpyDeviceToHost) != cudaSuccess) return LGP_ERR_CUDA;
    if (cudaMemset(base + kOffFlags, 0, sizeof words) != cudaSuccess) return LGP_ERR_CUDA;
    if (words[1]) return LGP_ERR_TIMEOUT;
    if (words[0]) return LGP_ERR_NONFINITE;
    return LGP_OK;
}
