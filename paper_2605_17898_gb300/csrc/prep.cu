// Input preparation: prescaled X, Rademacher probes, finiteness scans, column copies.
#include "lgp_internal.cuh"

namespace lgp {

namespace {

struct ScaleArg {
    float s[kMaxD];
};

// Xs[i, d] = X[i, d] * scale[d] for i < N, d < D; zero in the padded rows and columns.
__global__ void prep_x_kernel(const float *__restrict__ X, int64_t N, int D, int dpad, ScaleArg sc,
                              float *__restrict__ Xs, int64_t Np, int *err_flag) {
    const int64_t total = Np * dpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / dpad;
        const int d = (int)(e - i * dpad);
        float v = 0.0f;
        if (i < N && d < D) {
            const float x = X[i * D + d];
            if (!isfinite(x)) atomicOr(err_flag, 1);
            v = x * sc.s[d];
        }
        Xs[e] = v;
    }
}

// One output of splitmix64 for state `x`: advance by the golden gamma, then the
// two xor-shift-multiply rounds and a final xor-shift (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void rademacher_kernel(uint64_t seed, int64_t N, int m, float *__restrict__ Z, int64_t ldz, int col0) {
    const int64_t total = N * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int c = (int)(e - i * m);
        const uint64_t key = seed ^ (((uint64_t)c << 32) | (uint64_t)i);
        Z[i * ldz + col0 + c] = (splitmix64(key) >> 63) ? -1.0f : 1.0f;
    }
}

__global__ void scan_finite_kernel(const float *__restrict__ A, int64_t n, int *err_flag) {
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(A[e]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err_flag, 1);
}

__global__ void copy_cols_kernel(const float *__restrict__ src, int64_t lds, float *__restrict__ dst, int64_t ldd,
                                 int64_t rows, int cols, int dst_col0) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols;
        const int c = (int)(e - i * cols);
        dst[i * ldd + dst_col0 + c] = src[i * lds + c];
    }
}

inline int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 8192) g = 8192;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

void launch_prep_x(const float *X, int64_t N, int D, int dpad, const float *scale_host, float *Xs, int64_t Np,
                   int *err_flag, cudaStream_t st) {
    ScaleArg sc;
    for (int d = 0; d < kMaxD; ++d) sc.s[d] = d < D ? scale_host[d] : 0.0f;
    prep_x_kernel<<<grid_for(Np * dpad, 256), 256, 0, st>>>(X, N, D, dpad, sc, Xs, Np, err_flag);
}

void launch_rademacher(uint64_t seed, int64_t N, int m, float *Z, int64_t ldz, int col0, cudaStream_t st) {
    rademacher_kernel<<<grid_for(N * m, 256), 256, 0, st>>>(seed, N, m, Z, ldz, col0);
}

void launch_scan_finite(const float *A, int64_t n, int *err_flag, cudaStream_t st) {
    scan_finite_kernel<<<grid_for(n, 256), 256, 0, st>>>(A, n, err_flag);
}

void launch_copy_cols(const float *src, int64_t lds, float *dst, int64_t ldd, int64_t rows, int cols, int dst_col0,
                      cudaStream_t st) {
    copy_cols_kernel<<<grid_for(rows * cols, 256), 256, 0, st>>>(src, lds, dst, ldd, rows, cols, dst_col0);
}

}  // namespace lgp
