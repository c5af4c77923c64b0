// Posterior prediction pieces (Sec. 2: mu_* = K_*f K_y^-1 y, Sigma_* = K_** - K_*f K_y^-1 K_f*):
// kernel columns k(X, x*_j) as right-hand sides of the exact-variance solves, and the two
// variance finalisations (per-point dots, or the probe diagonal estimate). The products
// K(X*, X) V and K(X, X*) Z run on the SIMT cross product (mv_simt.cuh).
#include <algorithm>

#include "lgp_internal.cuh"

namespace lgp {

namespace {

inline int grid_for(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

// B[i, col0 + c] = k(xh_i, xs_{j0 + c}) for i < N, c < tc (prescaled coordinates, zero padded to
// dpad); B[i, col0 + c] = 0 for N <= i < Np.
template <int KIND>
__global__ void kernel_cols_kernel(const float *__restrict__ Xh, int64_t N, int64_t Np, int dpad,
                                   const float *__restrict__ Xsh, int64_t j0, int tc, float log2s2,
                                   float *__restrict__ B, int64_t ldb, int col0) {
    const int64_t total = Np * tc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / tc;
        const int c = (int)(e - i * tc);
        float k = 0.0f;
        if (i < N) {
            const float *a = Xh + i * dpad;
            const float *b = Xsh + (j0 + c) * dpad;
            float r2 = 0.0f;
            for (int d = 0; d < dpad; ++d) {
                const float dd = a[d] - b[d];
                r2 = fmaf(dd, dd, r2);
            }
            k = Entry<KIND>::k(r2, log2s2);
        }
        B[i * ldb + col0 + c] = k;
    }
}

// var[j0 + c - c0] = s2 - dots[c] for c0 <= c < t (dots: the float64 column dots b_c . (K_y^-1 b)_c)
__global__ void var_from_dots_kernel(const double *__restrict__ dots, int c0, int t, float s2, float *__restrict__ var,
                                     int64_t j0) {
    const int c = c0 + (int)threadIdx.x;
    if (c < t) var[j0 + c - c0] = (float)((double)s2 - dots[c]);
}

// var[i] = s2 - (1/m) sum_c Z[i, c] Q[i, c] (float64 accumulation)
__global__ void var_from_probes_kernel(const float *__restrict__ Z, int64_t ldz, const float *__restrict__ Q,
                                       int64_t ldq, int64_t M, int m, float s2, float *__restrict__ var) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < m; ++c) s += (double)Z[i * ldz + c] * (double)Q[i * ldq + c];
        var[i] = (float)((double)s2 - s / m);
    }
}

}  // namespace

void launch_kernel_cols(const KernelParams &kp, const float *Xh, int64_t N, int64_t Np, const float *Xsh, int64_t j0,
                        int tc, float *B, int64_t ldb, int col0, cudaStream_t st) {
    const int g = grid_for(Np * tc);
    switch (kp.kind) {
        case LGP_RBF:
            kernel_cols_kernel<LGP_RBF><<<g, 256, 0, st>>>(Xh, N, Np, kp.dpad, Xsh, j0, tc, kp.log2_s2, B, ldb, col0);
            break;
        case LGP_MATERN52:
            kernel_cols_kernel<LGP_MATERN52><<<g, 256, 0, st>>>(Xh, N, Np, kp.dpad, Xsh, j0, tc, kp.log2_s2, B, ldb,
                                                               col0);
            break;
        case LGP_MATERN12:
            kernel_cols_kernel<LGP_MATERN12><<<g, 256, 0, st>>>(Xh, N, Np, kp.dpad, Xsh, j0, tc, kp.log2_s2, B, ldb,
                                                               col0);
            break;
        case LGP_MATERN32:
            kernel_cols_kernel<LGP_MATERN32><<<g, 256, 0, st>>>(Xh, N, Np, kp.dpad, Xsh, j0, tc, kp.log2_s2, B, ldb,
                                                               col0);
            break;
    }
}

void launch_var_from_dots(const double *dots, int c0, int t, float s2, float *var, int64_t j0, cudaStream_t st) {
    var_from_dots_kernel<<<1, kMaxT, 0, st>>>(dots, c0, t, s2, var, j0);
}

void launch_var_from_probes(const float *Z, int64_t ldz, const float *Q, int64_t ldq, int64_t M, int m, float s2,
                            float *var, cudaStream_t st) {
    var_from_probes_kernel<<<grid_for(M), 256, 0, st>>>(Z, ldz, Q, ldq, M, m, s2, var);
}

}  // namespace lgp
