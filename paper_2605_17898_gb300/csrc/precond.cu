// Pivoted-Cholesky preconditioner for the CG solves: P = L L^T + sigma^2 I with L the rank-k
// partial pivoted Cholesky factor of K_ff (Harbrecht, Peters & Schneider 2012; the BBMM
// preconditioner of Gardner et al. 2018), the gap the paper names for its CG path (Sec. 5).
//
// Construction (once per call, float64): k steps, each an argmax of the residual diagonal
// (first index on ties) and one kernel column computed from the caller's float32 X with float64
// lengthscales, so the pivots match a float64 reference. Application inside the CG iterations
// (Woodbury): P^{-1} R = (R - L C^{-1} L^T R) / sigma^2, C = sigma^2 I_k + L^T L, as three
// launches: block partials of L^T R (float32 products summed per block, float64 across blocks in
// a fixed order), U = C^{-1} L^T R in float64 by one block, and the row update with the r^T z
// partials of the recurrence.
#include <math.h>

#include "lgp_internal.cuh"

namespace lgp {

namespace {

struct PivInfo {
    int piv;
    int ok;
    double sd;            // sqrt of the pivot's residual diagonal
    double xi[kMaxD];     // the pivot's raw coordinates
    double li[kMaxRank];  // L[q][piv] for the columns already built
};

struct InvLs {
    double v[kMaxD];
};

__device__ double phi64(int kind, double r2) {
    switch (kind) {
        case LGP_RBF: return exp(-0.5 * r2);
        case LGP_MATERN52: {
            const double r = sqrt(r2);
            return (1.0 + 2.23606797749979 * r + (5.0 / 3.0) * r2) * exp(-2.23606797749979 * r);
        }
        case LGP_MATERN12: return exp(-sqrt(r2));
        case LGP_MATERN32: {
            const double r = sqrt(r2);
            return (1.0 + 1.7320508075688772 * r) * exp(-1.7320508075688772 * r);
        }
    }
    return 0.0;
}

inline int grid_for(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

__global__ void pivchol_init_kernel(double *__restrict__ d, double *__restrict__ L, int64_t N, int64_t Np, int k,
                                    double s2) {
    const int64_t total = Np * (int64_t)(k + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < Np) d[e] = e < N ? s2 : 0.0;
        else L[e - Np] = 0.0;
    }
}

// One block: pivot = argmax d over rows < N (first index on ties), and the data the column
// kernel needs.
__global__ void pivchol_argmax_kernel(const double *__restrict__ d, int64_t N, const float *__restrict__ X, int D,
                                      const double *__restrict__ L, int64_t Np, int m, double floor_d, PivInfo *pi) {
    __shared__ double bv[1024];
    __shared__ int64_t bi[1024];
    double v = -1.0;
    int64_t idx = N;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
        if (d[i] > v) {
            v = d[i];
            idx = i;
        }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = bv[threadIdx.x + s];
            const int64_t oi = bi[threadIdx.x + s];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t p = bi[0];
        const double val = bv[0];
        // a residual at most floor_d (1e-10 s^2) means K_ff is reproduced: the remaining columns stay zero
        const int ok = p < N && val > floor_d && isfinite(val) && (m == 0 || pi->ok);
        pi->ok = ok;
        pi->piv = ok ? (int)p : 0;
        pi->sd = ok ? sqrt(val) : 1.0;
        for (int dd = 0; dd < kMaxD; ++dd) pi->xi[dd] = (ok && dd < D) ? (double)X[p * D + dd] : 0.0;
        for (int q = 0; q < kMaxRank; ++q) pi->li[q] = (ok && q < m) ? L[(int64_t)q * Np + p] : 0.0;
    }
}

// Column m: L[m][j] = (k(x_j, x_piv) - sum_q<m L[q][j] L[q][piv]) / sqrt(d_piv); d_j -= L[m][j]^2.
__global__ void pivchol_col_kernel(double *__restrict__ L, double *__restrict__ d, int64_t N, int64_t Np,
                                   const float *__restrict__ X, int D, InvLs inv_ls, double s2, int kind, int m,
                                   const PivInfo *__restrict__ pi) {
    const int ok = pi->ok;
    const int piv = pi->piv;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        if (!ok) {
            L[(int64_t)m * Np + j] = 0.0;
            continue;
        }
        double r2 = 0.0;
        for (int dd = 0; dd < D; ++dd) {
            const double diff = ((double)X[j * D + dd] - pi->xi[dd]) * inv_ls.v[dd];
            r2 += diff * diff;
        }
        double v = s2 * phi64(kind, r2);
        for (int q = 0; q < m; ++q) v -= L[(int64_t)q * Np + j] * pi->li[q];
        v /= pi->sd;
        L[(int64_t)m * Np + j] = v;
        d[j] = (j == piv) ? 0.0 : d[j] - v * v;
    }
}

// Block partials of the Gram matrix L^T L (rows split over the grid), [G][k * k].
__global__ void gram_kernel(const double *__restrict__ L, int64_t Np, int64_t N, int k, double *__restrict__ partial) {
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(N, (int64_t)blockIdx.x * per), r1 = min(N, r0 + per);
    for (int pq = threadIdx.x; pq < k * k; pq += blockDim.x) {
        const int q = pq / k, r = pq - q * k;
        const double *a = L + (int64_t)q * Np, *b = L + (int64_t)r * Np;
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += a[i] * b[i];
        partial[(int64_t)blockIdx.x * k * k + pq] = s;
    }
}

__global__ void to_f32_kernel(const double *__restrict__ src, float *__restrict__ dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

// Block partials of S = L^T R: partial[b][q t + c] = sum over block b's rows of L[q][i] R[i, c].
__global__ void pc_ltr_kernel(const float *__restrict__ L, int64_t Np, int k, const float *__restrict__ R,
                              int64_t ldr, int64_t N, int t, double *__restrict__ partial, const CgState *st) {
    if (st && st->done) return;
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(N, (int64_t)blockIdx.x * per), r1 = min(N, r0 + per);
    for (int pq = threadIdx.x; pq < k * t; pq += blockDim.x) {
        const int q = pq / t, c = pq - q * t;
        const float *lq = L + (int64_t)q * Np;
        float s = 0.0f;
        for (int64_t i = r0; i < r1; ++i) s = fmaf(lq[i], R[i * ldr + c], s);
        partial[(int64_t)blockIdx.x * k * t + pq] = (double)s;
    }
}

// One block of k * t threads: S = sum_b partial[b] (index order), U = C^{-1} S.
__global__ void pc_small_kernel(const double *__restrict__ partial, int G, int k, int t,
                                const double *__restrict__ Cinv, double *__restrict__ U, const CgState *st) {
    if (st && st->done) return;
    __shared__ double S[kMaxRank * kMaxT];
    const int pq = threadIdx.x;
    if (pq < k * t) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) s += partial[(int64_t)b * k * t + pq];
        S[pq] = s;
    }
    __syncthreads();
    if (pq < k * t) {
        const int q = pq / t, c = pq - q * t;
        double u = 0.0;
        for (int r = 0; r < k; ++r) u += Cinv[q * k + r] * S[r * t + c];
        U[pq] = u;
    }
}

// Z = (R - L U) / sigma^2 (and a copy into P when given), with block partials of r^T z per column.
__global__ void pc_apply_kernel(const float *__restrict__ L, int64_t Np, int k, const double *__restrict__ U,
                                const float *__restrict__ R, int64_t ldr, float *__restrict__ Z, int64_t ldz,
                                float *__restrict__ Pc, int64_t N, int t, double inv_noise,
                                double *__restrict__ rz_partial, const CgState *st) {
    if (st && st->done) return;
    __shared__ double red[256];
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(N, (int64_t)blockIdx.x * per), r1 = min(N, r0 + per);
    const int c = threadIdx.x % t;
    float u[kMaxRank];
#pragma unroll
    for (int q = 0; q < kMaxRank; ++q) u[q] = q < k ? (float)U[q * t + c] : 0.0f;
    float s_hi = 0.0f, s_lo = 0.0f;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const float rv = R[i * ldr + c];
        float acc = rv;
#pragma unroll
        for (int q = 0; q < kMaxRank; ++q)
            if (q < k) acc = fmaf(-L[(int64_t)q * Np + i], u[q], acc);
        const float zv = (float)((double)acc * inv_noise);
        Z[i * ldz + c] = zv;
        if (Pc) Pc[i * ldz + c] = zv;
        acc_prod2(s_hi, s_lo, rv, zv);
    }
    if (!rz_partial) return;
    // per-column block reduction (threads tid, tid + t, ... own column tid % t)
    red[threadIdx.x] = (double)s_hi + (double)s_lo;
    __syncthreads();
    const int nr = blockDim.x / t;
    int w = 1;
    while (w < nr) w <<= 1;
    for (w >>= 1; w >= 1; w >>= 1) {
        const int slot = threadIdx.x / t;
        if (slot < w && slot + w < nr) red[threadIdx.x] += red[threadIdx.x + w * t];
        __syncthreads();
    }
    if (threadIdx.x < t) rz_partial[(int64_t)blockIdx.x * t + threadIdx.x] = red[threadIdx.x];
}

// Probes with covariance P: rhs[i, col0 + c] = sum_q L[q][i] E[N + q, c] + sigma E[i, c].
__global__ void precond_probes_kernel(const double *__restrict__ L, int64_t Np, int k, const float *__restrict__ E,
                                      int64_t N, int m, double sigma, float *__restrict__ rhs, int64_t ldr, int col0) {
    const int64_t total = N * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int c = (int)(e - i * m);
        double v = sigma * (double)E[i * m + c];
        for (int q = 0; q < k; ++q) v += L[(int64_t)q * Np + i] * (double)E[(N + q) * m + c];
        rhs[i * ldr + col0 + c] = (float)v;
    }
}

}  // namespace

size_t pivinfo_bytes() { return sizeof(PivInfo); }

void launch_pivchol(const float *X, int64_t N, int64_t Np, int D, const double *inv_ls_host, double s2, int kind,
                    int k, double *L64, double *d, void *pinfo, cudaStream_t st) {
    InvLs il = {};
    for (int dd = 0; dd < D && dd < kMaxD; ++dd) il.v[dd] = inv_ls_host[dd];
    pivchol_init_kernel<<<grid_for(Np * (k + 1)), 256, 0, st>>>(d, L64, N, Np, k, s2);
    PivInfo *pi = (PivInfo *)pinfo;
    for (int m = 0; m < k; ++m) {
        pivchol_argmax_kernel<<<1, 1024, 0, st>>>(d, N, X, D, L64, Np, m, 1e-10 * s2, pi);
        pivchol_col_kernel<<<grid_for(N), 256, 0, st>>>(L64, d, N, Np, X, D, il, s2, kind, m, pi);
    }
}

void launch_gram(const double *L64, int64_t Np, int64_t N, int k, double *partial, int G, cudaStream_t st) {
    gram_kernel<<<G, 256, 0, st>>>(L64, Np, N, k, partial);
}

void launch_to_f32(const double *src, float *dst, int64_t n, cudaStream_t st) {
    to_f32_kernel<<<grid_for(n), 256, 0, st>>>(src, dst, n);
}

void launch_precond_apply(const Precond &pc, const float *R, int64_t ldr, float *Z, int64_t ldz, float *Pcopy,
                          int64_t N, int t, double *rz_partial, int G_vec, const CgState *state, cudaStream_t st) {
    pc_ltr_kernel<<<pc.G, 256, 0, st>>>(pc.L32, pc.Np, pc.k, R, ldr, N, t, pc.part, state);
    pc_small_kernel<<<1, pc.k * t, 0, st>>>(pc.part, pc.G, pc.k, t, pc.Cinv, pc.U, state);
    pc_apply_kernel<<<G_vec, (256 / t) * t, 0, st>>>(pc.L32, pc.Np, pc.k, pc.U, R, ldr, Z, ldz, Pcopy, N, t,
                                                     1.0 / pc.noise, rz_partial, state);
}

void launch_precond_probes(const double *L64, int64_t Np, int k, const float *E, int64_t N, int m, double sigma,
                           float *rhs, int64_t ldr, int col0, cudaStream_t st) {
    precond_probes_kernel<<<grid_for(N * m), 256, 0, st>>>(L64, Np, k, E, N, m, sigma, rhs, ldr, col0);
}

}  // namespace lgp
