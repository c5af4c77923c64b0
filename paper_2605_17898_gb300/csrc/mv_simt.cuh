// FP32 SIMT kernels of the matrix-free product family (templates; instantiated per kernel kind).
//
// All three kernels share one structure: a CTA of 128 threads owns a block of
// 128*R rows of the output; each thread keeps R prescaled rows xh_i in
// registers. The CTA sweeps a range of columns j in tiles of BN=64 staged in
// shared memory (prescaled x_j plus the matching right-hand-side rows), and
// every thread generates its R x BN kernel entries in registers, uses them and
// drops them: no entry is ever written to global memory (Sec. 3 "GPU
// backends": the fused product that never materialises K). A grid dimension
// splits the column range when the row blocks alone cannot fill the GPU; the
// partial sums are then reduced by a second, deterministic kernel.
//
// Summation: each thread sums one tile (64 columns) into a tile accumulator
// and adds that to its running total, so float32 rounding grows with the
// number of tiles rather than the number of columns.
#pragma once

#include "lgp_internal.cuh"

namespace lgp {

constexpr int kSimtThreads = 128;
constexpr int kSimtBN = 64;

struct SimtArgs {
    const float *Xs;   // prescaled column points [Np, DP]
    const float *Xr;   // prescaled row points [Npr, DP] (Xs itself for K_y V)
    const float *V;    // [N, ldv]
    float *out;        // [Nr, ldo] (direct mode)
    float *partial;    // [S, Npr, t] (split mode) or nullptr
    const int *skip;
    int64_t N, Np, ldv, ldo;
    int64_t Nr, Npr;   // rows of the output, and of Xr
    int cross;         // 1: out = K(Xr, Xs) V with no noise term
    int64_t cols_per_split;
    int t;
    float log2s2;
    float noise;
};

template <int D> struct DPad { static constexpr int value = D <= 4 ? 4 : 8; };

template <int D>
__device__ __forceinline__ void load_x_smem(const float *xs, float (&xj)[D]) {
    constexpr int DP = DPad<D>::value;
    const float4 q0 = *reinterpret_cast<const float4 *>(xs);
    xj[0] = q0.x;
    if (D > 1) xj[1 < D ? 1 : 0] = q0.y;
    if (D > 2) xj[2 < D ? 2 : 0] = q0.z;
    if (D > 3) xj[3 < D ? 3 : 0] = q0.w;
    if (DP == 8) {
        const float4 q1 = *reinterpret_cast<const float4 *>(xs + 4);
        if (D > 4) xj[4 < D ? 4 : 0] = q1.x;
        if (D > 5) xj[5 < D ? 5 : 0] = q1.y;
        if (D > 6) xj[6 < D ? 6 : 0] = q1.z;
        if (D > 7) xj[7 < D ? 7 : 0] = q1.w;
    }
}

template <int D>
__device__ __forceinline__ float sqdist(const float (&a)[D], const float (&b)[D]) {
    float d0 = a[0] - b[0];
    float r2 = d0 * d0;
#pragma unroll
    for (int d = 1; d < D; ++d) {
        const float dd = a[d] - b[d];
        r2 = fmaf(dd, dd, r2);
    }
    return r2;
}

// Stage x_j (and nothing else) for column tile [j0, j0 + BN).
template <int D>
__device__ __forceinline__ void stage_x(float *xs, const float *__restrict__ Xs, int64_t j0, int64_t Np) {
    constexpr int DP = DPad<D>::value;
    for (int e = threadIdx.x; e < kSimtBN * DP / 4; e += kSimtThreads) {
        const int jj = (e * 4) / DP;
        const int64_t j = j0 + jj;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < Np) v = *reinterpret_cast<const float4 *>(Xs + j0 * DP + e * 4);
        *reinterpret_cast<float4 *>(xs + e * 4) = v;
    }
}

// ------------------------------------------------------------------ product K_y V (columns c0..c0+TT-1)

template <int KIND, int D, int TT, int R>
__global__ void __launch_bounds__(kSimtThreads) mv_simt_kernel(SimtArgs a) {
    constexpr int DP = DPad<D>::value;
    constexpr int BM = kSimtThreads * R;
    __shared__ __align__(16) float xs[kSimtBN * DP];
    __shared__ __align__(16) float vs[kSimtBN * TT];
    if (a.skip && *a.skip) return;

    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int c0 = blockIdx.z * TT;
    const int64_t jb = (int64_t)blockIdx.y * a.cols_per_split;
    const int64_t je = min(a.N, jb + a.cols_per_split);

    float xi[R][D];
    float tot[R][TT];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = row0 + r * kSimtThreads + tid;
#pragma unroll
        for (int d = 0; d < D; ++d) xi[r][d] = (i < a.Npr) ? a.Xr[i * DP + d] : 0.0f;
#pragma unroll
        for (int c = 0; c < TT; ++c) tot[r][c] = 0.0f;
    }

    for (int64_t j0 = jb; j0 < je; j0 += kSimtBN) {
        __syncthreads();
        stage_x<D>(xs, a.Xs, j0, a.Np);
        for (int e = tid; e < kSimtBN * TT; e += kSimtThreads) {
            const int jj = e / TT;
            const int c = e - jj * TT;
            const int64_t j = j0 + jj;
            vs[e] = (j < je && c0 + c < a.t) ? a.V[j * a.ldv + c0 + c] : 0.0f;
        }
        __syncthreads();

        float acc[R][TT];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < TT; ++c) acc[r][c] = 0.0f;

#pragma unroll 2
        for (int jj = 0; jj < kSimtBN; ++jj) {
            float xj[D];
            load_x_smem<D>(xs + jj * DP, xj);
            float v[TT];
            if (TT % 4 == 0) {
#pragma unroll
                for (int c = 0; c < TT; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(vs + jj * TT + c);
                    v[c] = q.x; v[(c + 1) % TT] = q.y; v[(c + 2) % TT] = q.z; v[(c + 3) % TT] = q.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < TT; ++c) v[c] = vs[jj * TT + c];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float k = Entry<KIND>::k(sqdist<D>(xi[r], xj), a.log2s2);
#pragma unroll
                for (int c = 0; c < TT; ++c) acc[r][c] = fmaf(k, v[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < TT; ++c) tot[r][c] += acc[r][c];
    }

#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = row0 + r * kSimtThreads + tid;
        if (i >= a.Nr) continue;
        if (a.partial) {
            float *dst = a.partial + ((int64_t)blockIdx.y * a.Npr + i) * a.t + c0;
#pragma unroll
            for (int c = 0; c < TT; ++c)
                if (c0 + c < a.t) dst[c] = tot[r][c];
        } else {
#pragma unroll
            for (int c = 0; c < TT; ++c)
                if (c0 + c < a.t)
                    a.out[i * a.ldo + c0 + c] = a.cross ? tot[r][c] : fmaf(a.noise, a.V[i * a.ldv + c0 + c], tot[r][c]);
        }
    }
}

// ------------------------------------------------------------------ derivative blocks dK_p W

struct GradArgs {
    const float *Xs;
    const float *W;    // [N, t]
    float *G;          // [P, N, t] (direct) ; P = D + 2
    float *partial;    // [S, D + 1, Np, t] or nullptr
    int64_t N, Np;
    int64_t cols_per_split;
    int t;
    float log2s2;
    float noise;
};

template <int KIND, int D, int TT>
__global__ void __launch_bounds__(kSimtThreads) mv_grad_kernel(GradArgs a) {
    constexpr int DP = DPad<D>::value;
    constexpr int NB = D + 1;  // lengthscale blocks + outputscale block
    __shared__ __align__(16) float xs[kSimtBN * DP];
    __shared__ __align__(16) float ws[kSimtBN * TT];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kSimtThreads + tid;
    const int c0 = blockIdx.z * TT;
    const int64_t jb = (int64_t)blockIdx.y * a.cols_per_split;
    const int64_t je = min(a.N, jb + a.cols_per_split);

    float xi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) xi[d] = (i < a.Np) ? a.Xs[i * DP + d] : 0.0f;
    float tot[NB][TT];
#pragma unroll
    for (int p = 0; p < NB; ++p)
#pragma unroll
        for (int c = 0; c < TT; ++c) tot[p][c] = 0.0f;

    for (int64_t j0 = jb; j0 < je; j0 += kSimtBN) {
        __syncthreads();
        stage_x<D>(xs, a.Xs, j0, a.Np);
        for (int e = tid; e < kSimtBN * TT; e += kSimtThreads) {
            const int jj = e / TT;
            const int c = e - jj * TT;
            const int64_t j = j0 + jj;
            ws[e] = (j < je && c0 + c < a.t) ? a.W[j * a.t + c0 + c] : 0.0f;
        }
        __syncthreads();
        float acc[NB][TT];
#pragma unroll
        for (int p = 0; p < NB; ++p)
#pragma unroll
            for (int c = 0; c < TT; ++c) acc[p][c] = 0.0f;
        for (int jj = 0; jj < kSimtBN; ++jj) {
            float xj[D];
            load_x_smem<D>(xs + jj * DP, xj);
            float dd2[D];
            float r2 = 0.0f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float dd = xi[d] - xj[d];
                dd2[d] = dd * dd;
                r2 += dd2[d];
            }
            float k, psi;
            Entry<KIND>::k_psi(r2, a.log2s2, k, psi);
#pragma unroll
            for (int c = 0; c < TT; ++c) {
                const float w = ws[jj * TT + c];
                const float pw = psi * w;
#pragma unroll
                for (int d = 0; d < D; ++d) acc[d][c] = fmaf(pw, dd2[d], acc[d][c]);
                acc[D][c] = fmaf(k, w, acc[D][c]);
            }
        }
#pragma unroll
        for (int p = 0; p < NB; ++p)
#pragma unroll
            for (int c = 0; c < TT; ++c) tot[p][c] += acc[p][c];
    }
    if (i >= a.N) return;
#pragma unroll
    for (int p = 0; p < NB; ++p) {
#pragma unroll
        for (int c = 0; c < TT; ++c) {
            if (c0 + c >= a.t) continue;
            if (a.partial)
                a.partial[(((int64_t)blockIdx.y * NB + p) * a.Np + i) * a.t + c0 + c] = tot[p][c];
            else
                a.G[((int64_t)p * a.N + i) * a.t + c0 + c] = tot[p][c];
        }
    }
    if (!a.partial && blockIdx.y == 0) {
#pragma unroll
        for (int c = 0; c < TT; ++c)
            if (c0 + c < a.t)
                a.G[((int64_t)(D + 1) * a.N + i) * a.t + c0 + c] = a.noise * a.W[i * a.t + c0 + c];
    }
}

// ------------------------------------------------------------------ bilinear adjoint reduction

struct AdjArgs {
    const float *Xs;
    const float *A;      // [N, t]  rows i
    const float *B;      // [N, t]  rows j
    double *partial;     // [gridDim.x * gridDim.y, D + 1]
    int64_t N, Np;
    int64_t cols_per_split;
    int t;
    float log2s2;
};

// Kahan-compensated float accumulation.
__device__ __forceinline__ void kahan_add(float &s, float &comp, float x) {
    const float y = x - comp;
    const float t2 = s + y;
    comp = (t2 - s) - y;
    s = t2;
}

template <int KIND, int D, int TT>
__global__ void __launch_bounds__(kSimtThreads) adjoint_bilinear_kernel(AdjArgs a) {
    constexpr int DP = DPad<D>::value;
    constexpr int NB = D + 1;
    __shared__ __align__(16) float xs[kSimtBN * DP];
    __shared__ __align__(16) float bs[kSimtBN * TT];
    __shared__ double red[kSimtThreads / 32][NB];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kSimtThreads + tid;
    const int64_t jb = (int64_t)blockIdx.y * a.cols_per_split;
    const int64_t je = min(a.N, jb + a.cols_per_split);

    float xi[D];
    float ai[TT];
#pragma unroll
    for (int d = 0; d < D; ++d) xi[d] = (i < a.Np) ? a.Xs[i * DP + d] : 0.0f;
#pragma unroll
    for (int c = 0; c < TT; ++c) ai[c] = (i < a.N && c < a.t) ? a.A[i * a.t + c] : 0.0f;
    float tot[NB], comp[NB];
#pragma unroll
    for (int p = 0; p < NB; ++p) tot[p] = comp[p] = 0.0f;

    for (int64_t j0 = jb; j0 < je; j0 += kSimtBN) {
        __syncthreads();
        stage_x<D>(xs, a.Xs, j0, a.Np);
        for (int e = tid; e < kSimtBN * TT; e += kSimtThreads) {
            const int jj = e / TT;
            const int c = e - jj * TT;
            const int64_t j = j0 + jj;
            bs[e] = (j < je && c < a.t) ? a.B[j * a.t + c] : 0.0f;
        }
        __syncthreads();
        float acc[NB];
#pragma unroll
        for (int p = 0; p < NB; ++p) acc[p] = 0.0f;
#pragma unroll 2
        for (int jj = 0; jj < kSimtBN; ++jj) {
            float m = 0.0f;
            if (TT % 4 == 0) {
#pragma unroll
                for (int c = 0; c < TT; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(bs + jj * TT + c);
                    m = fmaf(ai[c], q.x, m);
                    m = fmaf(ai[(c + 1) % TT], q.y, m);
                    m = fmaf(ai[(c + 2) % TT], q.z, m);
                    m = fmaf(ai[(c + 3) % TT], q.w, m);
                }
            } else {
#pragma unroll
                for (int c = 0; c < TT; ++c) m = fmaf(ai[c], bs[jj * TT + c], m);
            }
            float xj[D];
            load_x_smem<D>(xs + jj * DP, xj);
            float dd2[D];
            float r2 = 0.0f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float dd = xi[d] - xj[d];
                dd2[d] = dd * dd;
                r2 += dd2[d];
            }
            float k, psi;
            Entry<KIND>::k_psi(r2, a.log2s2, k, psi);
            const float pm = psi * m;
#pragma unroll
            for (int d = 0; d < D; ++d) acc[d] = fmaf(pm, dd2[d], acc[d]);
            acc[D] = fmaf(k, m, acc[D]);
        }
#pragma unroll
        for (int p = 0; p < NB; ++p) kahan_add(tot[p], comp[p], acc[p]);
    }

    // Block reduction in float64 (fixed order: shuffle tree, then warps in index order).
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int p = 0; p < NB; ++p) {
        double v = (double)tot[p] - (double)comp[p];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][p] = v;
    }
    __syncthreads();
    if (tid < NB) {
        double s = 0.0;
        for (int w = 0; w < kSimtThreads / 32; ++w) s += red[w][tid];
        a.partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * NB + tid] = s;
    }
}

// Kind-specific dispatchers (one translation unit per kernel kind).
cudaError_t mv_simt_dispatch_rbf(int D, int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st);
cudaError_t mv_simt_dispatch_m52(int D, int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st);
cudaError_t mv_grad_dispatch_rbf(int D, int TT, dim3 grid, const GradArgs &a, cudaStream_t st);
cudaError_t mv_grad_dispatch_m52(int D, int TT, dim3 grid, const GradArgs &a, cudaStream_t st);
cudaError_t adjoint_dispatch_rbf(int D, int TT, dim3 grid, const AdjArgs &a, cudaStream_t st);
cudaError_t adjoint_dispatch_m52(int D, int TT, dim3 grid, const AdjArgs &a, cudaStream_t st);
cudaError_t mv_simt_dispatch_m12(int D, int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st);
cudaError_t mv_grad_dispatch_m12(int D, int TT, dim3 grid, const GradArgs &a, cudaStream_t st);
cudaError_t adjoint_dispatch_m12(int D, int TT, dim3 grid, const AdjArgs &a, cudaStream_t st);
cudaError_t mv_simt_dispatch_m32(int D, int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st);
cudaError_t mv_grad_dispatch_m32(int D, int TT, dim3 grid, const GradArgs &a, cudaStream_t st);
cudaError_t adjoint_dispatch_m32(int D, int TT, dim3 grid, const AdjArgs &a, cudaStream_t st);

}  // namespace lgp

// Instantiation helper used by the per-kind translation units.
#define LGP_DEFINE_SIMT_DISPATCH(KIND, SUFFIX)                                                                   \
    namespace lgp {                                                                                            \
    template <int D>                                                                                           \
    static cudaError_t mv_simt_d_##SUFFIX(int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st) {      \
        if (TT == 1 && R == 4) mv_simt_kernel<KIND, D, 1, 4><<<grid, kSimtThreads, 0, st>>>(a);                \
        else if (TT == 2 && R == 4) mv_simt_kernel<KIND, D, 2, 4><<<grid, kSimtThreads, 0, st>>>(a);           \
        else if (TT == 4 && R == 4) mv_simt_kernel<KIND, D, 4, 4><<<grid, kSimtThreads, 0, st>>>(a);           \
        else if (TT == 8 && R == 2) mv_simt_kernel<KIND, D, 8, 2><<<grid, kSimtThreads, 0, st>>>(a);           \
        else if (TT == 16 && R == 1) mv_simt_kernel<KIND, D, 16, 1><<<grid, kSimtThreads, 0, st>>>(a);         \
        else if (TT == 32 && R == 1) mv_simt_kernel<KIND, D, 32, 1><<<grid, kSimtThreads, 0, st>>>(a);         \
        else return cudaErrorInvalidValue;                                                                     \
        return cudaGetLastError();                                                                             \
    }                                                                                                          \
    cudaError_t mv_simt_dispatch_##SUFFIX(int D, int TT, int R, dim3 grid, const SimtArgs &a, cudaStream_t st) { \
        switch (D) {                                                                                           \
            case 1: return mv_simt_d_##SUFFIX<1>(TT, R, grid, a, st);                                          \
            case 2: return mv_simt_d_##SUFFIX<2>(TT, R, grid, a, st);                                          \
            case 3: return mv_simt_d_##SUFFIX<3>(TT, R, grid, a, st);                                          \
            case 4: return mv_simt_d_##SUFFIX<4>(TT, R, grid, a, st);                                          \
            case 5: return mv_simt_d_##SUFFIX<5>(TT, R, grid, a, st);                                          \
            case 6: return mv_simt_d_##SUFFIX<6>(TT, R, grid, a, st);                                          \
            case 7: return mv_simt_d_##SUFFIX<7>(TT, R, grid, a, st);                                          \
            case 8: return mv_simt_d_##SUFFIX<8>(TT, R, grid, a, st);                                          \
        }                                                                                                      \
        return cudaErrorInvalidValue;                                                                          \
    }                                                                                                          \
    template <int D>                                                                                           \
    static cudaError_t mv_grad_d_##SUFFIX(int TT, dim3 grid, const GradArgs &a, cudaStream_t st) {             \
        if (TT == 1) mv_grad_kernel<KIND, D, 1><<<grid, kSimtThreads, 0, st>>>(a);                             \
        else if (TT == 4) mv_grad_kernel<KIND, D, 4><<<grid, kSimtThreads, 0, st>>>(a);                        \
        else return cudaErrorInvalidValue;                                                                     \
        return cudaGetLastError();                                                                             \
    }                                                                                                          \
    cudaError_t mv_grad_dispatch_##SUFFIX(int D, int TT, dim3 grid, const GradArgs &a, cudaStream_t st) {      \
        switch (D) {                                                                                           \
            case 1: return mv_grad_d_##SUFFIX<1>(TT, grid, a, st);                                             \
            case 2: return mv_grad_d_##SUFFIX<2>(TT, grid, a, st);                                             \
            case 3: return mv_grad_d_##SUFFIX<3>(TT, grid, a, st);                                             \
            case 4: return mv_grad_d_##SUFFIX<4>(TT, grid, a, st);                                             \
            case 5: return mv_grad_d_##SUFFIX<5>(TT, grid, a, st);                                             \
            case 6: return mv_grad_d_##SUFFIX<6>(TT, grid, a, st);                                             \
            case 7: return mv_grad_d_##SUFFIX<7>(TT, grid, a, st);                                             \
            case 8: return mv_grad_d_##SUFFIX<8>(TT, grid, a, st);                                             \
        }                                                                                                      \
        return cudaErrorInvalidValue;                                                                          \
    }                                                                                                          \
    template <int D>                                                                                           \
    static cudaError_t adjoint_d_##SUFFIX(int TT, dim3 grid, const AdjArgs &a, cudaStream_t st) {              \
        switch (TT) {                                                                                          \
            case 1: adjoint_bilinear_kernel<KIND, D, 1><<<grid, kSimtThreads, 0, st>>>(a); break;              \
            case 2: adjoint_bilinear_kernel<KIND, D, 2><<<grid, kSimtThreads, 0, st>>>(a); break;              \
            case 4: adjoint_bilinear_kernel<KIND, D, 4><<<grid, kSimtThreads, 0, st>>>(a); break;              \
            case 8: adjoint_bilinear_kernel<KIND, D, 8><<<grid, kSimtThreads, 0, st>>>(a); break;              \
            case 16: adjoint_bilinear_kernel<KIND, D, 16><<<grid, kSimtThreads, 0, st>>>(a); break;            \
            case 32: adjoint_bilinear_kernel<KIND, D, 32><<<grid, kSimtThreads, 0, st>>>(a); break;            \
            case 64: adjoint_bilinear_kernel<KIND, D, 64><<<grid, kSimtThreads, 0, st>>>(a); break;            \
            default: return cudaErrorInvalidValue;                                                             \
        }                                                                                                      \
        return cudaGetLastError();                                                                             \
    }                                                                                                          \
    cudaError_t adjoint_dispatch_##SUFFIX(int D, int TT, dim3 grid, const AdjArgs &a, cudaStream_t st) {       \
        switch (D) {                                                                                           \
            case 1: return adjoint_d_##SUFFIX<1>(TT, grid, a, st);                                             \
            case 2: return adjoint_d_##SUFFIX<2>(TT, grid, a, st);                                             \
            case 3: return adjoint_d_##SUFFIX<3>(TT, grid, a, st);                                             \
            case 4: return adjoint_d_##SUFFIX<4>(TT, grid, a, st);                                             \
            case 5: return adjoint_d_##SUFFIX<5>(TT, grid, a, st);                                             \
            case 6: return adjoint_d_##SUFFIX<6>(TT, grid, a, st);                                             \
            case 7: return adjoint_d_##SUFFIX<7>(TT, grid, a, st);                                             \
            case 8: return adjoint_d_##SUFFIX<8>(TT, grid, a, st);                                             \
        }                                                                                                      \
        return cudaErrorInvalidValue;                                                                          \
    }                                                                                                          \
    }  // namespace lgp
