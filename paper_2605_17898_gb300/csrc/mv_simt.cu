// Host launchers of the FP32 SIMT product family: tile choice, column splits and the split reductions.
#include <algorithm>

#include "mv_simt.cuh"

namespace lgp {

namespace {

struct SimtShape {
    int TT, R;
};

SimtShape simt_shape(int t) {
    if (t == 1) return {1, 4};
    if (t == 2) return {2, 4};
    if (t <= 4) return {4, 4};
    if (t <= 8) return {8, 2};
    if (t <= 16) return {16, 1};
    return {32, 1};
}

// Column splits so that row blocks x splits x column groups fill the GPU a few
// times over; each split covers a whole number of BN tiles.
int64_t choose_split(int64_t N, int64_t row_blocks, int64_t col_groups, int num_sms, int64_t *cols_per_split) {
    const int64_t col_tiles = (N + kSimtBN - 1) / kSimtBN;
    const int64_t want = (int64_t)num_sms * 8;
    int64_t s = (want + row_blocks * col_groups - 1) / (row_blocks * col_groups);
    s = std::max<int64_t>(1, std::min<int64_t>(s, std::max<int64_t>(1, col_tiles / 4)));
    const int64_t tiles_per = (col_tiles + s - 1) / s;
    *cols_per_split = tiles_per * kSimtBN;
    return (N + *cols_per_split - 1) / *cols_per_split;
}

// Rows are the output's (N, padded Np); cross = 1 drops the noise term (V has other rows).
__global__ void reduce_split_kernel(const float *__restrict__ partial, int S, int64_t Np, int64_t N, int t,
                                    const float *__restrict__ V, int64_t ldv, float *__restrict__ out, int64_t ldo,
                                    float noise, int cross, const int *skip) {
    if (skip && *skip) return;
    const int64_t total = N * t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        float s = 0.0f;
        for (int k = 0; k < S; ++k) s += partial[((int64_t)k * Np + i) * t + c];
        out[i * ldo + c] = cross ? s : fmaf(noise, V[i * ldv + c], s);
    }
}

__global__ void reduce_grad_kernel(const float *__restrict__ partial, int S, int NB, int64_t Np, int64_t N, int t,
                                   const float *__restrict__ W, float noise, float *__restrict__ G) {
    const int64_t total = (int64_t)(NB + 1) * N * t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / (N * t);
        const int64_t rem = e - p * N * t;
        const int64_t i = rem / t;
        const int c = (int)(rem - i * t);
        if (p == NB) {
            G[e] = noise * W[i * t + c];
            continue;
        }
        float s = 0.0f;
        for (int k = 0; k < S; ++k) s += partial[(((int64_t)k * NB + p) * Np + i) * t + c];
        G[e] = s;
    }
}

inline int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

}  // namespace

int64_t mv_simt_partial_floats(int64_t N, int64_t Np, int t, int num_sms) {
    const SimtShape sh = simt_shape(t);
    const int64_t BM = (int64_t)kSimtThreads * sh.R;
    const int64_t rb = (N + BM - 1) / BM;
    const int64_t cg = (t + sh.TT - 1) / sh.TT;
    int64_t cps;
    const int64_t S = choose_split(N, rb, cg, num_sms, &cps);
    return S > 1 ? S * Np * t : 0;
}

int64_t mv_simt_cross_partial_floats(int64_t Nr, int64_t Npr, int64_t N, int t, int num_sms) {
    const SimtShape sh = simt_shape(t);
    const int64_t BM = (int64_t)kSimtThreads * sh.R;
    const int64_t rb = (Nr + BM - 1) / BM;
    const int64_t cg = (t + sh.TT - 1) / sh.TT;
    int64_t cps;
    const int64_t S = choose_split(N, rb, cg, num_sms, &cps);
    return S > 1 ? S * Npr * t : 0;
}

int mv_simt_launches(int64_t N, int64_t Np, int t, int num_sms) {
    return mv_simt_partial_floats(N, Np, t, num_sms) > 0 ? 2 : 1;
}

cudaError_t launch_mv_simt(const MvLaunch &m, cudaStream_t st) {
    const bool cross = m.Xr != nullptr;
    const int64_t Nr = cross ? m.Nr : m.N, Npr = cross ? m.Npr : m.Np;
    const SimtShape sh = simt_shape(m.t);
    const int64_t BM = (int64_t)kSimtThreads * sh.R;
    const int64_t rb = (Nr + BM - 1) / BM;
    const int64_t cg = (m.t + sh.TT - 1) / sh.TT;
    int64_t cps;
    int64_t S = choose_split(m.N, rb, cg, m.num_sms, &cps);
    if (S > 1 && (m.partial == nullptr || S * Npr * m.t > m.partial_cap)) {
        S = 1;
        cps = m.N;
    }
    SimtArgs a;
    a.Xs = m.Xs;
    a.Xr = cross ? m.Xr : m.Xs;
    a.Nr = Nr;
    a.Npr = Npr;
    a.cross = cross ? 1 : 0;
    a.V = m.V;
    a.out = m.out;
    a.partial = S > 1 ? m.partial : nullptr;
    a.skip = m.skip;
    a.N = m.N;
    a.Np = m.Np;
    a.ldv = m.ldv;
    a.ldo = m.ldo;
    a.cols_per_split = cps;
    a.t = m.t;
    a.log2s2 = m.kp->log2_s2;
    a.noise = m.kp->noise;
    const dim3 grid((unsigned)rb, (unsigned)S, (unsigned)cg);
    cudaError_t e;
    switch (m.kp->kind) {
        case LGP_RBF: e = mv_simt_dispatch_rbf(m.kp->D, sh.TT, sh.R, grid, a, st); break;
        case LGP_MATERN52: e = mv_simt_dispatch_m52(m.kp->D, sh.TT, sh.R, grid, a, st); break;
        case LGP_MATERN12: e = mv_simt_dispatch_m12(m.kp->D, sh.TT, sh.R, grid, a, st); break;
        case LGP_MATERN32: e = mv_simt_dispatch_m32(m.kp->D, sh.TT, sh.R, grid, a, st); break;
        default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || S == 1) return e;
    reduce_split_kernel<<<grid_for(Nr * m.t), 256, 0, st>>>(m.partial, (int)S, Npr, Nr, m.t, m.V, m.ldv, m.out,
                                                            m.ldo, m.kp->noise, a.cross, m.skip);
    return cudaGetLastError();
}

int64_t mv_grad_partial_floats(int64_t N, int64_t Np, int t, int D, int num_sms) {
    const int TT = t == 1 ? 1 : 4;
    const int64_t rb = (N + kSimtThreads - 1) / kSimtThreads;
    const int64_t cg = (t + TT - 1) / TT;
    int64_t cps;
    const int64_t S = choose_split(N, rb, cg, num_sms, &cps);
    return S > 1 ? S * (D + 1) * Np * t : 0;
}

cudaError_t launch_mv_grad(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *W, int t,
                           float *G, float *partial, int64_t partial_cap, int num_sms, cudaStream_t st) {
    const int TT = t == 1 ? 1 : 4;
    const int64_t rb = (N + kSimtThreads - 1) / kSimtThreads;
    const int64_t cg = (t + TT - 1) / TT;
    int64_t cps;
    int64_t S = choose_split(N, rb, cg, num_sms, &cps);
    const int NB = kp.D + 1;
    if (S > 1 && (partial == nullptr || S * NB * Np * t > partial_cap)) {
        S = 1;
        cps = N;
    }
    GradArgs a;
    a.Xs = Xs;
    a.W = W;
    a.G = G;
    a.partial = S > 1 ? partial : nullptr;
    a.N = N;
    a.Np = Np;
    a.cols_per_split = cps;
    a.t = t;
    a.log2s2 = kp.log2_s2;
    a.noise = kp.noise;
    const dim3 grid((unsigned)rb, (unsigned)S, (unsigned)cg);
    cudaError_t e;
    switch (kp.kind) {
        case LGP_RBF: e = mv_grad_dispatch_rbf(kp.D, TT, grid, a, st); break;
        case LGP_MATERN52: e = mv_grad_dispatch_m52(kp.D, TT, grid, a, st); break;
        case LGP_MATERN12: e = mv_grad_dispatch_m12(kp.D, TT, grid, a, st); break;
        case LGP_MATERN32: e = mv_grad_dispatch_m32(kp.D, TT, grid, a, st); break;
        default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || S == 1) return e;
    reduce_grad_kernel<<<grid_for((int64_t)(NB + 1) * N * t), 256, 0, st>>>(partial, (int)S, NB, Np, N, t, W,
                                                                           kp.noise, G);
    return cudaGetLastError();
}

static int adjoint_tt(int t) {
    int TT = 1;
    while (TT < t) TT *= 2;
    return TT;
}

int64_t adjoint_partial_doubles(int64_t N, int t, int D, int num_sms) {
    const int64_t rb = (N + kSimtThreads - 1) / kSimtThreads;
    int64_t cps;
    const int64_t S = choose_split(N, rb, 1, num_sms, &cps);
    return rb * S * (D + 1);
}

cudaError_t launch_adjoint_bilinear(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *A,
                                    const float *B, int t, double *block_partials, int64_t partial_cap, int *n_blocks,
                                    int num_sms, cudaStream_t st) {
    const int64_t rb = (N + kSimtThreads - 1) / kSimtThreads;
    int64_t cps;
    const int64_t S = choose_split(N, rb, 1, num_sms, &cps);
    if (rb * S * (kp.D + 1) > partial_cap) return cudaErrorInvalidValue;
    AdjArgs a;
    a.Xs = Xs;
    a.A = A;
    a.B = B;
    a.partial = block_partials;
    a.N = N;
    a.Np = Np;
    a.cols_per_split = cps;
    a.t = t;
    a.log2s2 = kp.log2_s2;
    *n_blocks = (int)(rb * S);
    const dim3 grid((unsigned)rb, (unsigned)S, 1);
    const int TT = adjoint_tt(t);
    switch (kp.kind) {
        case LGP_RBF: return adjoint_dispatch_rbf(kp.D, TT, grid, a, st);
        case LGP_MATERN52: return adjoint_dispatch_m52(kp.D, TT, grid, a, st);
        case LGP_MATERN12: return adjoint_dispatch_m12(kp.D, TT, grid, a, st);
        case LGP_MATERN32: return adjoint_dispatch_m32(kp.D, TT, grid, a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lgp
