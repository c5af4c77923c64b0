// Many independent GP solves of uneven size advanced together.
//
// Per CG iteration, one persistent launch computes K_y(g) p(g) for every problem g:
// its CTAs pull work items (problem, block of 256 rows) from a list sorted by cost
// (longest first) through an atomic counter, so large and small problems share the
// GPU without one launch per problem. Problems whose columns have all converged are
// skipped. The vector updates and the float64 scalar recurrences then run as segmented
// versions of the single-problem CG kernels: every vector block belongs to one problem,
// and each (problem, column) scalar is reduced from that problem's block partials in a
// fixed order, so the results do not depend on which CTA took which item.
#include "batch.cuh"
#include "mv_simt.cuh"

namespace lgp {

namespace {

constexpr int kBatchThreads = 128;
constexpr int kBatchR = 2;
constexpr int kBatchBM = kBatchThreads * kBatchR;

// One 256-row block of one problem: K_y p for those rows over all of the problem's columns. The
// distance runs over the problem's own D coordinates (the rows are stored padded to DP).
template <int KIND, int D, int TT>
__device__ void batch_item(const BatchGp &g, int64_t row0, int split, const float *__restrict__ Xs_all,
                           const float *__restrict__ p_all, float *__restrict__ kp_all, float *__restrict__ part,
                           int t, float *xs, float *vs) {
    constexpr int DP = D <= 4 ? 4 : 8;
    const int tid = threadIdx.x;
    const float *Xs = Xs_all + g.xs_off;
    const float *V = p_all + g.vec_off * t;
    float *out = kp_all + g.vec_off * t;
    float xi[kBatchR][D];
    float tot[kBatchR][TT];
#pragma unroll
    for (int r = 0; r < kBatchR; ++r) {
        const int64_t i = row0 + r * kBatchThreads + tid;
#pragma unroll
        for (int d = 0; d < D; ++d) xi[r][d] = (i < g.Np) ? Xs[i * DP + d] : 0.0f;
#pragma unroll
        for (int c = 0; c < TT; ++c) tot[r][c] = 0.0f;
    }
    const int64_t jb = (int64_t)split * g.cols_per_split;
    const int64_t je = min(g.N, jb + g.cols_per_split);
    for (int64_t j0 = jb; j0 < je; j0 += kSimtBN) {
        __syncthreads();
        for (int e = tid; e < kSimtBN * DP / 4; e += kBatchThreads) {
            const int64_t j = j0 + (e * 4) / DP;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < g.Np) v = *reinterpret_cast<const float4 *>(Xs + j0 * DP + e * 4);
            *reinterpret_cast<float4 *>(xs + e * 4) = v;
        }
        for (int e = tid; e < kSimtBN * TT; e += kBatchThreads) {
            const int jj = e / TT;
            const int c = e - jj * TT;
            const int64_t j = j0 + jj;
            vs[e] = (j < je && c < t) ? V[j * t + c] : 0.0f;
        }
        __syncthreads();
        float acc[kBatchR][TT];
#pragma unroll
        for (int r = 0; r < kBatchR; ++r)
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
                    v[c] = q.x;
                    v[(c + 1) % TT] = q.y;
                    v[(c + 2) % TT] = q.z;
                    v[(c + 3) % TT] = q.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < TT; ++c) v[c] = vs[jj * TT + c];
            }
#pragma unroll
            for (int r = 0; r < kBatchR; ++r) {
                const float k = Entry<KIND>::k(sqdist<D>(xi[r], xj), g.log2s2);
#pragma unroll
                for (int c = 0; c < TT; ++c) acc[r][c] = fmaf(k, v[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int r = 0; r < kBatchR; ++r)
#pragma unroll
            for (int c = 0; c < TT; ++c) tot[r][c] += acc[r][c];
    }
#pragma unroll
    for (int r = 0; r < kBatchR; ++r) {
        const int64_t i = row0 + r * kBatchThreads + tid;
        if (i >= g.N) continue;
        if (g.splits > 1) {
            float *dst = part + g.part_off + ((int64_t)split * g.Np + i) * t;
#pragma unroll
            for (int c = 0; c < TT; ++c)
                if (c < t) dst[c] = tot[r][c];
        } else {
#pragma unroll
            for (int c = 0; c < TT; ++c)
                if (c < t) out[i * t + c] = fmaf(g.noise, V[i * t + c], tot[r][c]);
        }
    }
}

template <int KIND, int TT>
__device__ __forceinline__ void batch_item_d(const BatchGp &g, int64_t row0, int split, const BatchArgs &a, float *xs,
                                             float *vs) {
    switch (g.D) {
        case 1: batch_item<KIND, 1, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 2: batch_item<KIND, 2, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 3: batch_item<KIND, 3, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 4: batch_item<KIND, 4, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 5: batch_item<KIND, 5, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 6: batch_item<KIND, 6, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        case 7: batch_item<KIND, 7, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs); break;
        default: batch_item<KIND, 8, TT>(g, row0, split, a.Xs, a.p, a.kp, a.part, a.t, xs, vs);
    }
}

template <int TT>
__global__ void __launch_bounds__(kBatchThreads) batch_mv_kernel(BatchArgs a) {
    __shared__ __align__(16) float xs[kSimtBN * 8];
    __shared__ __align__(16) float vs[kSimtBN * TT];
    __shared__ int item_s;
    if (a.done && *a.done) return;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = atomicAdd(a.item_counter, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= a.n_items) break;
        const BatchItem it = a.items[item];
        if (a.gp_done[it.gp]) continue;
        const BatchGp g = a.gps[it.gp];
        const int64_t row0 = (int64_t)it.row_block * kBatchBM;
        switch (g.kind) {
            case LGP_RBF: batch_item_d<LGP_RBF, TT>(g, row0, it.split, a, xs, vs); break;
            case LGP_MATERN52: batch_item_d<LGP_MATERN52, TT>(g, row0, it.split, a, xs, vs); break;
            case LGP_MATERN12: batch_item_d<LGP_MATERN12, TT>(g, row0, it.split, a, xs, vs); break;
            default: batch_item_d<LGP_MATERN32, TT>(g, row0, it.split, a, xs, vs);
        }
    }
}

// ---------------------------------------------------------------- segmented CG kernels

constexpr int kVec = 256;

__device__ void seg_col_reduce(double v, int t, double *red, double *out_row) {
    const int tid = threadIdx.x;
    const int nr = blockDim.x / t;
    red[tid] = v;
    __syncthreads();
    int s = 1;
    while (s < nr) s <<= 1;
    for (s >>= 1; s >= 1; s >>= 1) {
        const int slot = tid / t;
        if (slot < s && slot + s < nr) red[tid] += red[tid + s * t];
        __syncthreads();
    }
    if (tid < t) out_row[tid] = red[tid];
}

__global__ void binit_kernel(BatchArgs a) {
    __shared__ double red[kVec];
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    const int t = a.t;
    const int c = threadIdx.x % t;
    double s = 0.0;
    for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t) {
        const float b = g.B[i * t + c];
        const int64_t e = (g.vec_off + i) * t + c;
        a.x[e] = 0.0f;
        a.r[e] = b;
        a.p[e] = b;
        s += (double)b * (double)b;
    }
    seg_col_reduce(s, t, red, a.partial + (int64_t)blockIdx.x * t);
}

__global__ void bscal_init_kernel(BatchArgs a, double tol, int max_iter) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        a.st->iter = 0;
        a.st->max_iter = max_iter;
        a.st->tol = tol;
        a.st->status = 0;
        a.st->loop_chunks = 0;
        a.st->max_chunks = max_iter / 8 + 2;
    }
    if (k >= a.n_gp * a.t) return;
    const int gi = k / a.t, c = k % a.t;
    const BatchGp g = a.gps[gi];
    double s = 0.0;
    for (int b = g.blk0; b < g.blk1; ++b) s += a.partial[(int64_t)b * a.t + c];
    a.bnorm2[k] = s;
    a.rr[k] = s;
    a.alpha[k] = 0.0;
    a.beta[k] = 0.0;
    a.iters[k] = 0;
    const bool bad = !isfinite(s);
    a.active[k] = (s > 0.0) && !bad;
    if (bad) atomicOr(&a.st->status, 1);
}

__global__ void bdone_kernel(BatchArgs a, int first) {
    __shared__ int any_s;
    if (threadIdx.x == 0) any_s = 0;
    __syncthreads();
    if (!first && *a.done) return;
    int any = 0;
    for (int gi = threadIdx.x; gi < a.n_gp; gi += blockDim.x) {
        int act = 0;
        for (int c = 0; c < a.t; ++c) act |= a.active[gi * a.t + c];
        a.gp_done[gi] = !act;
        any |= act;
    }
    if (any) atomicOr(&any_s, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!first) a.st->iter += 1;
        *a.done = (!any_s || a.st->iter >= a.st->max_iter || (first && a.st->status)) ? 1 : 0;
    }
}

// K_y p for problems whose product was split over columns: the partial sums in split order plus
// sigma^2 p (one vector block per CTA).
__global__ void bsplit_reduce_kernel(BatchArgs a) {
    if (*a.done) return;
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    if (g.splits <= 1 || a.gp_done[vb.gp]) return;
    const int t = a.t;
    const int c = threadIdx.x % t;
    for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t) {
        float sum = 0.0f;
        for (int k = 0; k < g.splits; ++k) sum += a.part[g.part_off + ((int64_t)k * g.Np + i) * t + c];
        const int64_t e = (g.vec_off + i) * t + c;
        a.kp[e] = fmaf(g.noise, a.p[e], sum);
    }
}

__global__ void bpkp_kernel(BatchArgs a) {
    __shared__ double red[kVec];
    if (*a.done) return;
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    const int t = a.t;
    const int c = threadIdx.x % t;
    float hi = 0.0f, lo = 0.0f;
    if (!a.gp_done[vb.gp]) {
        for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t) {
            const int64_t e = (g.vec_off + i) * t + c;
            acc_prod2(hi, lo, a.p[e], a.kp[e]);
        }
    }
    seg_col_reduce((double)hi + (double)lo, t, red, a.partial + (int64_t)blockIdx.x * t);
}

__global__ void balpha_kernel(BatchArgs a) {
    if (*a.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n_gp * a.t) return;
    const int gi = k / a.t, c = k % a.t;
    double alpha = 0.0;
    if (a.active[k]) {
        const BatchGp g = a.gps[gi];
        double pkp = 0.0;
        for (int b = g.blk0; b < g.blk1; ++b) pkp += a.partial[(int64_t)b * a.t + c];
        if (!isfinite(pkp) || !(pkp > 0.0)) {
            a.active[k] = 0;
            atomicOr(&a.st->status, isfinite(pkp) ? 2 : 1);
        } else {
            alpha = a.rr[k] / pkp;
        }
    }
    a.alpha[k] = alpha;
}

__global__ void bxr_kernel(BatchArgs a) {
    __shared__ double red[kVec];
    if (*a.done) return;
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    const int t = a.t;
    const int c = threadIdx.x % t;
    const float alpha = (float)a.alpha[vb.gp * t + c];
    float hi = 0.0f, lo = 0.0f;
    for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t) {
        const int64_t e = (g.vec_off + i) * t + c;
        float rv = a.r[e];
        if (alpha != 0.0f) {
            a.x[e] = fmaf(alpha, a.p[e], a.x[e]);
            rv = fmaf(-alpha, a.kp[e], rv);
            a.r[e] = rv;
        }
        acc_prod2(hi, lo, rv, rv);
    }
    seg_col_reduce((double)hi + (double)lo, t, red, a.partial + (int64_t)blockIdx.x * t);
}

__global__ void bbeta_kernel(BatchArgs a) {
    if (*a.done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n_gp * a.t) return;
    const int gi = k / a.t, c = k % a.t;
    double beta = 0.0;
    if (a.active[k]) {
        const BatchGp g = a.gps[gi];
        double rr = 0.0;
        for (int b = g.blk0; b < g.blk1; ++b) rr += a.partial[(int64_t)b * a.t + c];
        beta = rr / a.rr[k];
        a.rr[k] = rr;
        a.iters[k] += 1;
        if (!(sqrt(rr) > a.st->tol * sqrt(a.bnorm2[k]))) a.active[k] = 0;
    }
    a.beta[k] = beta;
}

__global__ void bp_kernel(BatchArgs a) {
    if (*a.done) return;
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    const int t = a.t;
    const int c = threadIdx.x % t;
    if (!a.active[vb.gp * t + c]) return;
    const float beta = (float)a.beta[vb.gp * t + c];
    for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t) {
        const int64_t e = (g.vec_off + i) * t + c;
        a.p[e] = fmaf(beta, a.p[e], a.r[e]);
    }
}

__global__ void bcopy_out_kernel(BatchArgs a) {
    const BatchVecBlock vb = a.vblocks[blockIdx.x];
    const BatchGp g = a.gps[vb.gp];
    const int t = a.t;
    const int c = threadIdx.x % t;
    for (int64_t i = vb.r0 + threadIdx.x / t; i < vb.r1; i += blockDim.x / t)
        g.Xsol[i * t + c] = a.x[(g.vec_off + i) * t + c];
}

__global__ void batch_loop_condition_kernel(cudaGraphConditionalHandle h, BatchArgs a) {
    a.st->loop_chunks += 1;
    const bool more = !*a.done && a.st->loop_chunks < a.st->max_chunks;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

inline int vec_threads(int t) { return (kVec / t) * t; }

}  // namespace

int batch_item_rows() { return kBatchBM; }

cudaError_t launch_batch_init(const BatchArgs &a, double tol, int max_iter, cudaStream_t st) {
    binit_kernel<<<a.n_vblocks, vec_threads(a.t), 0, st>>>(a);
    const int n = a.n_gp * a.t;
    bscal_init_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, tol, max_iter);
    bdone_kernel<<<1, 256, 0, st>>>(a, 1);
    return cudaGetLastError();
}

cudaError_t launch_batch_product(const BatchArgs &a, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.item_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(a.n_items, num_sms * 6));
    switch (a.tt) {
        case 1: batch_mv_kernel<1><<<grid, kBatchThreads, 0, st>>>(a); break;
        case 2: batch_mv_kernel<2><<<grid, kBatchThreads, 0, st>>>(a); break;
        case 4: batch_mv_kernel<4><<<grid, kBatchThreads, 0, st>>>(a); break;
        case 8: batch_mv_kernel<8><<<grid, kBatchThreads, 0, st>>>(a); break;
        case 16: batch_mv_kernel<16><<<grid, kBatchThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    bsplit_reduce_kernel<<<a.n_vblocks, vec_threads(a.t), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(const BatchArgs &a, int num_sms, cudaStream_t st) {
    cudaError_t e = launch_batch_product(a, num_sms, st);
    if (e != cudaSuccess) return e;
    const int n = a.n_gp * a.t;
    const int sb = (n + 255) / 256;
    const int vt = vec_threads(a.t);
    bpkp_kernel<<<a.n_vblocks, vt, 0, st>>>(a);
    balpha_kernel<<<sb, 256, 0, st>>>(a);
    bxr_kernel<<<a.n_vblocks, vt, 0, st>>>(a);
    bbeta_kernel<<<sb, 256, 0, st>>>(a);
    bdone_kernel<<<1, 256, 0, st>>>(a, 0);
    bp_kernel<<<a.n_vblocks, vt, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_loop_condition(cudaGraphConditionalHandle h, const BatchArgs &a, cudaStream_t st) {
    batch_loop_condition_kernel<<<1, 1, 0, st>>>(h, a);
    return cudaGetLastError();
}

cudaError_t launch_batch_copy_out(const BatchArgs &a, cudaStream_t st) {
    bcopy_out_kernel<<<a.n_vblocks, vec_threads(a.t), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lgp
