// Conjugate-gradient vector updates, float64 scalar recurrences, stochastic Lanczos
// quadrature and the LML / gradient assembly.
//
// CG (Sec. 2 "CG-based inference"; Sec. 5 "our simpler CG loop"): x0 = 0, one recurrence per
// right-hand-side column, all columns advanced by the same launches. Per iteration, after
// Kp = K_y p, with z = P^{-1} r (z = r without a preconditioner):
//   alpha_c = r_c^T z_c / p_c^T Kp_c,  x_c += alpha_c p_c,  r_c -= alpha_c Kp_c,
//   z_c' = P^{-1} r_c',  beta_c = r_c'^T z_c' / r_c^T z_c,  p_c = z_c' + beta_c p_c,
// column c stops once ||r_c|| <= tol ||b_c||. The optional preconditioner is the pivoted-Cholesky
// P of precond.cu (the gap Sec. 5 names; plain CG is the paper's loop). Vectors are float32; the dot products
// are accumulated in float64 with a fixed reduction order (block partials, then one
// block sums them in index order), so results are reproducible run to run.
#include <math.h>

#include "lgp_internal.cuh"

namespace lgp {

namespace {

constexpr int kVecThreads = 256;

// Threads per block for column-interleaved work: a multiple of t not above 256.
__host__ __device__ inline int vec_block(int t) { return (kVecThreads / t) * t; }

// Block-level per-column reduction of vals (one per thread, column tid % t) into out[c].
__device__ void block_col_reduce(double v, int t, double *red, double *out_row) {
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

// Sum of partial[b * stride + c] over b < G by one warp: lane l adds b = l, l + 32, ... in order,
// then a fixed shuffle tree combines the lanes (same order every call).
__device__ __forceinline__ double warp_sum_partials(const double *__restrict__ partial, int G, int stride, int c) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += partial[(int64_t)b * stride + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    return __shfl_sync(0xffffffffu, s, 0);
}

// Row range of block b when G blocks share N rows.
__device__ __forceinline__ void block_rows(int64_t N, int64_t *r0, int64_t *r1) {
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    *r0 = min(N, (int64_t)blockIdx.x * per);
    *r1 = min(N, *r0 + per);
}

__global__ void cg_init_kernel(const float *__restrict__ B, int64_t ldb, int64_t N, int t, float *__restrict__ x,
                               float *__restrict__ r, float *__restrict__ p, double *__restrict__ partial) {
    __shared__ double red[kVecThreads];
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const float b = B[i * ldb + c];
        x[i * t + c] = 0.0f;
        r[i * t + c] = b;
        p[i * t + c] = b;
        s += (double)b * (double)b;
    }
    block_col_reduce(s, t, red, partial + (int64_t)blockIdx.x * t);
}

// Warm start: x = x0, r = b - K_y x0 (KX0 = K_y x0 computed before), p = r; block partials of
// b^T b (partial) and r^T r (rr_partial).
__global__ void cg_init_x0_kernel(const float *__restrict__ B, int64_t ldb, const float *__restrict__ X0, int64_t ldx0,
                                  const float *__restrict__ KX0, int64_t N, int t, float *__restrict__ x,
                                  float *__restrict__ r, float *__restrict__ p, double *__restrict__ partial,
                                  double *__restrict__ rr_partial) {
    __shared__ double red[kVecThreads];
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    double sb = 0.0, sr = 0.0;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const float b = B[i * ldb + c];
        const float rv = b - KX0[i * t + c];
        x[i * t + c] = X0[i * ldx0 + c];
        r[i * t + c] = rv;
        p[i * t + c] = rv;
        sb += (double)b * (double)b;
        sr += (double)rv * (double)rv;
    }
    block_col_reduce(sb, t, red, partial + (int64_t)blockIdx.x * t);
    __syncthreads();
    block_col_reduce(sr, t, red, rr_partial + (int64_t)blockIdx.x * t);
}

// Scalar kernels run as one block of 32 * min(t, 32) threads: warp w owns columns w, w + 32.
__global__ void cg_init_scalars_kernel(CgState *st, const double *__restrict__ partial, int G, int t, double tol,
                                       int max_iter, int hist_len, const double *__restrict__ rz_partial,
                                       const double *__restrict__ rr_partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int any = 0;
    int bad = 0;
    for (int c = warp; c < t; c += nw) {
        const double s = warp_sum_partials(partial, G, t, c);
        const double rr0 = rr_partial ? warp_sum_partials(rr_partial, G, t, c) : s;
        const double rz = rz_partial ? warp_sum_partials(rz_partial, G, t, c) : rr0;
        if (lane != 0) continue;
        st->bnorm2[c] = s;
        st->rr[c] = rr0;
        st->rz[c] = rz;
        st->w0[c] = rz;
        st->alpha[c] = 0.0;
        st->beta[c] = 0.0;
        st->iters[c] = 0;
        const int b_ = !isfinite(s) || !isfinite(rz) || !isfinite(rr0);
        bad |= b_;
        // a warm start that already meets the tolerance leaves the column inactive
        const int act = (s > 0.0) && (rz > 0.0) && !b_ && (sqrt(rr0) > tol * sqrt(s));
        st->active[c] = act;
        any |= act;
    }
    any = __syncthreads_or(any);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        st->iter = 0;
        st->t = t;
        st->tol = tol;
        st->max_iter = max_iter;
        st->hist_len = hist_len;
        st->status = bad ? (int)LGP_ERR_NONFINITE : 0;
        st->done = (!any || bad) ? 1 : 0;
        st->loop_chunks = 0;
        st->max_chunks = max_iter / 8 + 2;
    }
}

__global__ void cg_pkp_kernel(const float *__restrict__ p, const float *__restrict__ Kp, int64_t N, int t,
                              const CgState *st, double *__restrict__ partial) {
    __shared__ double red[kVecThreads];
    if (st->done) return;
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    float hi = 0.0f, lo = 0.0f;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) acc_prod2(hi, lo, p[i * t + c], Kp[i * t + c]);
    block_col_reduce((double)hi + (double)lo, t, red, partial + (int64_t)blockIdx.x * t);
}

__global__ void cg_alpha_kernel(CgState *st, const double *__restrict__ partial, int G, double *hist_alpha) {
    if (st->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int t = st->t;
    int bad = 0, nonfinite = 0;
    for (int c = warp; c < t; c += nw) {
        double alpha = 0.0;
        if (st->active[c]) {
            const double pkp = warp_sum_partials(partial, G, t, c);
            if (lane != 0) continue;
            if (!isfinite(pkp)) {
                nonfinite = 1;
                st->active[c] = 0;
            } else if (!(pkp > 0.0)) {
                bad = 1;
                st->active[c] = 0;
            } else {
                alpha = st->rz[c] / pkp;
            }
        }
        if (lane != 0) continue;
        st->alpha[c] = alpha;
        if (st->iter < st->hist_len) hist_alpha[(int64_t)st->iter * t + c] = alpha;
    }
    bad = __syncthreads_or(bad);
    nonfinite = __syncthreads_or(nonfinite);
    if (threadIdx.x == 0 && (bad || nonfinite) && st->status == 0)
        st->status = nonfinite ? (int)LGP_ERR_NONFINITE : (int)LGP_ERR_BREAKDOWN;
}

__global__ void cg_xr_kernel(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
                             const float *__restrict__ Kp, int64_t N, int t, const CgState *st,
                             double *__restrict__ partial) {
    __shared__ double red[kVecThreads];
    if (st->done) return;
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    const float alpha = (float)st->alpha[c];
    float hi = 0.0f, lo = 0.0f;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const int64_t e = i * t + c;
        float rv = r[e];
        if (alpha != 0.0f) {
            x[e] = fmaf(alpha, p[e], x[e]);
            rv = fmaf(-alpha, Kp[e], rv);
            r[e] = rv;
        }
        acc_prod2(hi, lo, rv, rv);
    }
    block_col_reduce((double)hi + (double)lo, t, red, partial + (int64_t)blockIdx.x * t);
}

__global__ void cg_beta_kernel(CgState *st, const double *__restrict__ partial, int G, double *hist_beta,
                               const double *__restrict__ rz_partial) {
    if (st->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int t = st->t;
    int any = 0;
    for (int c = warp; c < t; c += nw) {
        double beta = 0.0;
        if (st->active[c]) {
            const double rr = warp_sum_partials(partial, G, t, c);
            const double rz = rz_partial ? warp_sum_partials(rz_partial, G, t, c) : rr;
            if (lane != 0) continue;
            beta = rz / st->rz[c];
            st->rr[c] = rr;
            st->rz[c] = rz;
            st->iters[c] += 1;
            if (!(sqrt(rr) > st->tol * sqrt(st->bnorm2[c]))) st->active[c] = 0;
        }
        if (lane != 0) continue;
        st->beta[c] = beta;
        if (st->iter < st->hist_len) hist_beta[(int64_t)st->iter * t + c] = beta;
        any |= st->active[c];
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        st->iter += 1;
        if (!any || st->iter >= st->max_iter) st->done = 1;
    }
}

__global__ void cg_p_kernel(float *__restrict__ p, const float *__restrict__ r, int64_t N, int t,
                            const CgState *st) {
    if (st->done) return;
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    if (!st->active[c]) return;
    const float beta = (float)st->beta[c];
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const int64_t e = i * t + c;
        p[e] = fmaf(beta, p[e], r[e]);
    }
}

__global__ void cg_loop_condition_kernel(cudaGraphConditionalHandle h, CgState *st) {
    st->loop_chunks += 1;
    const bool more = !st->done && st->loop_chunks < st->max_chunks;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Host-driven form of the loop tail (no graph): only counts the chunk.
__global__ void cg_chunk_tally_kernel(CgState *st) { st->loop_chunks += 1; }

// Single-column solves assembled into one t-column result: column 0 of a t = 1 CG run (its state
// and the first hist_len Lanczos coefficients) becomes column c of dst; chunk counts add up.
__global__ void cg_gather_column_kernel(const CgState *__restrict__ src, const double *__restrict__ src_alpha,
                                        const double *__restrict__ src_beta, int hist_len, CgState *dst,
                                        double *__restrict__ dst_alpha, double *__restrict__ dst_beta, int t, int c) {
    for (int k = threadIdx.x; k < hist_len; k += blockDim.x) {
        dst_alpha[(int64_t)k * t + c] = src_alpha[k];
        dst_beta[(int64_t)k * t + c] = src_beta[k];
    }
    if (threadIdx.x == 0) {
        dst->active[c] = src->active[0];
        dst->iters[c] = src->iters[0];
        dst->bnorm2[c] = src->bnorm2[0];
        dst->rr[c] = src->rr[0];
        dst->rz[c] = src->rz[0];
        dst->w0[c] = src->w0[0];
        dst->alpha[c] = src->alpha[0];
        dst->beta[c] = src->beta[0];
        dst->loop_chunks += src->loop_chunks;
        dst->iter = max(dst->iter, src->iter);
        if (src->status != 0 && dst->status == 0) dst->status = src->status;
        dst->t = t;
        dst->hist_len = hist_len;
    }
}

__global__ void copy_out_kernel(const float *__restrict__ x, int64_t N, int t, float *__restrict__ out, int64_t ldo) {
    const int64_t total = N * t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        out[i * ldo + c] = x[e];
    }
}

__global__ void col_dots_kernel(const float *__restrict__ A, const float *__restrict__ B, int64_t N, int t,
                                double *__restrict__ partial) {
    __shared__ double red[kVecThreads];
    int64_t r0, r1;
    block_rows(N, &r0, &r1);
    const int c = threadIdx.x % t;
    double sab = 0.0, saa = 0.0;
    for (int64_t i = r0 + threadIdx.x / t; i < r1; i += blockDim.x / t) {
        const double a = A[i * t + c];
        sab += a * (double)B[i * t + c];
        saa += a * a;
    }
    block_col_reduce(sab, t, red, partial + (int64_t)blockIdx.x * 2 * t);
    __syncthreads();
    block_col_reduce(saa, t, red, partial + (int64_t)blockIdx.x * 2 * t + t);
}

__global__ void col_dots_final_kernel(const double *__restrict__ partial, int G, int t, double *out) {
    const int c = threadIdx.x;
    if (c >= 2 * t) return;
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partial[(int64_t)b * 2 * t + c];
    out[c] = s;
}

// e_1^T log(T) e_1 of each probe's Lanczos tridiagonal, the Gauss quadrature of the stochastic
// log-determinant (Sec. 3 "Inference"), without an eigendecomposition of T. For lambda > 0,
//   log lambda = int_R [s(v) - s(v - log lambda)] dv,   s(v) = 1 / (1 + e^-v),
// so with x = e^v and g(x) = e_1^T (T + x I)^{-1} e_1 = sum_j u_1j^2 / (lambda_j + x),
//   e_1^T log(T) e_1 = int_R [x / (1 + x) - x g(x)] dv.
// The integrand is a sum of differences of logistic functions: analytic in the strip |Im v| < pi
// and decaying like e^-|v| outside [log lambda_min, log lambda_max], so the trapezoidal rule with
// step h on [log lambda_lo - 36, log lambda_hi + 36] has discretisation error ~exp(-2 pi^2 / h)
// (8e-18 at h = 0.5) and truncation error ~e^-36 (Trefethen & Weideman, "The exponentially
// convergent trapezoidal rule", SIAM Review 2014). Bounds: lambda_max <= the Gershgorin bound of T;
// lambda_min >= 1 / tr(T^-1), where T = L D L^T with D = diag(1/alpha_k) and unit lower bidiagonal L
// of subdiagonal sqrt(beta_k) (the CG-Lanczos factorisation), which gives
// tr(T^-1) = sum_i alpha_i s_i, s_0 = 1, s_i = 1 + beta_{i-1} s_{i-1}.
// At each node g(x) = P_2 / P_1 with the trailing minors P_k = det((T + x I)[k:m, k:m]) from the
// division-free recurrence P_k = (a_k + x) P_{k+1} - b_k^2 P_{k+2}, rescaled by powers of two, and
//   x / (1 + x) - x P_2 / P_1 = x ((a_1 - 1) P_2 - b_1^2 P_3) / ((1 + x) P_1)
// (P_1 expanded along its first row), which has no cancellation between the two terms. All of it is
// float64: every thread of the block evaluates its own nodes, so each float64 instruction does the
// work of all its lanes on a part whose float64 rate is low.
constexpr int kSlqThreads = 256;
constexpr double kSlqStep = 0.5;   // h
constexpr double kSlqTail = 36.0;  // trapezoidal range beyond the spectrum bounds, in log units

// (p0, p1, p2) scaled by the power of two that brings max(|p0|, |p1|) into [1, 2): exact.
__device__ __forceinline__ void rescale_pow2(double &p0, double &p1, double &p2) {
    const double mx = fmax(fabs(p0), fabs(p1));
    if (!(mx > 0.0) || !isfinite(mx)) return;
    const int e = ((__double2hiint(mx) >> 20) & 0x7ff) - 1023;
    if (e <= -1022 || e >= 1023) return;
    const double sc = __hiloint2double((1023 - e) << 20, 0);
    p0 *= sc;
    p1 *= sc;
    p2 *= sc;
}

// One block per probe column c = blockIdx.x + 1: gamma_c = w_c e_1^T log(T_c) e_1 with
// w_c = z_c^T P^{-1} z_c (||z_c||^2 without a preconditioner), T_c from the first
// m = min(L, iterations of c) CG coefficients: T[k,k] = 1/alpha_k + beta_{k-1}/alpha_{k-1},
// T[k,k+1] = sqrt(beta_k)/alpha_k. Writes gamma[c] and bad[c] (1 if T_c is not positive definite
// or a value is not finite). Summation order is fixed.
__global__ void __launch_bounds__(kSlqThreads) slq_quad_kernel(const CgState *st, const double *__restrict__ hist_alpha,
                                                               const double *__restrict__ hist_beta, int t,
                                                               int hist_len, double *__restrict__ gamma,
                                                               double *__restrict__ bad) {
    __shared__ double sa[kMaxLanczos], sbb[kMaxLanczos], sal[kMaxLanczos], sbe[kMaxLanczos];
    __shared__ double red[kSlqThreads];
    __shared__ double s_vlo;
    __shared__ int s_nodes, s_bad;
    const int c = blockIdx.x + 1;
    const int tid = threadIdx.x;
    const int m = min(hist_len, st->iters[c]);
    if (m <= 0) {
        if (tid == 0) {
            gamma[c] = 0.0;
            bad[c] = 0.0;
        }
        return;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k = tid; k < m; k += kSlqThreads) {
        const double al = hist_alpha[(int64_t)k * t + c];
        const double be = hist_beta[(int64_t)k * t + c];
        sal[k] = al;
        sbe[k] = be;
        if (!(al > 0.0) || !isfinite(al) || (k + 1 < m && (!(be >= 0.0) || !isfinite(be)))) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    for (int k = tid; k < m; k += kSlqThreads) {
        double a = 1.0 / sal[k];
        if (k > 0) a += sbe[k - 1] / sal[k - 1];
        sa[k] = a;
        sbb[k] = k + 1 < m ? sbe[k] / (sal[k] * sal[k]) : 0.0;  // b_k^2
    }
    __syncthreads();
    // Gershgorin upper bound of the spectrum (max reduction over the rows)
    double g = 0.0;
    for (int k = tid; k < m; k += kSlqThreads) {
        double gk = sa[k];
        if (k > 0) gk += sqrt(sbb[k - 1]);
        if (k + 1 < m) gk += sqrt(sbb[k]);
        g = fmax(g, gk);
    }
    red[tid] = g;
    __syncthreads();
    for (int s = kSlqThreads / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
        __syncthreads();
    }
    if (tid == 0) {
        const double lam_hi = red[0];
        double sk = 1.0, tr = sal[0];
        for (int i = 1; i < m; ++i) {
            sk = fma(sbe[i - 1], sk, 1.0);
            tr = fma(sal[i], sk, tr);
        }
        const double lam_lo = 1.0 / tr;
        if (!(lam_hi > 0.0) || !isfinite(lam_hi) || !(lam_lo > 0.0) || !isfinite(tr)) s_bad = 1;
        const double vlo = log(lam_lo) - kSlqTail;
        const double vhi = log(lam_hi) + kSlqTail;
        s_vlo = vlo;
        s_nodes = s_bad ? 0 : (int)ceil((vhi - vlo) / kSlqStep) + 1;
    }
    __syncthreads();
    const int nodes = s_nodes;
    const double a1m1 = sa[0] - 1.0, b1sq = sbb[0];
    double acc = 0.0;
    int nonpos = 0;
    for (int n = tid; n < nodes; n += kSlqThreads) {
        const double x = exp(s_vlo + n * kSlqStep);
        double p0 = sa[m - 1] + x, p1 = 1.0, p2 = 0.0;  // (P_k, P_{k+1}, P_{k+2}) at k = m
        for (int k = m - 2, q = 0; k >= 0; --k, ++q) {
            p2 = p1;
            p1 = p0;
            p0 = fma(sa[k] + x, p1, -sbb[k] * p2);
            if ((q & 3) == 3) rescale_pow2(p0, p1, p2);
        }
        if (!(p0 > 0.0)) nonpos = 1;  // T + x I positive definite: every trailing minor is positive
        acc += x * fma(a1m1, p1, -b1sq * p2) / ((1.0 + x) * p0);
    }
    if (nonpos) atomicOr(&s_bad, 1);
    red[tid] = acc;
    __syncthreads();
    for (int s = kSlqThreads / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) {
        const double v = st->w0[c] * kSlqStep * red[0];
        gamma[c] = v;
        bad[c] = (s_bad || !isfinite(v)) ? 1.0 : 0.0;
    }
}

// logdet = logdet_P + mean_c gamma_c (logdet_P = log|P|, 0 without a preconditioner);
// LML = -1/2 (y^T K_y^{-1} y + logdet + N log 2 pi). Sums in column order.
__global__ void slq_lml_finish_kernel(const double *__restrict__ gamma, const double *__restrict__ bad, int t,
                                      const double *__restrict__ dots, int64_t N, double logdet_p, double *out) {
    double s = 0.0;
    int any_bad = 0;
    for (int k = 1; k < t; ++k) {
        s += gamma[k];
        any_bad |= bad[k] != 0.0;
    }
    const double logdet = logdet_p + (t > 1 ? s / (t - 1) : 0.0);
    const double quad = dots[0];
    out[0] = -0.5 * (quad + logdet + (double)N * 1.8378770664093453);  // log(2 pi)
    out[1] = quad;
    out[2] = logdet;
    out[3] = any_bad ? 1.0 : 0.0;
}

__global__ void adjoint_rhs_kernel(const float *__restrict__ A, const float *__restrict__ RHS, int64_t N, int t,
                                   float *__restrict__ Bp) {
    const int64_t total = N * t;
    const float inv_m = t > 1 ? -1.0f / (float)(t - 1) : 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        Bp[e] = c == 0 ? A[i * t] : inv_m * RHS[e];
    }
}

__global__ void grad_finalize_kernel(const double *__restrict__ bp, int n_blocks, int D, const double *__restrict__ dots,
                                     int t, float noise, double *grad_out) {
    const int p = threadIdx.x;
    if (p <= D) {
        double s = 0.0;
        for (int b = 0; b < n_blocks; ++b) s += bp[(int64_t)b * (D + 1) + p];
        grad_out[p] = 0.5 * s;
    } else if (p == D + 1) {
        double tr = 0.0;
        for (int c = 1; c < t; ++c) tr += dots[c];
        const double m = t > 1 ? (double)(t - 1) : 1.0;
        grad_out[p] = 0.5 * (double)noise * (dots[t] - tr / m);
    }
}

inline int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int cg_num_blocks(int64_t N, int t, int num_sms) {
    int64_t g = (N * t + 4095) / 4096;
    if (g > 2 * num_sms) g = 2 * num_sms;
    if (g < 1) g = 1;
    return (int)g;
}

void launch_cg_init(const float *B, int64_t ldb, int64_t N, int64_t Np, int t, const CgBuffers &b, double tol,
                    int max_iter, int hist_len, cudaStream_t st, const float *X0, int64_t ldx0) {
    (void)Np;
    double *rr_partial = nullptr;
    if (X0) {
        // b.Kp holds K_y x0; the r^T r partials go to the third slot of the partial buffer
        rr_partial = b.partial + (int64_t)2 * b.G * t;
        cg_init_x0_kernel<<<b.G, vec_block(t), 0, st>>>(B, ldb, X0, ldx0, b.Kp, N, t, b.x, b.r, b.p, b.partial,
                                                        rr_partial);
    } else {
        cg_init_kernel<<<b.G, vec_block(t), 0, st>>>(B, ldb, N, t, b.x, b.r, b.p, b.partial);
    }
    double *rz_partial = nullptr;
    if (b.pc.k > 0) {
        // z0 = P^{-1} b, p0 = z0, and the r^T z partials in the second half of the partial buffer
        rz_partial = b.partial + (int64_t)b.G * t;
        launch_precond_apply(b.pc, b.r, t, b.z, t, b.p, N, t, rz_partial, b.G, nullptr, st);
    }
    cg_init_scalars_kernel<<<1, 32 * (t < 32 ? t : 32), 0, st>>>(b.state, b.partial, b.G, t, tol, max_iter, hist_len,
                                                                 rz_partial, rr_partial);
}

void launch_cg_after_matvec(int64_t N, int64_t Np, int t, const CgBuffers &b, cudaStream_t st) {
    (void)Np;
    const int bd = vec_block(t);
    cg_pkp_kernel<<<b.G, bd, 0, st>>>(b.p, b.Kp, N, t, b.state, b.partial);
    const int sb = 32 * (t < 32 ? t : 32);
    cg_alpha_kernel<<<1, sb, 0, st>>>(b.state, b.partial, b.G, b.hist_alpha);
    cg_xr_kernel<<<b.G, bd, 0, st>>>(b.x, b.r, b.p, b.Kp, N, t, b.state, b.partial);
    double *rz_partial = nullptr;
    if (b.pc.k > 0) {
        rz_partial = b.partial + (int64_t)b.G * t;
        launch_precond_apply(b.pc, b.r, t, b.z, t, nullptr, N, t, rz_partial, b.G, b.state, st);
    }
    cg_beta_kernel<<<1, sb, 0, st>>>(b.state, b.partial, b.G, b.hist_beta, rz_partial);
    cg_p_kernel<<<b.G, bd, 0, st>>>(b.p, b.pc.k > 0 ? b.z : b.r, N, t, b.state);
}

void launch_cg_loop_condition(cudaGraphConditionalHandle h, CgState *state, cudaStream_t st) {
    cg_loop_condition_kernel<<<1, 1, 0, st>>>(h, state);
}

void launch_cg_chunk_tally(CgState *state, cudaStream_t st) { cg_chunk_tally_kernel<<<1, 1, 0, st>>>(state); }

void launch_cg_gather_column(const CgBuffers &b1, int hist_len, CgState *dst, double *dst_alpha, double *dst_beta,
                             int t, int c, cudaStream_t st) {
    cg_gather_column_kernel<<<1, 64, 0, st>>>(b1.state, b1.hist_alpha, b1.hist_beta, hist_len, dst, dst_alpha,
                                              dst_beta, t, c);
}

void launch_cg_copy_out(const CgBuffers &b, int64_t N, int t, float *Xsol, int64_t ldx, cudaStream_t st) {
    copy_out_kernel<<<grid_for(N * t), 256, 0, st>>>(b.x, N, t, Xsol, ldx);
}

void launch_col_dots(const float *A, const float *B, int64_t N, int t, double *partial, int G, double *out,
                     cudaStream_t st) {
    col_dots_kernel<<<G, vec_block(t), 0, st>>>(A, B, N, t, partial);
    col_dots_final_kernel<<<1, 2 * kMaxT, 0, st>>>(partial, G, t, out);
}

void launch_slq_lml(const CgBuffers &b, int t, int hist_len, const double *dots, int64_t N, double *out,
                    cudaStream_t st) {
    // per-column gamma and bad flags in the CG partial-sum buffer (3 G t >= 2 t doubles, free after
    // the column dots have been reduced)
    double *gamma = b.partial;
    double *bad = b.partial + t;
    if (t > 1)
        slq_quad_kernel<<<t - 1, kSlqThreads, 0, st>>>(b.state, b.hist_alpha, b.hist_beta, t, hist_len, gamma, bad);
    slq_lml_finish_kernel<<<1, 1, 0, st>>>(gamma, bad, t, dots, N, b.pc.k > 0 ? b.pc.logdet : 0.0, out);
}

void launch_adjoint_rhs(const float *A, const float *RHS, int64_t N, int t, float *Bp, cudaStream_t st) {
    adjoint_rhs_kernel<<<grid_for(N * t), 256, 0, st>>>(A, RHS, N, t, Bp);
}

void launch_grad_finalize(const double *block_partials, int n_blocks, int D, const double *dots, int t, float noise,
                          double *grad_out, cudaStream_t st) {
    grad_finalize_kernel<<<1, 32, 0, st>>>(block_partials, n_blocks, D, dots, t, noise, grad_out);
}

}  // namespace lgp
