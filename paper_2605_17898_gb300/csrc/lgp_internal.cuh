// Internal declarations shared by the CUDA translation units of the library.
//
// Coordinates. Every product works on prescaled inputs xh_d = c_kind * x_d / l_d
// so that one kernel entry is a short register computation:
//   RBF:        c = sqrt(log2(e) / 2), rh2 = c^2 r^2,  k = 2^(log2 s^2 - rh2)
//   Matern-5/2: c = sqrt(5),           rh  = sqrt(5) r, k = (1 + rh + rh^2/3) 2^(log2 s^2 - rh log2 e)
// Both equal the standard forms k = s^2 exp(-r^2/2) and
// k = s^2 (1 + sqrt5 r + 5 r^2/3) exp(-sqrt5 r) with r^2 = sum_d ((x_d - x'_d)/l_d)^2.
// Lengthscale derivatives in the same coordinates: dk/dlog l_d = psi * (dxh_d)^2 with
//   RBF:        psi = 2 ln2 * k
//   Matern-5/2: psi = (1 + rh) * s^2 2^(-rh log2 e) / 3
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgp.h"

namespace lgp {

constexpr int kMaxD = 8;
constexpr int kMaxT = 64;
// Lanczos steps kept per column for the log-determinant quadrature (the quadrature kernel holds the
// tridiagonal in shared memory: 4 x 8 bytes per step)
constexpr int kMaxLanczos = 1024;
constexpr int kMaxRank = 32;  // largest pivoted-Cholesky preconditioner rank
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTwoLn2 = 1.3862943611198906f;
constexpr float kLn2 = 0.6931471805599453f;

// Padded row width of the prescaled X buffer (floats): 4 for D <= 4, else 8.
inline int dpad_of(int D) { return D <= 4 ? 4 : 8; }

struct KernelParams {
    int kind;
    int D;
    int dpad;
    float log2_s2;   // log2(s^2)
    float s2;        // s^2
    float noise;     // sigma_n^2
    float scale[kMaxD];
};

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Accumulates a * b into the float pair (hi, lo) without float64 arithmetic: the product's rounding
// error exactly by FMA (TwoProduct) and the running sum's by Knuth's TwoSum, as in the compensated
// dot product of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005).
// Each operation is an explicitly rounded intrinsic, so the compiler cannot contract it into an FMA.
// hi + lo carries the partial sum to about 2^-44 relative; the block and column reductions then run in
// float64. (The float64 pipe of this GPU is slow enough that converting every element to double set
// the time of these kernels.)
__device__ __forceinline__ void acc_prod2(float &hi, float &lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

template <int KIND> struct Entry;

template <> struct Entry<LGP_RBF> {
    // k from the prescaled squared distance.
    static __device__ __forceinline__ float k(float rh2, float log2s2) { return ex2_approx(log2s2 - rh2); }
    // k and psi (dk/dlog l_d = psi * dxh_d^2).
    static __device__ __forceinline__ void k_psi(float rh2, float log2s2, float &k, float &psi) {
        k = ex2_approx(log2s2 - rh2);
        psi = kTwoLn2 * k;
    }
};

template <> struct Entry<LGP_MATERN52> {
    static __device__ __forceinline__ float k(float rh2, float log2s2) {
        const float rh = sqrt_approx(rh2);
        const float e = ex2_approx(fmaf(-rh, kLog2e, log2s2));
        const float poly = fmaf(rh2, 1.0f / 3.0f, rh) + 1.0f;
        return poly * e;
    }
    static __device__ __forceinline__ void k_psi(float rh2, float log2s2, float &k, float &psi) {
        const float rh = sqrt_approx(rh2);
        const float e = ex2_approx(fmaf(-rh, kLog2e, log2s2));
        const float poly = fmaf(rh2, 1.0f / 3.0f, rh) + 1.0f;
        k = poly * e;
        psi = (1.0f + rh) * e * (1.0f / 3.0f);
    }
};

// Matern-1/2 on x = log2(e) x / l: rh = r log2 e, k = 2^(log2 s^2 - rh). dk/dlog l_d = s^2 e^-r r_d^2 / r
// = k ln2 dxh_d^2 / rh for r > 0, and 0 at r = 0 (where every dxh_d is 0).
template <> struct Entry<LGP_MATERN12> {
    static __device__ __forceinline__ float k(float rh2, float log2s2) { return ex2_approx(log2s2 - sqrt_approx(rh2)); }
    static __device__ __forceinline__ void k_psi(float rh2, float log2s2, float &k, float &psi) {
        k = ex2_approx(log2s2 - sqrt_approx(rh2));
        psi = rh2 > 0.0f ? k * kLn2 * rsqrtf(rh2) : 0.0f;
    }
};

// Matern-3/2 on x = sqrt3 x / l: rh = sqrt3 r, k = (1 + rh) e with e = 2^(log2 s^2 - rh log2 e);
// dk/dlog l_d = 3 s^2 e^(-sqrt3 r) r_d^2 = e dxh_d^2.
template <> struct Entry<LGP_MATERN32> {
    static __device__ __forceinline__ float k(float rh2, float log2s2) {
        const float rh = sqrt_approx(rh2);
        const float e = ex2_approx(fmaf(-rh, kLog2e, log2s2));
        return fmaf(e, rh, e);
    }
    static __device__ __forceinline__ void k_psi(float rh2, float log2s2, float &k, float &psi) {
        const float rh = sqrt_approx(rh2);
        const float e = ex2_approx(fmaf(-rh, kLog2e, log2s2));
        k = fmaf(e, rh, e);
        psi = e;
    }
};

// Host: the kind is one the library implements.
inline bool kind_supported(int kind) {
    return kind == LGP_RBF || kind == LGP_MATERN52 || kind == LGP_MATERN12 || kind == LGP_MATERN32;
}

// Host: the factor c of the prescaled coordinates x = c x / l, chosen so that each entry needs one
// ex2: RBF sqrt(log2(e) / 2) (rh^2 = r^2 log2(e) / 2), M52 sqrt5, M32 sqrt3, M12 log2(e).
inline double prescale_of(int kind) {
    switch (kind) {
        case LGP_RBF: return 0.8493218002880191;     // sqrt(0.5 / ln 2)
        case LGP_MATERN52: return 2.23606797749979;  // sqrt 5
        case LGP_MATERN32: return 1.7320508075688772;  // sqrt 3
        case LGP_MATERN12: return 1.4426950408889634;  // log2 e
    }
    return 0.0;
}

// ---------------------------------------------------------------- CG state on the device

// Per-column CG scalars (float64) and flags, plus the Lanczos history.
struct CgState {
    int iter;          // iterations done (global counter)
    int done;          // 1 when no column is active or iter reached max_iter
    int status;        // 0 ok, else an lgp_status (breakdown / nonfinite)
    int max_iter;
    int hist_len;      // Lanczos steps kept per column
    int t;
    int loop_chunks;   // chunks run by the device-side while loop
    int max_chunks;    // hard cap on loop_chunks (the loop ends even if `done` were never set)
    double tol;
    int active[kMaxT];
    int iters[kMaxT];
    double bnorm2[kMaxT];
    double rr[kMaxT];
    double rz[kMaxT];  // r^T z with z = P^{-1} r (= rr without a preconditioner)
    double w0[kMaxT];  // b^T P^{-1} b: the Lanczos quadrature weight of each column
    double alpha[kMaxT];
    double beta[kMaxT];
};

// ---------------------------------------------------------------- launchers (defined in the .cu files)

// prep.cu
void launch_prep_x(const float *X, int64_t N, int D, int dpad, const float *scale_host, float *Xs, int64_t Np,
                   int *err_flag, cudaStream_t st);
void launch_rademacher(uint64_t seed, int64_t N, int m, float *Z, int64_t ldz, int col0, cudaStream_t st);
void launch_scan_finite(const float *A, int64_t n, int *err_flag, cudaStream_t st);
void launch_copy_cols(const float *src, int64_t lds, float *dst, int64_t ldd, int64_t rows, int cols, int dst_col0,
                      cudaStream_t st);

// predict.cu
void launch_kernel_cols(const KernelParams &kp, const float *Xh, int64_t N, int64_t Np, const float *Xsh, int64_t j0,
                        int tc, float *B, int64_t ldb, int col0, cudaStream_t st);
void launch_var_from_dots(const double *dots, int c0, int t, float s2, float *var, int64_t j0, cudaStream_t st);
void launch_var_from_probes(const float *Z, int64_t ldz, const float *Q, int64_t ldq, int64_t M, int m, float s2,
                            float *var, cudaStream_t st);

// mv_simt.cu
struct MvLaunch {
    const KernelParams *kp;
    const float *Xs;      // prescaled [Np, dpad]
    int64_t N, Np;
    const float *V;       // [N, ldv] (rows >= N are never read)
    int64_t ldv;
    float *out;           // [N, ldo]
    int64_t ldo;
    int t;
    float *partial;       // split-column partial sums (workspace) or nullptr
    int64_t partial_cap;  // floats available in partial
    const int *skip;      // device flag: skip all work when *skip != 0 (may be nullptr)
    int num_sms;
    // Cross product out = K(Xr, Xs) V (no noise term): prescaled row points [Npr, dpad] and their
    // count; Xr == nullptr gives the square product K_y V.
    const float *Xr = nullptr;
    int64_t Nr = 0, Npr = 0;
};
cudaError_t launch_mv_simt(const MvLaunch &m, cudaStream_t st);
int mv_simt_launches(int64_t N, int64_t Np, int t, int num_sms);
int64_t mv_simt_partial_floats(int64_t N, int64_t Np, int t, int num_sms);
// Split partial floats of the cross product with Nr output rows (Npr padded) and N columns.
int64_t mv_simt_cross_partial_floats(int64_t Nr, int64_t Npr, int64_t N, int t, int num_sms);

cudaError_t launch_mv_grad(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *W, int t,
                           float *G, float *partial, int64_t partial_cap, int num_sms, cudaStream_t st);
int64_t mv_grad_partial_floats(int64_t N, int64_t Np, int t, int D, int num_sms);

// Bilinear adjoint reduction: acc[p] = sum_ij dK_p[i,j] * (A_i . B_j) for p < D (lengthscales), p = D (log s^2).
cudaError_t launch_adjoint_bilinear(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *A,
                                    const float *B, int t, double *block_partials, int64_t partial_cap, int *n_blocks,
                                    int num_sms, cudaStream_t st);
int64_t adjoint_partial_doubles(int64_t N, int t, int D, int num_sms);

// mv_tc.cu
bool tc_supported(int t);
int64_t tc_vsplit_bytes(int64_t Np, int t);
// fmt: 0 = bfloat16 halves, 1 = scaled float16 halves
// forced_splits > 0 overrides the column-split count (the autotuner's choice); 0 = wave-efficiency heuristic;
// kTcSymmetric = the symmetric-tile kernel (mv_tcs.cuh), which adds onto out instead of writing partials.
constexpr int kTcSymmetric = -1;
// operands_ready: the operands that depend on X alone are already in vsplit (launch_tc_operands, once
// per prepared X): the transposed X and, where the symmetric product may take the dot form, its
// distance operands; otherwise the product builds them first.
// dist_form (symmetric product with the dot form allowed): -1 = not known on the host, so both distance
// instances launch and the device gate word lets one of them work; 0 / 1 = only the difference / dot
// instance launches (the caller read the gate word, which must then give the same answer).
// ev_begin / ev_end (optional): recorded on st immediately before and after the product kernel's
// launch(es), after the V split and operand kernels (the kernel timing of lgp_last_kernel_ms).
cudaError_t launch_mv_tc(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *V, int64_t ldv,
                         float *out, int64_t ldo, int t, int fmt, void *vsplit, float *partial, int64_t partial_cap,
                         const int *skip, int *err_flag, long long wait_budget, int num_sms, cudaStream_t st,
                         int forced_splits = 0, bool operands_ready = false, int dist_form = -1,
                         cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);
// The operands of the tensor-core products that depend on X alone, into the t-column V-split workspace:
// the transposed prescaled X, and with dot = true the dot-form distance data of the symmetric product
// (box, centred split operands, squared norms, the gate word).
cudaError_t launch_tc_operands(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, int t, void *vsplit,
                               bool dot, cudaStream_t st);
int64_t mv_tc_partial_floats(int64_t Np, int t, int num_sms);
int64_t mv_tc_partial_floats(int64_t Np, int t, int num_sms, int forced_splits);
// Kernels one split tensor-core product launches (arguments as launch_mv_tc).
int mv_tc_launches(int64_t Np, int t, int num_sms, int fmt, int forced_splits = 0, int kind = -1, int D = 0,
                   bool operands_ready = false, int dist_form = -1);
// Up to four kernel choices worth timing: kTcSymmetric (when tc_symmetric_ok) and the three most
// wave-efficient split counts.
void tc_split_candidates(int64_t Np, int num_sms, int *cand, int *n);
bool tc_symmetric_ok(int64_t Np);
// Dot-form distance of the symmetric product: whether it is considered for (kind, D), its limit on
// max |u|^2, and the byte offset of the word holding the measured max in the V-split workspace.
bool dot_form_allowed(int kind, int D);
float dot_gate_limit(int kind);
int64_t tc_dot_gate_offset(int64_t Np, int t);

// precond.cu: the rank-k pivoted-Cholesky preconditioner P = L L^T + sigma^2 I (k = 0: none).
struct Precond {
    int k = 0;
    int64_t Np = 0;                // row stride of the L columns
    const double *L64 = nullptr;   // [k][Np] (column q contiguous over rows)
    const float *L32 = nullptr;    // float32 copy used inside the CG iterations
    const double *Cinv = nullptr;  // [k][k] inverse of C = sigma^2 I + L^T L
    double *part = nullptr;        // [G][k t] block partials of L^T R
    double *U = nullptr;           // [k][t] C^{-1} L^T R
    int G = 0;                     // blocks of the L^T R reduction
    double noise = 0.0;
    double logdet = 0.0;           // log|P| = (N - k) log sigma^2 + log|C|
};

size_t pivinfo_bytes();
// k pivoted-Cholesky steps of K_ff from the raw float32 X [N, D] (float64 arithmetic): L64 [k][Np], residual d [Np]
void launch_pivchol(const float *X, int64_t N, int64_t Np, int D, const double *inv_ls_host, double s2, int kind,
                    int k, double *L64, double *d, void *pinfo, cudaStream_t st);
// Block partials [G][k * k] of L^T L
void launch_gram(const double *L64, int64_t Np, int64_t N, int k, double *partial, int G, cudaStream_t st);
void launch_to_f32(const double *src, float *dst, int64_t n, cudaStream_t st);
// Z = P^{-1} R for rows < N (t <= 32, k t <= 1024); Pcopy (may be null) receives Z too; rz_partial (may be
// null) gets [G_vec][t] block partials of r^T z; state (may be null) skips the work once the CG is done.
void launch_precond_apply(const Precond &pc, const float *R, int64_t ldr, float *Z, int64_t ldz, float *Pcopy,
                          int64_t N, int t, double *rz_partial, int G_vec, const CgState *state, cudaStream_t st);
// rhs[:, col0 + c] = L E[N:, c] + sigma E[:N, c] for the [N + k, m] Rademacher block E
void launch_precond_probes(const double *L64, int64_t Np, int k, const float *E, int64_t N, int m, double sigma,
                           float *rhs, int64_t ldr, int col0, cudaStream_t st);

// solver.cu
struct CgBuffers {
    float *x, *r, *p, *Kp;   // [Np, t]
    float *z;                // [Np, t] P^{-1} r (preconditioned solves only)
    double *partial;         // [G, 3t] block partial dots
    int G;                   // blocks of the vector kernels
    CgState *state;
    double *hist_alpha;      // [hist_len, t]
    double *hist_beta;       // [hist_len, t]
    Precond pc;              // pc.k == 0: plain CG
};
// X0 (may be null): warm start x0 [N, ldx0], with K_y x0 already in b.Kp.
void launch_cg_init(const float *B, int64_t ldb, int64_t N, int64_t Np, int t, const CgBuffers &b, double tol,
                    int max_iter, int hist_len, cudaStream_t st, const float *X0 = nullptr, int64_t ldx0 = 0);
void launch_cg_after_matvec(int64_t N, int64_t Np, int t, const CgBuffers &b, cudaStream_t st);
void launch_cg_copy_out(const CgBuffers &b, int64_t N, int t, float *Xsol, int64_t ldx, cudaStream_t st);
// Column 0 of the single-column run b1 (state, first hist_len Lanczos coefficients) into column c of a
// t-column state and history; dst->loop_chunks accumulates.
void launch_cg_gather_column(const CgBuffers &b1, int hist_len, CgState *dst, double *dst_alpha, double *dst_beta,
                             int t, int c, cudaStream_t st);
// Body tail of the device-side CG loop: sets the while-node condition to "not done and under the chunk cap".
void launch_cg_loop_condition(cudaGraphConditionalHandle h, CgState *state, cudaStream_t st);
// Host-driven loop (LGP_CG_GRAPH=0): counts one chunk in state->loop_chunks.
void launch_cg_chunk_tally(CgState *state, cudaStream_t st);
int cg_num_blocks(int64_t N, int t, int num_sms);

// Column dot products sum_i A[i,c] B[i,c] and sum_i A[i,c]^2 (float64), c < t: out[2t].
void launch_col_dots(const float *A, const float *B, int64_t N, int t, double *partial, int G, double *out,
                     cudaStream_t st);
// Stochastic Lanczos quadrature over probe columns 1..t-1 and the LML assembly.
// out: [0] lml, [1] quad, [2] logdet, [3] status flag (0 ok, else nonpositive Ritz value)
void launch_slq_lml(const CgBuffers &b, int t, int hist_len, const double *dots, int64_t N, double *out,
                    cudaStream_t st);
// B'[:,0] = A[:,0]; B'[:,c] = -Z[:,c] / m for c >= 1 (the right factor of the gradient's bilinear form)
void launch_adjoint_rhs(const float *A, const float *RHS, int64_t N, int t, float *Bp, cudaStream_t st);
// Sum block partials and form grad[p] = 1/2 acc[p] (p <= D); grad[D+1] from the noise term.
void launch_grad_finalize(const double *block_partials, int n_blocks, int D, const double *dots, int t, float noise,
                          double *grad_out, cudaStream_t st);

}  // namespace lgp
