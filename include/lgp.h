/*
 * lgp.h - C ABI of the GB300 matrix-free Gaussian-process library.
 *
 * The library computes, on one NVIDIA GB300 (sm_103a) GPU, the hot path of
 * CG-based exact GP inference described in "LightGP: Lightweight Gaussian
 * Process Inference in C++ on Metal and CUDA" (arXiv 2605.17898):
 *
 *   - the fused matrix-free product K_y V = (K_ff + sigma_n^2 I) V, whose kernel
 *     entries are generated on the fly and never stored, so memory stays O(N)
 *     (Sec. 2 "CG-based inference", Sec. 3 "GPU backends", Table 3);
 *   - conjugate-gradient solves K_y^{-1} B that need only that product
 *     (Sec. 2, Sec. 3 "Inference");
 *   - the log marginal likelihood -1/2 [y^T K_y^{-1} y + log|K_y| + N log 2 pi]
 *     (Sec. 2) with a stochastic Lanczos log-determinant (Sec. 3 "Inference")
 *     over Rademacher probes (Sec. 4.3), and its hyperparameter gradient, which
 *     the paper obtains by 2P+1 finite-difference fits (Sec. 5) and this library
 *     obtains analytically in one matrix-free adjoint pass.
 *
 * Kernels (the paper names RBF and Matern-{1/2, 3/2, 5/2}, Sec. 3 "Kernels"; the forms
 * used here are the standard ones, with per-dimension ARD lengthscales l_d):
 *   r^2 = sum_d ((x_d - x'_d) / l_d)^2
 *   LGP_RBF:       k = s^2 exp(-r^2 / 2)
 *   LGP_MATERN52:  k = s^2 (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r)
 *   LGP_MATERN32:  k = s^2 (1 + sqrt3 r) exp(-sqrt3 r)
 *   LGP_MATERN12:  k = s^2 exp(-r)
 *
 * Conventions shared by every entry point:
 *   - All arrays are row-major float32 unless stated. X is [N, D], right-hand
 *     sides and results are [N, t] with row stride t. Device pointers must be
 *     4-byte aligned and point to device (or managed) memory of the context's
 *     device; a host pointer where a device array is expected is rejected with
 *     LGP_ERR_INVALID_ARG before anything is launched.
 *   - Ownership: the caller owns every array passed in. The library owns only
 *     the context and its workspace (grown on demand, released by lgp_destroy).
 *   - Streams: work is ordered on the caller's stream (a cudaStream_t passed as
 *     lgp_stream; NULL means the legacy default stream). Entry points that
 *     return host scalars synchronise that stream before returning.
 *   - Errors: arguments are checked before any launch. A negative status means
 *     the outputs are undefined; a positive status means they are valid with a
 *     warning. lgp_last_error_message() describes the last failure.
 *   - Limits: 1 <= D <= 8, 1 <= t <= 64, N >= 1, 1 <= lanczos_steps <= 1024.
 *   - Thread safety: a context must not be used by two host threads at once.
 */
#ifndef LGP_H
#define LGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LGP_OK = 0,
    LGP_WARN_NOT_CONVERGED = 1,   /* some column hit max_iter; outputs valid */
    LGP_ERR_INVALID_ARG = -1,     /* bad pointer, size, alignment or value */
    LGP_ERR_UNSUPPORTED = -2,     /* a size or mode the library does not handle */
    LGP_ERR_CUDA = -3,            /* a CUDA runtime call failed */
    LGP_ERR_NONFINITE = -4,       /* NaN/Inf in inputs or in a CG scalar */
    LGP_ERR_BREAKDOWN = -5,       /* p^T K_y p <= 0 in CG (K_y not positive definite) */
    LGP_ERR_TIMEOUT = -6,         /* a bounded device-side wait ran out */
    LGP_ERR_WORKSPACE = -7        /* workspace allocation failed */
} lgp_status;

typedef enum { LGP_RBF = 0, LGP_MATERN52 = 1, LGP_MATERN12 = 2, LGP_MATERN32 = 3 } lgp_kernel;

/* Arithmetic of the K_y V contraction.
 * FP32: entries and products in float32 FMA (any t).
 * SPLIT_BF16: entries generated in float32, split as k = hi + lo with
 *   hi = bf16_rn(k), lo = bf16_rn(k - hi) (likewise V), contracted on tcgen05
 *   tensor cores as hi*hi + hi*lo + lo*hi with float32 accumulation (about 16
 *   significant bits per factor).
 * SPLIT_F16: the same three-product contraction on float16 halves of values
 *   scaled by exact powers of two (entries by 2^15 / s^2, each V column so that
 *   its largest magnitude is below 2^15), about 22 bits per factor.
 * The split kernels take t in {16, 32}. lgp_kernel_matvec and lgp_cg_solve also accept an explicit split
 * precision for any other t <= 32: they run it on the columns zero-padded to 16 (t < 16) or 32, and return
 * the caller's t. Single right-hand sides at large N gain most: at N = 100000, D = 8, the padded split
 * product takes about 2.9 ms against 7.5 ms for the float32 one. lgp_lml_and_grad and lgp_predict keep
 * t in {16, 32} for the split modes.
 * AUTO picks SPLIT_F16 for t in {16, 32} and FP32 otherwise. */
typedef enum {
    LGP_PREC_AUTO = 0,
    LGP_PREC_FP32 = 1,
    LGP_PREC_SPLIT_BF16 = 2,
    LGP_PREC_SPLIT_F16 = 3
} lgp_precision;

typedef struct {
    int32_t kind;                  /* lgp_kernel */
    int32_t D;                     /* input dimension, 1..8 */
    const float *log_lengthscale;  /* HOST pointer to D values of log l_d */
    float log_outputscale;         /* log s^2 */
    float log_noise;               /* log sigma_n^2 */
} lgp_hyper;

typedef struct {
    double tol;              /* stop column c when ||r_c|| / ||b_c|| <= tol (recursive residual) */
    int32_t max_iter;        /* CG iteration cap, >= 1 */
    int32_t lanczos_steps;   /* L: CG steps per probe kept for the Lanczos tridiagonal (1..1024).
                              * The log-determinant quadrature uses min(L, that probe's CG
                              * iterations) steps. Too few steps bias it when K_y is badly
                              * conditioned. With L at least the iteration count, the whole
                              * Krylov space of the solve is used. */
    int32_t n_probes;        /* m Rademacher probes; the solve block is [y, z_1..z_m], t = m + 1 */
    int32_t prec;            /* lgp_precision of the products inside the solve */
    uint64_t seed;           /* probe seed (see lgp_rademacher_probes) */
    int32_t precond_rank;    /* 0: plain CG (the paper's loop); k in 1..32: CG preconditioned by
                                P = L L^T + sigma_n^2 I, L the rank-k pivoted Cholesky factor of K_ff
                                (solves of at most 32 columns) */
    int32_t flags;           /* LGP_OPT_* bits, 0 for the defaults */
} lgp_options;

/* lgp_options.flags:
 * LGP_OPT_WARM_START: lgp_cg_solve starts from the initial guess held in Xsol on entry instead of
 *   x0 = 0 (a warm start, e.g. from the previous optimiser step's solution); columns whose initial
 *   residual already meets tol take no iteration. Ignored by the other entry points.
 * LGP_OPT_SINGLE_RHS: lgp_lml_and_grad solves the t = 1 + n_probes columns one at a time, each by
 *   its own CG run with the float32 one-column product, and computes the gradient with one adjoint
 *   pass per column: the paper's plain single-right-hand-side CG path (Sec. 5), kept as the
 *   comparison for the batched path. Same estimator and results up to float32 rounding; prec is
 *   ignored (always FP32); precond_rank must be 0. Ignored by the other entry points. */
enum { LGP_OPT_WARM_START = 1, LGP_OPT_SINGLE_RHS = 2 };
/* Largest lgp_options.lanczos_steps accepted. */
enum { LGP_MAX_LANCZOS_STEPS = 1024 };

typedef struct {
    double lml;              /* log marginal likelihood estimate */
    double quad;             /* y^T K_y^{-1} y */
    double logdet;           /* stochastic Lanczos estimate of log|K_y| */
    double max_rel_resid;    /* largest final recursive ||r||/||b|| over the t columns */
    int32_t iters_max;       /* most CG iterations over the columns */
    int32_t iters_min;       /* fewest CG iterations over the columns */
    int32_t t;               /* columns solved (1 + n_probes) */
    int32_t prec_used;       /* lgp_precision actually used for the products */
    int32_t launches;        /* kernel launches this call made on the device */
    int32_t cg_chunks;       /* CUDA-graph replays of the CG iteration chunk */
    double logdet_precond;   /* log|P| of the preconditioner (0 without one); included in logdet */
} lgp_lml_info;

typedef struct {
    int32_t solves;          /* batched CG solves run */
    int32_t iters_max;       /* most CG iterations over all solved columns */
    double max_rel_resid;    /* largest final recursive ||r||/||b|| over all solved columns */
    int32_t var_probes;      /* probes of the variance estimate (0: exact per-point variance) */
    int32_t prec_used;       /* lgp_precision of the products inside the first solve */
} lgp_predict_info;

typedef struct lgp_ctx lgp_ctx;
typedef void *lgp_stream;    /* a cudaStream_t */

/* Library version as 10000*major + 100*minor + patch. */
int32_t lgp_version(void);

/* Human-readable name of a status code (static storage). */
const char *lgp_status_string(int32_t status);

/* Environment variables read by a context (none changes results beyond float32 rounding):
 *   LGP_AUTOTUNE=0      the tensor-core product keeps the row kernel with its wave-efficiency
 *                       column split instead of timing the candidate kernels on first use of
 *                       a shape;
 *   LGP_TC_SYMMETRIC=1  force the symmetric-tile tensor-core kernel (shapes with N > 768);
 *                       =0 never use it. It adds its tiles' contributions with float32
 *                       atomic reductions, so its last bits can vary between runs;
 *   LGP_AUTOTUNE_CACHE=<file>  keep the autotuner's choices in a text file (one line per device and
 *                       shape, appended after tuning), so later processes skip the timing runs;
 *   LGP_CG_GRAPH=0      run the CG iteration loop from the host (one launch per kernel, the
 *                       done flag read back every 8 iterations) instead of one CUDA graph with
 *                       a device-side while loop; meant for profilers;
 *   LGP_DISTANCE=diff   keep the symmetric-tile kernel on the difference form of the squared
 *                       distance (see lgp_tc_distance_form); its results then differ from the
 *                       default dot form by that form's rounding (column errors of a few 1e-6);
 *   LGP_TC_BANDS=1      let the symmetric-tile kernel's dot form visit its tiles in column bands
 *                       whose operands stay in L2 (N above about 157000 at t = 32, 262000 at
 *                       t = 16): at N = 500000, t = 32 about 1 GB of DRAM traffic per product
 *                       instead of 115 GB, for a product about 4% slower (measured 68.2 against
 *                       65.6 ms); for GPUs whose memory bandwidth other work needs meanwhile. */

/* Create a context bound to CUDA device `device` (its workspace starts empty).
 * Returns LGP_ERR_INVALID_ARG for a NULL ctx or a device that does not exist,
 * LGP_ERR_UNSUPPORTED if the device is not compute capability 10.3. */
lgp_status lgp_create(lgp_ctx **ctx, int32_t device);

/* Release the context and its workspace. Waits for the context's device work. NULL is ignored. */
void lgp_destroy(lgp_ctx *ctx);

/* Message of the last failing call on this context ("" if none; static for a NULL ctx). */
const char *lgp_last_error_message(const lgp_ctx *ctx);

/* Workspace bytes currently held by the context. */
int64_t lgp_workspace_bytes(const lgp_ctx *ctx);

/* The lgp_precision lgp_kernel_matvec would use for t columns when asked for `prec`
 * (resolves LGP_PREC_AUTO); a negative lgp_status if that request is unsupported. */
int32_t lgp_matvec_precision(const lgp_ctx *ctx, int32_t t, int32_t prec);

/* Which tensor-core kernel this context uses for the product of an N-row, D-dimensional
 * `kind` problem with t columns at precision `prec` (diagnostic; no counterpart in the paper):
 * LGP_TC_UNTUNED before the first product of that shape, LGP_TC_ROW for the row kernel
 * (column range split over CTAs), LGP_TC_SYMMETRIC for the symmetric-tile kernel; a negative
 * lgp_status for invalid arguments or a precision that does not use the tensor cores. */
enum { LGP_TC_UNTUNED = 0, LGP_TC_ROW = 1, LGP_TC_SYMMETRIC = 2 };
int32_t lgp_tc_kernel_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t, int32_t prec);

/* How the last symmetric-tile product launched through this context formed its squared
 * distances (diagnostic). The difference form sums (x_id - x_jd)^2 over d in float32; the dot
 * form takes r^2 = |u_i|^2 + |u_j|^2 - 2 u_i . u_j for the box-centred coordinates u, with the
 * inner products on the tensor cores (split float16 operands, float32 accumulation; Sec. 3 names
 * this rewriting of the distance as the reason its product time barely depends on D). The dot
 * form is used for RBF, Matern-3/2 and Matern-5/2 at D >= 2 when max_j |u_j|^2 stays below a
 * per-kernel limit that bounds its rounding error; otherwise, for Matern-1/2, D = 1, or with
 * LGP_DISTANCE=diff in the environment, the difference form runs.
 * *form receives LGP_DIST_NONE (no symmetric product yet), LGP_DIST_DIFF or LGP_DIST_DOT;
 * *norm_max (may be NULL) the measured max_j |u_j|^2 when the dot form was considered, else -1.
 * Waits for the context's work and the given stream to finish. */
enum { LGP_DIST_NONE = -1, LGP_DIST_DIFF = 0, LGP_DIST_DOT = 1 };
lgp_status lgp_tc_distance_form(lgp_ctx *ctx, lgp_stream stream, int32_t *form, float *norm_max);

/* Bound, in GPU clock cycles, on every device-side wait of the tensor-core product
 * (pipeline barriers between its copy, generation and MMA stages). A wait that
 * runs out sets the context's device error word and the kernel returns early;
 * the calling entry point (or lgp_check_device_status) then reports
 * LGP_ERR_TIMEOUT. cycles <= 0 restores the default (about 4e9 cycles). */
void lgp_set_wait_budget(lgp_ctx *ctx, int64_t cycles);

/* Synchronise `stream`, read and clear the context's device error word:
 * LGP_OK, LGP_ERR_TIMEOUT (a bounded wait ran out) or LGP_ERR_CUDA. */
lgp_status lgp_check_device_status(lgp_ctx *ctx, lgp_stream stream);

/*
 * out = (K_ff + sigma_n^2 I) V: the fused matrix-free product (Sec. 3 "GPU
 * backends"; Table 3 times it for one column). X [N, D], V [N, t], out [N, t]
 * are device arrays; out must not alias V or X. `prec` selects the contraction
 * arithmetic (lgp_precision). Asynchronous on `stream`; no host sync.
 * A NaN/Inf in X or V propagates to out (no scan is made here).
 */
lgp_status lgp_kernel_matvec(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *V,
                             float *out, int64_t N, int32_t t, int32_t prec, lgp_stream stream);

/*
 * Derivative blocks G_p = (dK_y / dtheta_p) W for theta = (log l_1..log l_D,
 * log s^2, log sigma_n^2), P = D + 2: the matrix-free adjoint product whose
 * bilinear forms give the LML gradient (the quantity Sec. 5 obtains by finite
 * differences). W is [N, t] device, dK_W is a device array [P, N, t]
 * (block p at offset p*N*t). FP32 arithmetic. Asynchronous; no host sync.
 */
lgp_status lgp_kernel_matvec_grad(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *W,
                                  float *dK_W, int64_t N, int32_t t, lgp_stream stream);

/*
 * Xsol = K_y^{-1} B by unpreconditioned conjugate gradients from x0 = 0, one
 * recurrence per column, all t columns advanced together (Sec. 2 "CG-based
 * inference"; Sec. 5 "our simpler CG loop"). B and Xsol are device [N, t] and
 * may not alias. The vectors are float32; the CG scalars (dot products, alpha,
 * beta, residual norms) are accumulated in float64. iters (HOST [t], may be
 * NULL) receives the iterations per column, rel_resid (HOST [t], may be NULL)
 * the final recursive ||r||/||b||. Synchronises `stream`.
 * Returns LGP_WARN_NOT_CONVERGED if a column reached max_iter, LGP_ERR_NONFINITE
 * for NaN/Inf in X or B, LGP_ERR_BREAKDOWN if p^T K_y p <= 0.
 */
lgp_status lgp_cg_solve(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *B, float *Xsol,
                        int64_t N, int32_t t, const lgp_options *opt, int32_t *iters, double *rel_resid,
                        lgp_stream stream);

/*
 * Log marginal likelihood and its gradient (Sec. 2) by batched CG on
 * [y, z_1..z_m] (m = opt->n_probes Rademacher probes from opt->seed):
 *   quad   = y^T a, a = K_y^{-1} y;
 *   logdet = mean_i ||z_i||^2 e_1^T log(T_i) e_1, T_i the Lanczos tridiagonal of
 *            the first min(L, iterations) CG steps of probe i (Sec. 3 "CG with
 *            stochastic Lanczos log-determinant");
 *   lml    = -1/2 (quad + logdet + N log 2 pi);
 *   grad_p = 1/2 a^T dK_p a - 1/2 mean_i u_i^T dK_p z_i, u_i = K_y^{-1} z_i,
 *            for theta = (log l_1..log l_D, log s^2, log sigma_n^2).
 * X [N, D] and y [N] are device arrays. lml (HOST, may be NULL), grad (HOST
 * [D + 2], may be NULL: the adjoint pass is then skipped), info (HOST, may be
 * NULL). n_probes >= 1 and 1 <= lanczos_steps <= 1024. Synchronises `stream`.
 */
lgp_status lgp_lml_and_grad(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *y, int64_t N,
                            const lgp_options *opt, double *lml, double *grad, lgp_lml_info *info,
                            lgp_stream stream);

/*
 * Posterior prediction at M test points X* (Sec. 2):
 *   mean[j] = (K_*f K_y^{-1} y)_j,
 *   var[j]  = (K_** - K_*f K_y^{-1} K_f*)_jj   (latent f, no noise added),
 * with K_y^{-1} applied by batched CG (tol and max_iter from opt; the products use
 * opt->prec where the column count allows it).
 *   opt->n_probes = 0: exact variance. The right-hand sides [y, k(X, x*_1), ...]
 *     are solved in blocks of up to 32 columns; var[j] = s^2 - k_j . K_y^{-1} k_j.
 *   opt->n_probes = m in 1..31: the probe estimate of the diagonal (the CG
 *     "Hutchinson" route whose CPU/GPU agreement Sec. 4 reports as 3e-3): one
 *     solve of [y, K_f* z_1 .. K_f* z_m] with Rademacher z_c over the test points
 *     (the lgp_rademacher_probes stream with opt->seed, N replaced by M), then
 *     var[j] = s^2 - mean_c z_c[j] (K_*f K_y^{-1} K_f* z_c)[j].
 * X [N, D], y [N], Xs [M, D], mean [M] and var [M] are device arrays; var may be
 * NULL (mean only: one single-column solve). info (HOST) may be NULL. The cross
 * products K_*f v and K_f* Z run on the FP32 path. Errors as lgp_cg_solve (NaN or
 * Inf in X or Xs gives LGP_ERR_NONFINITE); LGP_WARN_NOT_CONVERGED if a column hit
 * max_iter. Synchronises `stream`.
 */
lgp_status lgp_predict(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *y, int64_t N,
                       const float *Xs, int64_t M, const lgp_options *opt, float *mean, float *var,
                       lgp_predict_info *info, lgp_stream stream);

/*
 * The probes lgp_lml_and_grad draws: Z[i, c] = +1 if bit 63 of
 * splitmix64(seed XOR (c * 2^32 + i)) is 0, else -1, for 0 <= i < N, 0 <= c < m
 * (splitmix64: Steele, Lea & Flood, OOPSLA 2014; independent Rademacher probes
 * as in Sec. 4.3). Z is a device array [N, ldz] (ldz >= m), written in columns
 * 0..m-1. Asynchronous; no host sync.
 */
lgp_status lgp_rademacher_probes(lgp_ctx *ctx, uint64_t seed, int64_t N, int32_t m, float *Z, int64_t ldz,
                                 lgp_stream stream);

/*
 * Many independent GP solves of uneven size in one call: for g < n_gp,
 * Xsol[g] = K_y(g)^{-1} B[g] with K_y(g) from hyp[g] and X[g] ([N[g], hyp[g].D]),
 * B[g] and Xsol[g] device [N[g], t], 1 <= t <= 16. Each problem takes one of two routes,
 * chosen per shape (padded N, D, kind, t) by timing, once, what a CG iteration of that
 * problem costs on each route on the caller's own data (the Sec. 5 gap: no batched solves):
 *   - the persistent batch: all such problems advance together, each CG iteration one
 *     float32 product launch over a work list of (problem, row block, column range)
 *     items plus one launch per vector update, the loop one CUDA graph with a
 *     device-side while node. A problem's cost there is its float32 product less that
 *     product's launch floor (timed on its first 256 rows), which the batch pays once;
 *   - the tensor-core route (problems of at least 2048 rows whose standalone CG iteration
 *     with the split-F16 product, columns zero-padded to 16, measures at least 10% cheaper
 *     than that marginal cost): its own CG solve with that product, as lgp_cg_solve with
 *     prec = LGP_PREC_SPLIT_F16.
 * opt->prec = LGP_PREC_FP32 keeps every problem in the persistent batch; LGP_AUTOTUNE=0
 * too. iters (HOST [n_gp * t], may be NULL) and rel_resid (HOST [n_gp * t], may be NULL)
 * are per problem and column. Synchronises `stream`.
 */
lgp_status lgp_batch_cg_solve(lgp_ctx *ctx, int32_t n_gp, const lgp_hyper *hyp, const float *const *X,
                              const float *const *B, float *const *Xsol, const int64_t *N, int32_t t,
                              const lgp_options *opt, int32_t *iters, double *rel_resid, lgp_stream stream);

/* Which route lgp_batch_cg_solve chose for problems of N rows, dimension D, kernel `kind`
 * and t columns (diagnostic; no counterpart in the paper): LGP_BATCH_UNTUNED before the
 * first batched solve with that shape, LGP_BATCH_PERSISTENT or LGP_BATCH_TENSOR; a
 * negative lgp_status for invalid arguments. */
enum { LGP_BATCH_UNTUNED = 0, LGP_BATCH_PERSISTENT = 1, LGP_BATCH_TENSOR = 2 };
int32_t lgp_batch_route_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t);

/* Column splits of the persistent batched product that lgp_batch_cg_solve chose for a problem of N rows,
 * dimension D, kernel `kind` and t columns (diagnostic; no counterpart in the paper). Each problem's
 * 256-row blocks are split S ways over whole 64-column tiles. S is timed per shape on the caller's own
 * data, with the problem alone in the work list (its last iterations, when no other problem is left),
 * among the fixed rule's count and a quarter, half, double and four times it. Returns S >= 1, 0 before
 * the first batched solve with that shape, or a negative lgp_status for invalid arguments. */
int32_t lgp_batch_split_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t);
/* The fixed rule's split count for a problem of N rows alone: about two items per CTA slot of the
 * persistent launch, at least four 64-column tiles per split (diagnostic). */
int32_t lgp_batch_split_rule(const lgp_ctx *ctx, int64_t N);

/*
 * Measurement support (no counterpart in the paper): throughput of one GPU pipe on the
 * current device, timed with CUDA events on `stream` at the clock the GPU runs.
 * which: 0 float32 FMA results/s, 1 packed float32x2 FMA results/s (two per lane),
 * 2 MUFU ex2.approx results/s, 3 MUFU sqrt.approx results/s. Synchronises `stream`.
 */
lgp_status lgp_measure_pipe_peak(int32_t which, double *ops_per_s, lgp_stream stream);

/*
 * Measurement support (no counterpart in the paper): the duration of the product kernel alone.
 * With timing on, every K_y V product that is not being captured into a CUDA graph records two
 * CUDA events on the stream it launches on. They sit immediately before and after the product
 * kernel's launch(es), after the per-call V split and the operand kernels. lgp_last_kernel_ms
 * synchronises on the second event of the last such product and returns the time between the
 * two, in milliseconds. It returns LGP_ERR_INVALID_ARG if no product was timed since timing was
 * switched on. Switching timing on creates the two events once per context.
 */
lgp_status lgp_set_kernel_timing(lgp_ctx *ctx, int32_t on);
lgp_status lgp_last_kernel_ms(lgp_ctx *ctx, float *ms);

/*
 * Allocation-free K_y V for callers that cannot allocate device memory: programs whose
 * device memory belongs to another allocator (a framework's caching pool, a fixed arena
 * sized at start-up) and must not have a library allocate behind their back; services
 * under a fixed device-memory budget, where an allocation failing mid-request cannot be
 * retried; and latency-critical loops, where cudaMalloc/cudaFree could synchronise the
 * device. The paper has no counterpart of this entry point; it is a deployment variant
 * of lgp_kernel_matvec's tensor-core path (the row kernel).
 *
 * Same arguments and result as lgp_kernel_matvec with prec in {AUTO, SPLIT_F16,
 * SPLIT_BF16} (AUTO = SPLIT_F16), but no context: it works on the current CUDA
 * device and calls no cudaMalloc, cudaFree or other allocating routine. Its
 * scratch is one fixed device array of about 17.3 MiB inside the library, held by
 * every GPU that loads the library until the process exits.
 *   - Limits: 1 <= N <= 8192, t in {16, 32}, 1 <= D <= 8; larger sizes return
 *     LGP_ERR_UNSUPPORTED before anything is launched.
 *   - Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the one array: calls whose work overlaps on the GPU (on
 *     different streams, or from several threads) race and corrupt each other.
 *     Order them on one stream.
 *   - Asynchronous on `stream`. The call itself returns LGP_ERR_INVALID_ARG for bad
 *     pointers or values and LGP_ERR_CUDA if a launch fails; it reads nothing back, so
 *     LGP_OK does not mean the device work succeeded. If a bounded device-side wait of
 *     the product runs out, the kernel returns early and `out` is left partly written
 *     (undefined); a NaN/Inf in X or V propagates to out. Both conditions are recorded
 *     in status words of the scratch array: see lgp_kernel_matvec_noalloc_status.
 */
lgp_status lgp_kernel_matvec_noalloc(const lgp_hyper *hyp, const float *X, const float *V, float *out,
                                     int64_t N, int32_t t, int32_t prec, lgp_stream stream);

/*
 * Status of the allocation-free product calls on the current device since the last
 * status read (no counterpart in the paper): synchronises `stream`, reads and clears the
 * scratch array's status words. Returns LGP_ERR_TIMEOUT if a bounded wait ran out in one
 * of those calls (its `out` is undefined), else LGP_ERR_NONFINITE if one of them had a
 * NaN/Inf in X, else LGP_OK; LGP_ERR_CUDA if the read fails. Allocates nothing. Work of
 * those calls still running on other streams must be finished by the caller first.
 */
lgp_status lgp_kernel_matvec_noalloc_status(lgp_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* LGP_H */
