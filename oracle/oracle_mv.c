/*
 * FP64 streaming product rows of K_y V for the CPU oracle (test infrastructure only).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load this
 * library. It shares no code with the CUDA path.
 *
 * out[r, c] = sum_j s2 * phi(r2(x_row, x_j)) * V[j, c] + noise * V[row, c]
 * for every requested row, the matrix-free product of Sec. 3 ("GPU backends",
 * Table 3) evaluated entry by entry in double precision without storing K.
 *
 *   r2  = sum_d ((x_row,d - x_j,d) / l_d)^2
 *   RBF (kind 0):        phi = exp(-r2 / 2)
 *   Matern-5/2 (kind 1): phi = (1 + sqrt5 r + 5 r2 / 3) exp(-sqrt5 r)
 *   Matern-1/2 (kind 2): phi = exp(-r)
 *   Matern-3/2 (kind 3): phi = (1 + sqrt3 r) exp(-sqrt3 r)
 *
 * oracle_kxv_rows is the same sum over a second point set: out[r, c] =
 * sum_j s2 * phi(r2(xr_row, x_j)) * V[j, c] (the cross-kernel product K_*f V of the
 * predictive mean, Sec. 2), without the noise term.
 *
 * X is [N, D] float32 row-major, V is [N, t] float32 row-major, rows is
 * [nrows] int64 (NULL: all rows 0..N-1), out is [nrows, t] float64.
 * Rows are distributed over OpenMP threads; returns the thread count used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double phi_of(int32_t kind, double r2)
{
    switch (kind) {
    case 0: return exp(-0.5 * r2);
    case 1: {
        double r = sqrt(r2);
        return (1.0 + sqrt(5.0) * r + (5.0 / 3.0) * r2) * exp(-sqrt(5.0) * r);
    }
    case 2: return exp(-sqrt(r2));
    case 3: {
        double r = sqrt(r2);
        return (1.0 + sqrt(3.0) * r) * exp(-sqrt(3.0) * r);
    }
    }
    return NAN;
}

/* out[q, c] = sum_j s2 phi(r2(xr_q, x_j)) V[j, c] (+ noise V[row, c] when with_noise). */
static int rows_product(const float *Xr, const int64_t *rows, int64_t nrows, const float *X, int64_t N, int32_t D,
                        const double *lengthscale, double s2, double noise, int with_noise, int32_t kind,
                        const float *V, int32_t t, double *out, int32_t n_threads)
{
    int used = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows ? rows[q] : q;
        double xi[64];
        double acc[256];
        for (int d = 0; d < D; ++d) xi[d] = (double)Xr[i * D + d];
        for (int c = 0; c < t; ++c) acc[c] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double r2 = 0.0;
            for (int d = 0; d < D; ++d) {
                double diff = (xi[d] - (double)X[j * D + d]) / lengthscale[d];
                r2 += diff * diff;
            }
            const double k = s2 * phi_of(kind, r2);
            const float *vj = V + j * (int64_t)t;
            for (int c = 0; c < t; ++c) acc[c] += k * (double)vj[c];
        }
        for (int c = 0; c < t; ++c)
            out[q * t + c] = acc[c] + (with_noise ? noise * (double)V[i * (int64_t)t + c] : 0.0);
    }
    return used;
}

int oracle_kyv_rows(const float *X, int64_t N, int32_t D, const double *lengthscale,
                    double s2, double noise, int32_t kind, const float *V, int32_t t,
                    const int64_t *rows, int64_t nrows, double *out, int32_t n_threads)
{
    if (rows == NULL) nrows = N;
    return rows_product(X, rows, nrows, X, N, D, lengthscale, s2, noise, 1, kind, V, t, out, n_threads);
}

int oracle_kxv_rows(const float *Xr, int64_t Nr, const float *X, int64_t N, int32_t D, const double *lengthscale,
                    double s2, int32_t kind, const float *V, int32_t t, double *out, int32_t n_threads)
{
    return rows_product(Xr, NULL, Nr, X, N, D, lengthscale, s2, 0.0, 0, kind, V, t, out, n_threads);
}
