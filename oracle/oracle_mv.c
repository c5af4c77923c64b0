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

int oracle_kyv_rows(const float *X, int64_t N, int32_t D, const double *lengthscale,
                    double s2, double noise, int32_t kind, const float *V, int32_t t,
                    const int64_t *rows, int64_t nrows, double *out, int32_t n_threads)
{
    int used = 1;
    if (rows == NULL) nrows = N;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#endif
    const double sqrt5 = sqrt(5.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows ? rows[q] : q;
        double xi[64];
        double acc[256];
        for (int d = 0; d < D; ++d) xi[d] = (double)X[i * D + d];
        for (int c = 0; c < t; ++c) acc[c] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double r2 = 0.0;
            for (int d = 0; d < D; ++d) {
                double diff = (xi[d] - (double)X[j * D + d]) / lengthscale[d];
                r2 += diff * diff;
            }
            double k;
            if (kind == 0) {
                k = s2 * exp(-0.5 * r2);
            } else {
                double r = sqrt(r2);
                k = s2 * (1.0 + sqrt5 * r + (5.0 / 3.0) * r2) * exp(-sqrt5 * r);
            }
            const float *vj = V + j * (int64_t)t;
            for (int c = 0; c < t; ++c) acc[c] += k * (double)vj[c];
        }
        for (int c = 0; c < t; ++c) out[q * t + c] = acc[c] + noise * (double)V[i * (int64_t)t + c];
    }
    return used;
}
