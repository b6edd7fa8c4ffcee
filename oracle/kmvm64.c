/*
 * FP64 kernel product for the CPU oracle (TEST INFRASTRUCTURE ONLY: used by the tests,
 * the smoke check and the benchmark's CPU baseline; the CUDA path never links it).
 *
 * out[r][q] = sum_j exp(-||x_{rows[r]} - x_j||^2 / (2 sigma^2)) V[j][q] + beta V[rows[r]][q]
 *
 * the discrete Gauss transform of Section 2.4, Eq. (6), with h^2 = 2 sigma^2, plus the ridge
 * term of Eq. (2), written straight from the definition: explicit coordinate differences,
 * libm exp, FP64 sums in index order.  X is n x d row-major, V and out are row-major with
 * nrhs columns (V: n x nrhs, out: nrows x nrhs).  rows == NULL means every row.  Rows are
 * shared among OpenMP threads; each output row is summed by one thread, so the result does
 * not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_kmvm(const double* X, long long n, int d, const double* V, int nrhs, double sigma,
                 double beta, const long long* rows, long long nrows, double* out) {
    const double inv = 1.0 / (2.0 * sigma * sigma);
    const long long m = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < m; ++r) {
        const long long i = rows ? rows[r] : r;
        const double* xi = X + i * d;
        double* o = out + r * nrhs;
        for (int q = 0; q < nrhs; ++q) o[q] = 0.0;
        for (long long j = 0; j < n; ++j) {
            const double* xj = X + j * d;
            double dist2 = 0.0;
            for (int c = 0; c < d; ++c) {
                const double diff = xi[c] - xj[c];
                dist2 += diff * diff;
            }
            const double kij = exp(-dist2 * inv);
            const double* vj = V + j * nrhs;
            for (int q = 0; q < nrhs; ++q) o[q] += kij * vj[q];
        }
        for (int q = 0; q < nrhs; ++q) o[q] += beta * V[i * nrhs + q];
    }
}
