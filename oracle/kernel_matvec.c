/* Exact product Y = A X with the exponential covariance matrix (oracle; test infrastructure).
 *
 * Section 6: A_ij = exp(-||x_i - x_j||_2 / ell) + nugget * delta_ij for the points x (N x d,
 * row-major).  Every entry is generated from its definition and used once; nothing is stored.
 * X and Y are N x nrhs, column-major.  Rows are shared out over OpenMP threads; each row's sum
 * runs over j in increasing order.  Only the tests, the golden-value scripts beside them and the
 * CPU baseline call this. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

int oracle_kernel_matvec(const double* x, int64_t N, int d, double ell, double nugget, int nrhs,
                         const double* X, double* Y) {
  if (N < 0 || d < 1 || d > 3 || nrhs < 1 || nrhs > 64 || !(ell > 0.0)) return -1;
#pragma omp parallel for schedule(dynamic, 32)
  for (int64_t i = 0; i < N; ++i) {
    double acc[64];
    for (int c = 0; c < nrhs; ++c) acc[c] = 0.0;
    const double* xi = x + i * d;
    for (int64_t j = 0; j < N; ++j) {
      const double* xj = x + j * d;
      double s = 0.0;
      for (int t = 0; t < d; ++t) {
        const double diff = xi[t] - xj[t];
        s += diff * diff;
      }
      const double a = exp(-sqrt(s) / ell);
      for (int c = 0; c < nrhs; ++c) acc[c] += a * X[j + c * N];
    }
    for (int c = 0; c < nrhs; ++c) Y[i + c * N] = acc[c] + nugget * X[i + c * N];
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
