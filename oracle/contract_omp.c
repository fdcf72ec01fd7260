/*
 * contract_omp.c -- test infrastructure: the CPU baseline of the benchmark.
 *
 * The oracle's mode-1 contraction loop (Algorithm 3 step (i): unfold_1 of
 * A.(X,Y)_{2,3}) written as plain C over the stored entries grouped by
 * row, FP64, with OpenMP over rows so that it runs on every host core:
 *
 *   out[i + m (a + p b)] = sum over stored (i, j, k) of v X[j + m a] Y[k + n b]
 *
 * X is m x p and Y n x q, column-major; rowptr[i] .. rowptr[i+1] are the
 * stored entries of row i.  Only the benchmark's CPU-baseline leg calls it;
 * it shares nothing with the CUDA library.
 */
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_omp_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

/* nthreads: OpenMP threads (the caller passes the host's core count) */
void oracle_mode1_omp(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* j,
                      const int32_t* k, const double* v, const double* X, int p, const double* Y,
                      int q, double* out, int nthreads) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (i = 0; i < m; ++i) {
    double acc[64];
    int c, a, b;
    int64_t e;
    for (c = 0; c < p * q; ++c) acc[c] = 0.0;
    for (e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double ve = v[e];
      for (b = 0; b < q; ++b) {
        const double vy = ve * Y[k[e] + n * b];
        for (a = 0; a < p; ++a) acc[a + p * b] += vy * X[j[e] + m * a];
      }
    }
    for (c = 0; c < p * q; ++c) out[i + m * c] = acc[c];
  }
}
