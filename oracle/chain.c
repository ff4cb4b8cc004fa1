/*
 * Trailing-update arithmetic of the oracle's LU in the factorisation's own
 * arithmetic precision T (fp32 or fp64).
 *
 * TEST INFRASTRUCTURE ONLY: built and loaded by oracle/native.py, used by
 * oracle/lu.py.  It shares no code with the CUDA library.
 *
 * Algorithm 4 (first step) factors A in precision u_f.  A dot product "in
 * precision T" is taken here as the plain left-to-right accumulation with a
 * fused multiply-add in T for each term, starting from zero, so that every
 * term costs exactly one rounding:
 *
 *     acc = 0;  for m = 0 .. K-1:  acc = fma_T(L[i][m], U[m][j], acc)
 *     C[i][j] = fl_T(C[i][j] - acc)
 *
 * fmaf / fma are the C99 fused multiply-adds (exact product and sum, one
 * rounding to nearest even; glibc provides them in software where the CPU
 * lacks the instruction).  Build with -ffp-contract=off so that the
 * compiler fuses nothing else.  Rows are independent, so the OpenMP loop
 * gives the same bits for any thread count.
 *
 * Layout: row-major; L is M x K (leading dimension ldl), U is K x N (ldu),
 * C is M x N (ldc), all updated in place in C.
 */
#include <math.h>
#include <stdlib.h>

void oracle_chain_update_f32(long M, long N, long K, const float* L, long ldl,
                             const float* U, long ldu, float* C, long ldc) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < M; ++i) {
    float* acc = (float*)calloc((size_t)(N > 0 ? N : 1), sizeof(float));
    for (long m = 0; m < K; ++m) {
      const float l = L[i * ldl + m];
      const float* u = U + m * ldu;
      for (long j = 0; j < N; ++j) acc[j] = fmaf(l, u[j], acc[j]);
    }
    float* c = C + i * ldc;
    for (long j = 0; j < N; ++j) c[j] = c[j] - acc[j];
    free(acc);
  }
}

void oracle_chain_update_f64(long M, long N, long K, const double* L, long ldl,
                             const double* U, long ldu, double* C, long ldc) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < M; ++i) {
    double* acc = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    for (long m = 0; m < K; ++m) {
      const double l = L[i * ldl + m];
      const double* u = U + m * ldu;
      for (long j = 0; j < N; ++j) acc[j] = fma(l, u[j], acc[j]);
    }
    double* c = C + i * ldc;
    for (long j = 0; j < N; ++j) c[j] = c[j] - acc[j];
    free(acc);
  }
}
