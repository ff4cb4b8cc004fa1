// Ingest / conversion launchers (ingest.cu).
#pragma once

#include <cuda_runtime.h>

namespace msir {

cudaError_t ingest_matrix(const double* Ain, int lda, int n, int u0, void* Au, int ldu, cudaStream_t st);
cudaError_t row_stats(const void* Au, int ldu, int n, int u0, double* rowsum, double* rowmax,
                      cudaStream_t st);
cudaError_t squeeze_scalings(const void* Au, int ldu, int n, int u0, double* rowmax, double* R,
                             double* colmax, double* S, cudaStream_t st);
cudaError_t make_factor_matrix(const void* Au, int ldu, int n, int u0, int uf, void* Af, int ldf,
                               const double* R, const double* S, double mu, cudaStream_t st);
cudaError_t round_vec(const double* in, int n, int fmt, double* out, cudaStream_t st);
cudaError_t max_abs(const double* v, int n, int absval, double* out, cudaStream_t st);
cudaError_t ipiv_to_perm(const int* ipiv, int n, int* perm, cudaStream_t st);
cudaError_t iota(int* p, int n, cudaStream_t st);
cudaError_t copy_vec(const double* src, int n, double* dst, cudaStream_t st);

}  // namespace msir
