// Ingest and conversion kernels.
//
//  * A_u = fl_u0(A): the caller's fp64 column-major matrix becomes the
//    working-precision copy, row-major (32x32 tiles through shared memory
//    so both sides stay coalesced).  Algorithm 4 keeps A in the working
//    precision; this fixes the system that is solved for the whole run.
//  * row sums / row maxima of |A_u| (infinity norm, squeezing scalings);
//    column maxima of |R A_u|.
//  * A_f = fl_uf(A_u), optionally scaled: fl_uf(fl_32(mu R_i a_ij S_j))
//    with power-of-two R, S, mu (the two-sided scaling of Sec. 2.1.2).
//  * vector rounding b_u = fl_u0(b) and infinity norms.
#include "common.cuh"
#include "ingest.h"

namespace msir {

template <typename U0>
__global__ void ingest_matrix_kernel(const double* __restrict__ Ain, int lda, int n, U0* Au, int ldu) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // bx: column block, by: row block
  const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
  for (int r = 0; r < 32; r += 8) {
    const int col = bx + ty + r, row = by + tx;
    tile[ty + r][tx] = (col < n && row < n) ? Ain[(size_t)col * lda + row] : 0.0;
  }
  __syncthreads();
  for (int r = 0; r < 32; r += 8) {
    const int row = by + ty + r, col = bx + tx;
    if (row < n && col < n) Au[(size_t)row * ldu + col] = (U0)tile[tx][ty + r];
  }
}

template <typename U0>
__global__ void row_stats_kernel(const U0* Au, int ldu, int n, double* rowsum, double* rowmax) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const U0* row = Au + (size_t)warp * ldu;
  double s = 0.0, m = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double v = fabs((double)row[j]);
    s = __dadd_rn(s, v);
    m = nanmax(m, v);
  }
  s = warp_sum_d(s);
  m = warp_nanmax_d(m);
  if (lane == 0) {
    if (rowsum) rowsum[warp] = s;
    if (rowmax) rowmax[warp] = m;
  }
}

// scale = 2^-e where m = f 2^e, f in [1/2, 1) (1 for m == 0)
__device__ __forceinline__ double pow2_inv(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 1.0;
  int e;
  frexp(m, &e);
  return ldexp(1.0, -e);
}

__global__ void pow2_scale_kernel(const double* m, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = pow2_inv(m[i]);
}

template <typename U0>
__global__ void col_max_scaled_kernel(const U0* Au, int ldu, int n, const double* R, double* colmax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double m = 0.0;
  for (int i = 0; i < n; ++i) m = nanmax(m, fabs((double)Au[(size_t)i * ldu + j] * R[i]));
  colmax[j] = m;
}

template <typename U0, typename F>
__global__ void make_factor_kernel(const U0* Au, int ldu, int n, F* Af, int ldf, const double* R,
                                   const double* S, double mu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  double v = (double)Au[(size_t)i * ldu + j];
  if (R) v = v * R[i] * S[j] * mu;
  Af[(size_t)i * ldf + j] = from_d<F>(v);
}

__global__ void round_vec_kernel(const double* in, int n, int fmt, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = round_to(in[i], fmt);
}

// single-block NaN-propagating max of |v| or v
__global__ void max_kernel(const double* v, int n, int absval, double* out) {
  __shared__ double sw[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = nanmax(m, absval ? fabs(v[i]) : v[i]);
  m = warp_nanmax_d(m);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
    m = warp_nanmax_d(m);
    if (threadIdx.x == 0) *out = m;
  }
}

__global__ void copy_strided_kernel(const double* src, int n, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// The interchanges are sequential by nature: one thread applies them to a
// permutation held in shared memory (the block stages ipiv and perm).
__global__ void ipiv_to_perm_kernel(const int* ipiv, int n, int* perm) {
  extern __shared__ int sm[];
  int* sp = sm;
  int* si = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { sp[i] = i; si[i] = ipiv[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < n; ++j) {
      const int p = si[j];
      if (p != j) {
        const int t = sp[j];
        sp[j] = sp[p];
        sp[p] = t;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = sp[i];
}

__global__ void iota_kernel(int* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

// ------------------------------------------------------------ launchers

cudaError_t ingest_matrix(const double* Ain, int lda, int n, int u0, void* Au, int ldu, cudaStream_t st) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  if (u0 == MSIR_FP32)
    ingest_matrix_kernel<float><<<grid, block, 0, st>>>(Ain, lda, n, (float*)Au, ldu);
  else
    ingest_matrix_kernel<double><<<grid, block, 0, st>>>(Ain, lda, n, (double*)Au, ldu);
  return cudaGetLastError();
}

cudaError_t row_stats(const void* Au, int ldu, int n, int u0, double* rowsum, double* rowmax,
                      cudaStream_t st) {
  const int threads = 256, blocks = (n * 32 + threads - 1) / threads;
  if (u0 == MSIR_FP32)
    row_stats_kernel<float><<<blocks, threads, 0, st>>>((const float*)Au, ldu, n, rowsum, rowmax);
  else
    row_stats_kernel<double><<<blocks, threads, 0, st>>>((const double*)Au, ldu, n, rowsum, rowmax);
  return cudaGetLastError();
}

cudaError_t squeeze_scalings(const void* Au, int ldu, int n, int u0, double* rowmax, double* R,
                             double* colmax, double* S, cudaStream_t st) {
  cudaError_t e = row_stats(Au, ldu, n, u0, nullptr, rowmax, st);
  if (e != cudaSuccess) return e;
  pow2_scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(rowmax, n, R);
  if (u0 == MSIR_FP32)
    col_max_scaled_kernel<float><<<(n + 127) / 128, 128, 0, st>>>((const float*)Au, ldu, n, R, colmax);
  else
    col_max_scaled_kernel<double><<<(n + 127) / 128, 128, 0, st>>>((const double*)Au, ldu, n, R, colmax);
  pow2_scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(colmax, n, S);
  return cudaGetLastError();
}

template <typename U0>
static cudaError_t make_factor_u0(const U0* Au, int ldu, int n, int uf, void* Af, int ldf,
                                  const double* R, const double* S, double mu, cudaStream_t st) {
  dim3 grid((n + 255) / 256, n);
  switch (uf) {
    case MSIR_FP16: make_factor_kernel<U0, __half><<<grid, 256, 0, st>>>(Au, ldu, n, (__half*)Af, ldf, R, S, mu); break;
    case MSIR_BF16: make_factor_kernel<U0, __nv_bfloat16><<<grid, 256, 0, st>>>(Au, ldu, n, (__nv_bfloat16*)Af, ldf, R, S, mu); break;
    case MSIR_FP32: make_factor_kernel<U0, float><<<grid, 256, 0, st>>>(Au, ldu, n, (float*)Af, ldf, R, S, mu); break;
    case MSIR_FP64: make_factor_kernel<U0, double><<<grid, 256, 0, st>>>(Au, ldu, n, (double*)Af, ldf, R, S, mu); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t make_factor_matrix(const void* Au, int ldu, int n, int u0, int uf, void* Af, int ldf,
                               const double* R, const double* S, double mu, cudaStream_t st) {
  if (u0 == MSIR_FP32) return make_factor_u0<float>((const float*)Au, ldu, n, uf, Af, ldf, R, S, mu, st);
  return make_factor_u0<double>((const double*)Au, ldu, n, uf, Af, ldf, R, S, mu, st);
}

cudaError_t round_vec(const double* in, int n, int fmt, double* out, cudaStream_t st) {
  round_vec_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, n, fmt, out);
  return cudaGetLastError();
}

cudaError_t max_abs(const double* v, int n, int absval, double* out, cudaStream_t st) {
  max_kernel<<<1, 1024, 0, st>>>(v, n, absval, out);
  return cudaGetLastError();
}

cudaError_t ipiv_to_perm(const int* ipiv, int n, int* perm, cudaStream_t st) {
  const size_t smem = (size_t)2 * n * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(ipiv_to_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ipiv_to_perm_kernel<<<1, 1024, smem, st>>>(ipiv, n, perm);
  return cudaGetLastError();
}

cudaError_t iota(int* p, int n, cudaStream_t st) {
  iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

cudaError_t copy_vec(const double* src, int n, double* dst, cudaStream_t st) {
  copy_strided_kernel<<<(n + 255) / 256, 256, 0, st>>>(src, n, dst);
  return cudaGetLastError();
}

}  // namespace msir
