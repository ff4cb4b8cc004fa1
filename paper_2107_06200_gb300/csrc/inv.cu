// Inverses of the 64x64 diagonal blocks of the packed LU factors, used by
// the block substitutions of the refinement kernel (each diagonal block of
// L and U is applied through its inverse; see refine_impl.cuh).  One CTA
// per (block, triangle); the arithmetic is in inv_impl.cuh.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "inv_impl.cuh"
#include "kernels.h"

namespace msir {
namespace {

template <typename F>
__global__ void __launch_bounds__(kInvThreads, 1)
    inv_diag_kernel(const F* __restrict__ LU, int ldf, int n, int nblk, float* inv32,
                    double* inv_hi, double* inv_lo) {
  extern __shared__ __align__(16) double sm_inv[];
  inv_diag_block<F>(LU, ldf, n, nblk, blockIdx.x, blockIdx.y == 0, inv32, inv_hi, inv_lo, sm_inv);
}

template <typename F>
cudaError_t launch_inv_t(const void* LU, int ldf, int n, float* inv32, double* inv_hi,
                         double* inv_lo, cudaStream_t st) {
  const int nblk = (n + kIB - 1) / kIB;
  const size_t smem = kInvSmem;
  cudaError_t e = cudaFuncSetAttribute(inv_diag_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  inv_diag_kernel<F><<<dim3(nblk, 2), kInvThreads, smem, st>>>((const F*)LU, ldf, n, nblk, inv32,
                                                               inv_hi, inv_lo);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_inv_diag(int fmt, const void* LU, int ldf, int n, float* inv32, double* inv_hi,
                            double* inv_lo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (fmt) {
    case MSIR_FP16: return launch_inv_t<__half>(LU, ldf, n, inv32, inv_hi, inv_lo, st);
    case MSIR_BF16: return launch_inv_t<__nv_bfloat16>(LU, ldf, n, inv32, inv_hi, inv_lo, st);
    case MSIR_FP32: return launch_inv_t<float>(LU, ldf, n, inv32, inv_hi, inv_lo, st);
    case MSIR_FP64: return launch_inv_t<double>(LU, ldf, n, inv32, inv_hi, inv_lo, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace msir
