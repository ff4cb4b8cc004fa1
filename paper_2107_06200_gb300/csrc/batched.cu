// Launchers of the batched engine (batched_impl.cuh): the persistent solve
// kernel for each working precision, and the batched factorisation.
#include <algorithm>

#include "batched_impl.cuh"

namespace msir {

void* batched_solve_entry_f32();
void* batched_solve_entry_f64();

size_t batch_smem_bytes(int kcap) {
  const size_t lu = std::max(cta_lu_smem<float>(32), cta_lu_smem<double>(16));
  const size_t refine = refine_smem_bytes(kcap);
  return std::max(std::max(lu, kInvSmem), refine);
}

int batched_max_grid(int u0, int kcap) {
  void* fn = u0 == MSIR_FP32 ? batched_solve_entry_f32() : batched_solve_entry_f64();
  const size_t smem = batch_smem_bytes(kcap);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_batched(int u0, const BatchArgs& args, int grid, cudaStream_t st) {
  void* fn = u0 == MSIR_FP32 ? batched_solve_entry_f32() : batched_solve_entry_f64();
  const size_t smem = batch_smem_bytes(args.layout.kcap);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BatchArgs copy = args;
  void* params[] = {&copy};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kBatchThreads), params, smem, st);
}

// a 32-bit integer hash of (index, seed) mapped to [-1, 1)
__global__ void fill_random_kernel(double* A, size_t count, unsigned seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ (unsigned)(i >> 32) * 40503u ^ seed * 2246822519u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    A[i] = (double)h * (2.0 / 4294967296.0) - 1.0;
  }
}

cudaError_t launch_fill_random(double* A, size_t count, unsigned seed, cudaStream_t st) {
  fill_random_kernel<<<1024, 256, 0, st>>>(A, count, seed);
  return cudaGetLastError();
}

size_t batched_factor_ws_bytes(int fmt) {
  const size_t es = fmt == MSIR_FP64 ? 8 : (fmt == MSIR_FP32 ? 4 : 2);
  return ((size_t)kBatchMaxN * kBatchMaxN * es + (size_t)kBatchMaxN * 4 + 255) / 256 * 256;
}

template <typename F>
static cudaError_t launch_factor_t(const BatchFactorTask* tasks, int count, char* ws, size_t ws_stride, int nb,
                                   int nbo, int grid, cudaStream_t st) {
  const size_t smem = cta_lu_smem<F>(nb);
  cudaError_t e = cudaFuncSetAttribute(batched_factor_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  batched_factor_kernel<F><<<grid, kBatchThreads, smem, st>>>(tasks, count, ws, ws_stride, nb, nbo);
  return cudaGetLastError();
}

cudaError_t launch_batched_factor(int fmt, const BatchFactorTask* tasks, int count, char* ws, size_t ws_stride,
                                  int nb, int nbo, int grid, cudaStream_t st) {
  switch (fmt) {
    case MSIR_FP16: return launch_factor_t<__half>(tasks, count, ws, ws_stride, nb, nbo, grid, st);
    case MSIR_BF16: return launch_factor_t<__nv_bfloat16>(tasks, count, ws, ws_stride, nb, nbo, grid, st);
    case MSIR_FP32: return launch_factor_t<float>(tasks, count, ws, ws_stride, nb, nbo, grid, st);
    case MSIR_FP64: return launch_factor_t<double>(tasks, count, ws, ws_stride, nb, nbo, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace msir
