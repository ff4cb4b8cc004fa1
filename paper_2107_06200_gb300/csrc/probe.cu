// Throughput probe of the fp64 and fp32 fused multiply-add pipes.
//
// Measurement helper only (the paper has no counterpart): the refinement
// kernel's residual, u^2 operator and double-double arithmetic run on the
// fp64 pipe, and its roofline needs that pipe's peak as measured on this
// device rather than a nominal figure.  Every thread runs kChains
// independent dependent chains of a = fma(a, m, c) (kChains-way
// instruction-level parallelism hides the pipe latency); the grid fills every
// SM several times over.  Work per launch = 2 flops x threads x kChains x
// iters; time = CUDA events around the launch on the caller's stream.
#include <cuda_runtime.h>

#include "../../include/msir.h"
#include "common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T* sink, int iters, T m, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k + 1) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // never true for the values used (keeps the chains live without a store)
  if (s == (T)-1.2345) sink[blockIdx.x] = s;
}

template <typename T>
msir_status run_probe(int device, int iters, double* tflops, double* seconds) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return MSIR_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return MSIR_ERR_CUDA;
  const int blocks = sms * 8;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MSIR_ERR_CUDA;
  msir_status out = MSIR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    out = MSIR_ERR_CUDA;
  } else {
    const T m = (T)0.999999, c = (T)1e-7;
    fma_probe_kernel<T><<<blocks, kProbeThreads, 0, st>>>(nullptr, iters / 8 + 1, m, c);  // warm-up
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<blocks, kProbeThreads, 0, st>>>(nullptr, iters, m, c);
    cudaEventRecord(e1, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      out = MSIR_ERR_CUDA;
    } else {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double flops = 2.0 * (double)blocks * kProbeThreads * kChains * (double)iters;
      *seconds = ms * 1e-3;
      *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return out;
}

// One block enters the library's grid barrier for a grid of two blocks, so
// the second arrival never comes: the barrier's bounded wait runs out after
// limit_ns, records MSIR_ERR_TIMEOUT in err and returns, and so does the
// kernel.
__global__ void wait_timeout_probe_kernel(unsigned* count, int* err, unsigned long long limit_ns) {
  (void)msir::grid_barrier_for(count, err, 2u, limit_ns);
}

// Every fp32 bit pattern: widen_special() must flag exactly the
// subnormals, infinities and NaNs, and widen_normal() must equal the
// hardware conversion, bit for bit, on every other pattern.
__global__ void widen_check_kernel(unsigned long long* out) {
  unsigned long long bad = 0, checked = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32);
       i += stride) {
    const float f = __uint_as_float((unsigned)i);
    const float a = fabsf(f);
    const bool expect = isnan(f) || isinf(f) || (a != 0.0f && a < 1.17549435e-38f);
    const bool sp = msir::widen_special(f);
    if (sp != expect) ++bad;
    if (!sp) {
      ++checked;
      if (__double_as_longlong(msir::widen_normal(f)) != __double_as_longlong((double)f)) ++bad;
    }
  }
  atomicAdd(out, bad);
  atomicAdd(out + 1, checked);
}

}  // namespace

extern "C" msir_status msir_probe_widen_check(int device, unsigned long long* mismatches,
                                              unsigned long long* checked) {
  if (!mismatches || !checked) return MSIR_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return MSIR_ERR_CUDA;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MSIR_ERR_CUDA;
  unsigned long long* d = nullptr;
  msir_status out = MSIR_OK;
  unsigned long long h[2] = {0, 0};
  if (cudaMallocAsync((void**)&d, 16, st) != cudaSuccess || cudaMemsetAsync(d, 0, 16, st) != cudaSuccess) {
    out = MSIR_ERR_CUDA;
  } else {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    widen_check_kernel<<<sms * 8, 256, 0, st>>>(d);
    if (cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      out = MSIR_ERR_CUDA;
  }
  if (d) cudaFreeAsync(d, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  *mismatches = h[0];
  *checked = h[1];
  return out;
}

extern "C" msir_status msir_probe_wait_timeout(int device, double limit_s, int* status) {
  if (!status || !(limit_s > 0.0) || limit_s > 10.0) return MSIR_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return MSIR_ERR_CUDA;
  unsigned* count = nullptr;
  int* err = nullptr;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MSIR_ERR_CUDA;
  msir_status out = MSIR_OK;
  if (cudaMallocAsync((void**)&count, 64, st) != cudaSuccess ||
      cudaMallocAsync((void**)&err, 32 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(count, 0, 64, st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, 32 * sizeof(int), st) != cudaSuccess) {
    out = MSIR_ERR_CUDA;
  } else {
    wait_timeout_probe_kernel<<<1, 32, 0, st>>>(count, err, (unsigned long long)(limit_s * 1e9));
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      out = MSIR_ERR_CUDA;
    else
      *status = h;
  }
  if (count) cudaFreeAsync(count, st);
  if (err) cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  return out;
}

extern "C" msir_status msir_probe_fma_rate(int device, int fmt, int iters, double* tflops,
                                           double* seconds) {
  if (!tflops || !seconds || iters <= 0) return MSIR_ERR_INVALID;
  if (fmt == MSIR_FP64) return run_probe<double>(device, iters, tflops, seconds);
  if (fmt == MSIR_FP32) return run_probe<float>(device, iters, tflops, seconds);
  return MSIR_ERR_INVALID;
}
