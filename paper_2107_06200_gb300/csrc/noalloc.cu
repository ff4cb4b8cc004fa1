// msir_residual_noalloc: the residual r = b - A x of Algorithm 4 computed
// without any device allocation, for callers that may not allocate.
//
// Some callers cannot call cudaMalloc at all: code embedded in a host
// runtime whose memory manager owns every device allocation (plugins,
// serving frameworks with fixed pools), or code that must not trigger an
// allocation while a stream is being captured.  This entry point takes the
// caller's input and output buffers and keeps its only scratch -- one
// partial maximum per thread block and a completion counter -- in a
// file-scope device array that every GPU loading the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNaThreads = 128;                 // one row per thread
constexpr int kNaMaxBlocks = 1024;              // scratch holds one slot per block
constexpr int kNaMaxN = kNaThreads * kNaMaxBlocks;  // 131072 rows

struct NoallocScratch {
  double partial[kNaMaxBlocks];  // per-block max |r_i|
  unsigned count;                // blocks finished; back to 0 after each call
  unsigned pad[63];
};

// The scratch of every call on this device (modest: about 8 KB).
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__device__ __forceinline__ double to_u0(double v, int u0) {
  return u0 == MSIR_FP32 ? (double)__double2float_rn(v) : v;
}

// Row i per thread; A column-major, so a warp reads 32 consecutive rows of a
// column at a time.  The working copy A_u = fl_u0(A) is formed on the fly.
__global__ void __launch_bounds__(kNaThreads)
    residual_noalloc_kernel(int n, const double* __restrict__ A, int lda, int u0,
                            const double* __restrict__ x, const double* __restrict__ b, int ur,
                            double* r, double* s_out, NoallocScratch* scr) {
  __shared__ double s_w[kNaThreads / 32];
  __shared__ bool s_last;
  const int i = blockIdx.x * kNaThreads + threadIdx.x;
  double m = 0.0;
  if (i < n) {
    const double bi = to_u0(b[i], u0);
    if (ur == MSIR_DD) {
      double sh = 0.0, sc = 0.0;
      for (int j = 0; j < n; ++j) {
        const msir::dd_t p = msir::two_prod(to_u0(A[(size_t)j * lda + i], u0), x[j]);
        const msir::dd_t t = msir::two_sum(sh, p.hi);
        sh = t.hi;
        sc = __dadd_rn(sc, __dadd_rn(t.lo, p.lo));
      }
      const msir::dd_t ax = msir::fast_two_sum(sh, sc);
      const msir::dd_t rr = msir::dd_sub(msir::dd_t{bi, 0.0}, ax);
      r[i] = rr.hi;
      r[n + i] = rr.lo;
      m = fabs(rr.hi);
    } else {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc = __fma_rn(to_u0(A[(size_t)j * lda + i], u0), x[j], acc);
      const double rv = __dsub_rn(bi, acc);
      r[i] = rv;
      m = fabs(rv);
    }
  }
  m = msir::warp_nanmax_d(m);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bm = s_w[0];
    for (int w = 1; w < kNaThreads / 32; ++w) bm = msir::nanmax(bm, s_w[w]);
    scr->partial[blockIdx.x] = bm;
    __threadfence();
    const unsigned done = atomicAdd(&scr->count, 1u);
    s_last = done == gridDim.x - 1;
  }
  __syncthreads();
  // the last block to finish reduces the partials and clears the counter
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double sm = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) sm = msir::nanmax(sm, ((volatile double*)scr->partial)[k]);
    *s_out = sm;
    scr->count = 0;
  }
}

std::mutex g_mu;
NoallocScratch* g_scratch_addr[64] = {};

// Device address of the scratch array for the current device, resolved
// once per device (with that device current) and cached.
NoallocScratch* scratch_for_current_device(cudaError_t* err) {
  int dev = -1;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = (NoallocScratch*)p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" msir_status msir_residual_noalloc(int n, const double* A_dev, int lda, int u0,
                                             const double* x_dev, const double* b_dev, int ur,
                                             double* r_dev, double* s_dev, void* cuda_stream) {
  if (n <= 0 || lda < n || !A_dev || !x_dev || !b_dev || !r_dev || !s_dev) return MSIR_ERR_INVALID;
  if (n > kNaMaxN) return MSIR_ERR_INVALID;
  if ((u0 != MSIR_FP32 && u0 != MSIR_FP64) || (ur != MSIR_FP64 && ur != MSIR_DD)) return MSIR_ERR_INVALID;
  // an error left pending by earlier work on this thread would otherwise be
  // read back below as this launch's failure: report it before launching
  if (cudaPeekAtLastError() != cudaSuccess) return MSIR_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  NoallocScratch* scr = scratch_for_current_device(&e);
  if (!scr) return MSIR_ERR_CUDA;
  const int blocks = (n + kNaThreads - 1) / kNaThreads;
  residual_noalloc_kernel<<<blocks, kNaThreads, 0, (cudaStream_t)cuda_stream>>>(
      n, A_dev, lda, u0, x_dev, b_dev, ur, r_dev, s_dev, scr);
  return cudaGetLastError() == cudaSuccess ? MSIR_OK : MSIR_ERR_CUDA;
}
