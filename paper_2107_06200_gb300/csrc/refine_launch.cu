// Dispatch of the persistent refinement kernel instantiations.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "refine.h"

namespace msir {

template <typename A0, typename F> void* refine_entry();

// ---------------------------------------------------------- launchers

size_t refine_smem_bytes(int kcap) {
  return kTrsvSmem + kScaledSmem + kInboxSmem +
         sizeof(double) * (3 * ((size_t)kcap + 2) + 2 * ((size_t)kcap + 1));
}

template <typename A0, typename F>
static void* refine_fn() {
  return refine_entry<A0, F>();
}

static void* pick(int a_fmt, int f_fmt) {
  if (a_fmt == MSIR_FP32) {
    switch (f_fmt) {
      case MSIR_FP16: return refine_fn<float, __half>();
      case MSIR_BF16: return refine_fn<float, __nv_bfloat16>();
      case MSIR_FP32: return refine_fn<float, float>();
      case MSIR_FP64: return refine_fn<float, double>();
    }
  } else {
    switch (f_fmt) {
      case MSIR_FP16: return refine_fn<double, __half>();
      case MSIR_BF16: return refine_fn<double, __nv_bfloat16>();
      case MSIR_FP32: return refine_fn<double, float>();
      case MSIR_FP64: return refine_fn<double, double>();
    }
  }
  return nullptr;
}

int refine_max_grid(int a_fmt, int f_fmt, int kcap) {
  void* fn = pick(a_fmt, f_fmt);
  if (!fn) return 0;
  const size_t smem = refine_smem_bytes(kcap);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRefThreads, smem) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

static cudaLaunchConfig_t cluster_config(int grid, size_t smem, cudaStream_t st, int cluster,
                                          cudaLaunchAttribute (&at)[2]) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kRefThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cfg;
}

int refine_max_cluster_grid(int a_fmt, int kcap, int cluster) {
  if (cluster < 2 || cluster > kMaxCluster) return 0;
  const size_t smem = refine_smem_bytes(kcap);
  int best = -1;
  for (int f : {MSIR_FP16, MSIR_BF16, MSIR_FP32, MSIR_FP64}) {
    void* fn = pick(a_fmt, f);
    if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(cluster, smem, nullptr, cluster, at);
    cfg.numAttrs = 1;  // the occupancy query takes the cluster shape only
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = best < 0 ? ncl : std::min(best, ncl);
  }
  return best > 0 ? best * cluster : 0;
}

cudaError_t launch_refine(int a_fmt, int f_fmt, const RefineArgs& a, int grid, cudaStream_t st) {
  void* fn = pick(a_fmt, f_fmt);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = refine_smem_bytes(a.kcap);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  RefineArgs copy = a;
  if (a.cluster > 1) {
    if (grid % a.cluster != 0) return cudaErrorInvalidValue;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(grid, smem, st, a.cluster, at);
    void* params[] = {&copy};
    return cudaLaunchKernelExC(&cfg, fn, params);
  }
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kRefThreads), params, smem, st);
}

}  // namespace msir
