// Trailing update of the bf16/fp16 LU on the 5th-generation tensor cores:
//   A22 <- fl_f(fl_32(A22 - L21 U12))
// (Algorithm 4, first step: the O(n^3) part of the factorisation in u_f).
//
// Persistent, warp-specialised kernel (one CTA per SM, 192 threads):
//   warp 0      TMA producer: 128x64 tiles of L21 (from the matrix) and of
//               U12^T (a K-major copy written by lu_outer_swap_trsm) into a
//               4-stage shared-memory ring, 128-byte swizzled;
//   warp 1      allocates 256 TMEM columns (two 128x128 fp32 accumulators)
//               and, from one thread, issues tcgen05.mma (kind::f16, M=128,
//               N=128, K=16) and tcgen05.commit;
//   warps 2..5  epilogue: tcgen05.ld of one accumulator while the other is
//               being filled, subtract from A22 in fp32, round to u_f, store.
// Every mbarrier wait is bounded; on timeout the kernel records
// MSIR_ERR_TIMEOUT, every role leaves its loop, TMEM is freed and the kernel
// returns.  No multicast is used.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"

namespace msir {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 4, TC_THREADS = 192;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr uint32_t TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_TMEM_COLS = 2 * TC_BN;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase.  false: timed out (recorded) or aborted.
__device__ __noinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int* abort_flag,
                                       int* err) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(addr, parity)) return true;
    if ((i & 31u) == 31u) {
      if (*abort_flag) return false;
      unsigned long long t = gtimer();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kWaitTimeoutNs) {
        *abort_flag = 1;
        record_timeout(err, 4, (int)addr, (int)parity, (int)threadIdx.x);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::f16: fp32 accumulator, A/B fp16 (0) or bf16
// (1), both K-major, N = 128, M = 128.
__device__ __forceinline__ uint32_t make_idesc(int ab_fmt) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) |
         ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <typename F> __device__ __forceinline__ F cvt_out(float v);
template <> __device__ __forceinline__ __half cvt_out<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// One epilogue row's C in full 32-column chunks of tile column tn (the
// chunks that reach past N are left alone; the epilogue reads them itself).
template <typename F>
__device__ __forceinline__ void load_c_row(const F* C, int ldc, int M, int N, int row, int tn,
                                           uint4 (&dst)[TC_BN / 32][4]) {
#pragma unroll
  for (int cc = 0; cc < TC_BN / 32; ++cc) {
    const int col0 = tn * TC_BN + cc * 32;
    if (row < M && col0 + 32 <= N) {
      const uint4* src = (const uint4*)(C + (size_t)row * ldc + col0);
#pragma unroll
      for (int v = 0; v < 4; ++v) dst[cc][v] = src[v];
    }
  }
}

template <typename F>
__global__ void __launch_bounds__(TC_THREADS, 1)
    lu_update_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 TcUpdateArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (a.M + TC_BM - 1) / TC_BM;
  const int tiles_n = (a.N + TC_BN - 1) / TC_BN;
  const int ntiles = tiles_m * tiles_n;
  const int KC = a.K / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull_bar[b]), 1);
      mbar_init(smem_u32(&tempty_bar[b]), 128);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int s = 0;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x) {
      const int tm = t % tiles_m, tn = t / tiles_m;
      for (int kc = 0; kc < KC; ++kc) {
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &s_abort, a.err)) break;
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, TC_STAGE_BYTES);
        const uint32_t sa = base + s * TC_STAGE_BYTES;
        tma_load_2d(sa, &tmA, a.a_col0 + kc * TC_BK, a.a_row0 + tm * TC_BM, fb);
        tma_load_2d(sa + TC_A_BYTES, &tmB, kc * TC_BK, a.b_row0 + tn * TC_BN, fb);
        if (++s == TC_STAGES) { s = 0; ph ^= 1u; }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // --------------------------------------------------------- MMA issue
    const uint32_t idesc = make_idesc(Fmt<F>::code == MSIR_BF16 ? 1 : 0);
    int s = 0;
    uint32_t ph = 0;
    int tl = 0;
    for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x, ++tl) {
      const int ab = tl & 1;
      const uint32_t aph = (uint32_t)(tl >> 1) & 1u;
      if (!mbar_wait(smem_u32(&tempty_bar[ab]), aph ^ 1u, &s_abort, a.err)) break;
      tc_fence_after();
      const uint32_t dt = tmem + (uint32_t)(ab * TC_BN);
      bool ok = true;
      for (int kc = 0; kc < KC; ++kc) {
        if (!mbar_wait(smem_u32(&full_bar[s]), ph, &s_abort, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = base + s * TC_STAGE_BYTES;
        const uint32_t sb = sa + TC_A_BYTES;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          umma_f16(dt, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc,
                   (kc | kk) != 0 ? 1u : 0u);
        umma_commit(smem_u32(&empty_bar[s]));
        if (++s == TC_STAGES) { s = 0; ph ^= 1u; }
      }
      if (!ok) break;
      umma_commit(smem_u32(&tfull_bar[ab]));
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    F* C = (F*)a.C;
    int tl = 0;
    // this row's C is loaded one tile ahead (C does not depend on the
    // accumulator, and tiles' C regions are disjoint): the loads of the
    // next tile are in flight while this one waits for its accumulator and
    // is written back
    uint4 cnext[TC_BN / 32][4];
    if ((int)blockIdx.x < ntiles)
      load_c_row<F>(C, a.ldc, a.M, a.N, ((int)blockIdx.x % tiles_m) * TC_BM + q * 32 + lane,
                    (int)blockIdx.x / tiles_m, cnext);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int ab = tl & 1;
      const uint32_t aph = (uint32_t)(tl >> 1) & 1u;
      const int tm = t % tiles_m, tn = t / tiles_m;
      const int row = tm * TC_BM + q * 32 + lane;
      uint4 craw[TC_BN / 32][4];
#pragma unroll
      for (int cc = 0; cc < TC_BN / 32; ++cc)
#pragma unroll
        for (int v = 0; v < 4; ++v) craw[cc][v] = cnext[cc][v];
      const int t2 = t + (int)gridDim.x;
      if (t2 < ntiles)
        load_c_row<F>(C, a.ldc, a.M, a.N, (t2 % tiles_m) * TC_BM + q * 32 + lane, t2 / tiles_m, cnext);
      if (!mbar_wait(smem_u32(&tfull_bar[ab]), aph, &s_abort, a.err)) break;
      tc_fence_after();
#pragma unroll
      for (int cc = 0; cc < TC_BN / 32; ++cc) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * TC_BN + cc * 32), r);
        const int col0 = tn * TC_BN + cc * 32;
        if (row < a.M && col0 < a.N) {
          F* crow = C + (size_t)row * a.ldc + col0;
          if (col0 + 32 <= a.N) {
            uint4 raw[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) raw[v] = craw[cc][v];
            F* h = (F*)raw;
#pragma unroll
            for (int e = 0; e < 32; ++e)
              h[e] = cvt_out<F>(__fsub_rn(to_f(h[e]), __uint_as_float(r[e])));
#pragma unroll
            for (int v = 0; v < 4; ++v) ((uint4*)crow)[v] = raw[v];
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (col0 + e < a.N) crow[e] = cvt_out<F>(__fsub_rn(to_f(crow[e]), __uint_as_float(r[e])));
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[ab]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

cudaError_t launch_update_tc(int fmt, const void* tmA, const void* tmB, const TcUpdateArgs& a,
                             int max_ctas, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.K % TC_BK || max_ctas < 1) return cudaErrorInvalidValue;
  const int ntiles = ((a.M + TC_BM - 1) / TC_BM) * ((a.N + TC_BN - 1) / TC_BN);
  const int grid = ntiles < max_ctas ? ntiles : max_ctas;
  const size_t smem = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024;
  CUtensorMap A, B;
  memcpy(&A, tmA, sizeof(CUtensorMap));
  memcpy(&B, tmB, sizeof(CUtensorMap));
  cudaError_t e;
  if (fmt == MSIR_FP16) {
    e = cudaFuncSetAttribute(lu_update_tc<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    lu_update_tc<__half><<<grid, TC_THREADS, smem, st>>>(A, B, a);
  } else if (fmt == MSIR_BF16) {
    e = cudaFuncSetAttribute(lu_update_tc<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lu_update_tc<__nv_bfloat16><<<grid, TC_THREADS, smem, st>>>(A, B, a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace msir
