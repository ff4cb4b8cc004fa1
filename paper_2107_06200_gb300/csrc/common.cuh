// Device-side helpers shared by the MSIR kernels: number formats, explicit
// IEEE rounding, double-double arithmetic, bounded waits and the grid
// barrier of the persistent kernels.
//
// Every arithmetic step whose rounding the method fixes uses an explicitly
// rounded intrinsic (__fmul_rn, __fsub_rn, __dadd_rn, ...), which the
// compiler never contracts into a fused multiply-add.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/msir.h"

namespace msir {

// ------------------------------------------------------------------ formats

template <typename F> struct Fmt;
template <> struct Fmt<__half> {
  using T = float;  // arithmetic precision of the panel and the u_f solves
  static constexpr int code = MSIR_FP16;
};
template <> struct Fmt<__nv_bfloat16> {
  using T = float;
  static constexpr int code = MSIR_BF16;
};
template <> struct Fmt<float> {
  using T = float;
  static constexpr int code = MSIR_FP32;
};
template <> struct Fmt<double> {
  using T = double;
  static constexpr int code = MSIR_FP64;
};

__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

template <typename F> __device__ __forceinline__ F from_t(float v);
template <> __device__ __forceinline__ __half from_t<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_t<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ float from_t<float>(float v) { return v; }
template <typename F> __device__ __forceinline__ F from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __half from_d<__half>(double v) {
  return __float2half_rn(__double2float_rn(v));  // 16-bit formats round from fp32
}
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn(__double2float_rn(v));
}

// Round a double to the format with code `fmt` and return it as a double.
__device__ __forceinline__ double round_to(double v, int fmt) {
  switch (fmt) {
    case MSIR_FP32: return (double)__double2float_rn(v);
    case MSIR_FP16: return (double)__half2float(__float2half_rn(__double2float_rn(v)));
    case MSIR_BF16: return (double)__bfloat162float(__float2bfloat16_rn(__double2float_rn(v)));
    default: return v;
  }
}
__device__ __forceinline__ float round_f(float v, int fmt) {
  switch (fmt) {
    case MSIR_FP16: return __half2float(__float2half_rn(v));
    case MSIR_BF16: return __bfloat162float(__float2bfloat16_rn(v));
    default: return v;
  }
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ------------------------------------------------------------ double-double
// Knuth TwoSum, Dekker FastTwoSum, TwoProduct via fma, and the accurate dd
// addition of Hida, Li and Bailey's QD library (restated from its paper).

struct dd_t {
  double hi, lo;
};

__device__ __forceinline__ dd_t two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd_t fast_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double e = __dsub_rn(b, __dsub_rn(s, a));
  return {s, e};
}
// The sum and error of two_sum in three fp64 instructions: Dekker's
// FastTwoSum is exact once its first operand is the larger in magnitude,
// and the magnitudes are ordered here on the bit patterns (integer
// instructions; the order of non-negative doubles is that of their bits).
__device__ __forceinline__ dd_t two_sum_ord(double a, double b) {
  const unsigned long long ia = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
  const unsigned long long ib = (unsigned long long)__double_as_longlong(b) & 0x7fffffffffffffffull;
  const bool ab = ia >= ib;
  const double x = ab ? a : b, y = ab ? b : a;
  const double s = __dadd_rn(x, y);
  return {s, __dsub_rn(y, __dsub_rn(s, x))};
}
__device__ __forceinline__ dd_t two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  double e = __fma_rn(a, b, -p);
  return {p, e};
}
// The same error-free transformations in fp32, for the compensated fp32
// sums (Ogita, Rump and Oishi's Dot2): a running sum s and the sum c of the
// exact rounding errors of every product and addition; fl(s + c) is the
// accurately rounded sum except within about n u^2 of a rounding boundary.
struct ff_t {
  float s, c;
};
// FastTwoSum with the operands ordered by magnitude on their bit patterns
// (exact sum and error, as Knuth's TwoSum gives them).
__device__ __forceinline__ void two_sum_ord_f(float a, float b, float& s, float& e) {
  const unsigned ia = __float_as_uint(a) & 0x7fffffffu, ib = __float_as_uint(b) & 0x7fffffffu;
  const bool ab = ia >= ib;
  const float x = ab ? a : b, y = ab ? b : a;
  s = __fadd_rn(x, y);
  e = __fsub_rn(y, __fsub_rn(s, x));
}
// acc + x*y with the product's and the sum's rounding errors kept in acc.c
__device__ __forceinline__ ff_t ff_fma(float x, float y, ff_t acc) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);
  float s, e;
  two_sum_ord_f(acc.s, p, s, e);
  return ff_t{s, __fadd_rn(acc.c, __fadd_rn(e, pe))};
}
__device__ __forceinline__ ff_t ff_merge(ff_t a, ff_t b) {
  float s, e;
  two_sum_ord_f(a.s, b.s, s, e);
  return ff_t{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
}
__device__ __forceinline__ float ff_fin(ff_t a) { return __fadd_rn(a.s, a.c); }
// fl(w - (a.s + a.c)): the difference w - a.s is formed exactly first
__device__ __forceinline__ float ff_sub_from(float w, ff_t a) {
  float s, e;
  two_sum_ord_f(w, -a.s, s, e);
  return __fadd_rn(s, __fsub_rn(e, a.c));
}
__device__ __forceinline__ ff_t ff_shfl_xor(ff_t a, int m) {
  return ff_t{__shfl_xor_sync(0xffffffffu, a.s, m), __shfl_xor_sync(0xffffffffu, a.c, m)};
}

__device__ __forceinline__ dd_t dd_add(dd_t a, dd_t b) {
  dd_t s = two_sum(a.hi, b.hi);
  dd_t t = two_sum(a.lo, b.lo);
  double e = __dadd_rn(s.lo, t.hi);
  dd_t u = fast_two_sum(s.hi, e);
  e = __dadd_rn(u.lo, t.lo);
  return fast_two_sum(u.hi, e);
}
__device__ __forceinline__ dd_t dd_neg(dd_t a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd_t dd_sub(dd_t a, dd_t b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd_t dd_mul_d(dd_t a, double d) {
  dd_t p = two_prod(a.hi, d);
  double e = __dadd_rn(p.lo, __dmul_rn(a.lo, d));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dd_t dd_mul(dd_t a, dd_t b) {
  dd_t p = two_prod(a.hi, b.hi);
  double e = __dadd_rn(p.lo, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dd_t dd_div_d(dd_t a, double d) {
  double q1 = __ddiv_rn(a.hi, d);
  dd_t r = dd_sub(a, dd_mul_d(dd_t{d, 0.0}, q1));
  double q2 = __ddiv_rn(r.hi, d);
  r = dd_sub(r, dd_mul_d(dd_t{d, 0.0}, q2));
  double q3 = __ddiv_rn(r.hi, d);
  dd_t q = fast_two_sum(q1, q2);
  return dd_add(q, dd_t{q3, 0.0});
}
__device__ __forceinline__ dd_t dd_shfl_xor(dd_t a, int m) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

// ------------------------------------------------------------ widening

// fp32 -> fp64 from the IEEE 754 binary32 and binary64 layouts: the sign
// bit stays, the 8-bit exponent is rebiased from 127 to 1023 (+896) into the
// 11-bit field, and the 23 fraction bits become the top of the 52-bit
// fraction.  Integer instructions only; exact for zeros and normal numbers.
// Subnormals, infinities and NaNs need the hardware conversion: callers test
// widen_special() first (one warp vote for a group of values).  On GB300 the
// hardware conversion runs on the narrow fp64 pipe, where it costs as much
// as the fused multiply-add it feeds.
__device__ __forceinline__ double widen_normal(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned mag = b & 0x7fffffffu;
  const unsigned hi = mag == 0u ? (b & 0x80000000u) : ((b & 0x80000000u) | ((mag >> 3) + 0x38000000u));
  return __hiloint2double((int)hi, (int)(b << 29));
}
// subnormal (magnitude bits 1 .. 2^23 - 1), infinity or NaN (exponent 255)
__device__ __forceinline__ bool widen_special(float f) {
  const unsigned mag = __float_as_uint(f) & 0x7fffffffu;
  return mag - 1u < 0x007fffffu || mag >= 0x7f800000u;
}
__device__ __forceinline__ bool widen_special4(const float4& f) {
  return widen_special(f.x) | widen_special(f.y) | widen_special(f.z) | widen_special(f.w);
}

// ------------------------------------------------------------ waits

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

// Deadline of every device-side wait.  A legitimate wait lasts micro- to
// milliseconds; after this the waiter records MSIR_ERR_TIMEOUT and returns.
constexpr unsigned long long kWaitTimeoutNs = 4000000000ull;

// Record a wait that ran out: the first one sets *err to MSIR_ERR_TIMEOUT
// and leaves, in err[22..26], where it happened (site, block, three
// site-specific values) for the host's diagnostics.  err points into an
// int array of at least 27 entries.
__device__ __forceinline__ void record_timeout(int* err, int site, int v0, int v1, int v2) {
  if (atomicCAS(err, 0, (int)MSIR_ERR_TIMEOUT) == 0) {
    err[22] = site;
    err[23] = (int)blockIdx.x;
    err[24] = v0;
    err[25] = v1;
    err[26] = v2;
  }
}

// Grid-wide barrier for a cooperative launch of G blocks.  `count` grows by
// G per episode and is zeroed by the host before the launch.  Returns false
// (after recording the error) on timeout or if another block failed.
__device__ __forceinline__ bool grid_barrier_for(unsigned* count, int* err, unsigned G,
                                                 unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    unsigned old = atom_add_release_u32(count, 1u);
    unsigned target = (old / G + 1u) * G;
    unsigned long long t0 = gtimer();
    unsigned spins = 0;
    while ((int)(ld_acquire_u32(count) - target) < 0) {
      __nanosleep(20);
      if ((++spins & 63u) == 0u) {
        if (ld_volatile_i32(err) != 0) { ok = 0; break; }
        if (gtimer() - t0 > limit_ns) {
          record_timeout(err, 1, (int)ld_acquire_u32(count), (int)target, (int)G);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
__device__ __forceinline__ bool grid_barrier(unsigned* count, int* err, unsigned G) {
  return grid_barrier_for(count, err, G, kWaitTimeoutNs);
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
__device__ __forceinline__ dd_t warp_sum_dd(dd_t v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = dd_add(v, dd_shfl_xor(v, m));
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// max that propagates NaN (an Inf/NaN anywhere must reach the controller)
__device__ __forceinline__ double nanmax(double a, double b) {
  if (isnan(a) || isnan(b)) return __longlong_as_double(0x7ff8000000000000ll);
  return a > b ? a : b;
}
__device__ __forceinline__ double warp_nanmax_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

}  // namespace msir
