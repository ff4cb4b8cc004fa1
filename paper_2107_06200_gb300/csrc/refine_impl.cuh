// Persistent refinement kernel: the loop of Algorithm 4 after the LU.
//
// One cooperative launch runs SIR, SGMRES-IR and GMRES-IR steps, the
// stopping criteria of Sec. 2.1.1 and the stage switches, entirely on the
// device; it returns to the host only when the run has converged, has
// nothing left to try, or needs the factorisation redone in a finer u_f
// (the host then relaunches it in phase PH_ESCALATED).
//
// Work distribution: rows are grouped in blocks of kBlk = 64; CTA c owns
// blocks c, c+G, c+2G, ...  Residual and operator rows are produced in the
// pivoted order i -> perm[i], so the forward substitution of a block needs
// only rows its own CTA computed.  Triangular solves are wavefronts: a CTA
// accumulates the off-diagonal products of its block as soon as the blocks
// it depends on publish their values (epoch-tagged 64-bit words), then
// applies the inverse of its diagonal block and publishes.
// Grid barriers are used only where a full vector is needed (matrix-vector
// products) or a global reduction (norms, Gram-Schmidt coefficients).  The
// stage controller is replicated in every CTA: all CTAs compute the same
// decisions from the same reduced values, so control flow stays uniform.
// All waits are bounded (MSIR_ERR_TIMEOUT).
#pragma once

#include "common.cuh"
#include <type_traits>

#include "refine.h"

namespace msir {

// ----------------------------------------------------------- helpers

struct Cx {
  int G, cta, tid, lane, warp, n, nblk;
  int team_k;  // RefineArgs::team_k
  unsigned epoch;
  int redbuf;
  unsigned long long* t_ns;  // per-phase timers (CTA 0, thread 0), shared memory
  unsigned char* tsm;        // shared scratch of the substitutions (kTrsvSmem bytes)
  unsigned char* ssm;        // shared staging of the scaled-block construction (kScaledSmem)
  unsigned mready;           // RefState::mready of this launch (uniform)
  int C;                     // CTAs per cluster (1: no clusters)
  unsigned long long* inbox; // [kMaxCluster][kBlk][kLLWords] words written by cluster peers
};

// Phase timer: CTA 0 / thread 0 accumulates %globaltimer deltas.
struct PhaseTimer {
  Cx& cx;
  int ph;
  unsigned long long t0;
  __device__ PhaseTimer(Cx& c, int p) : cx(c), ph(p), t0(0) {
    if (cx.cta == 0 && cx.tid == 0) t0 = gtimer();
  }
  __device__ ~PhaseTimer() {
    if (cx.cta == 0 && cx.tid == 0) cx.t_ns[ph] += gtimer() - t0;
  }
};

static __device__ __forceinline__ double urnd(double v, int u) {
  return u == MSIR_FP32 ? (double)__double2float_rn(v) : v;
}
static __device__ __forceinline__ double umul(double a, double b, int u) {
  return u == MSIR_FP32 ? (double)__fmul_rn((float)a, (float)b) : __dmul_rn(a, b);
}
static __device__ __forceinline__ double uadd(double a, double b, int u) {
  return u == MSIR_FP32 ? (double)__fadd_rn((float)a, (float)b) : __dadd_rn(a, b);
}
static __device__ __forceinline__ double usub(double a, double b, int u) {
  return u == MSIR_FP32 ? (double)__fsub_rn((float)a, (float)b) : __dsub_rn(a, b);
}
static __device__ __forceinline__ double udiv(double a, double b, int u) {
  return u == MSIR_FP32 ? (double)__fdiv_rn((float)a, (float)b) : __ddiv_rn(a, b);
}
static __device__ __forceinline__ double usqrt(double a, int u) {
  return u == MSIR_FP32 ? (double)__fsqrt_rn((float)a) : __dsqrt_rn(a);
}
static __device__ __forceinline__ int square_of(int u) { return u == MSIR_FP32 ? MSIR_FP64 : MSIR_DD; }
static __device__ __forceinline__ double unit_roundoff(int f) {
  switch (f) {
    case MSIR_BF16: return 0x1p-8;
    case MSIR_FP16: return 0x1p-11;
    case MSIR_FP32: return 0x1p-24;
    case MSIR_FP64: return 0x1p-53;
    default: return 0x1p-106;
  }
}

template <typename A0> struct AV;
template <> struct AV<float> {
  static __device__ __forceinline__ double ld(const float* p) { return (double)__ldg(p); }
};
template <> struct AV<double> {
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
};

// Four consecutive values widened to double from a 16-byte aligned
// address: matrix rows through the read-only path, vectors through L2
// (they are rewritten during the kernel).
template <typename T> struct Ld4;
template <> struct Ld4<float> {
  static __device__ __forceinline__ void row(const float* p, double (&v)[4]) {
    const float4 f = __ldg((const float4*)p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  }
  static __device__ __forceinline__ void vec(const float* p, double (&v)[4]) {
    const float4 f = __ldcg((const float4*)p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  }
};
template <> struct Ld4<double> {
  static __device__ __forceinline__ void row(const double* p, double (&v)[4]) {
    const double2 f = __ldg((const double2*)p), g = __ldg((const double2*)p + 1);
    v[0] = f.x; v[1] = f.y; v[2] = g.x; v[3] = g.y;
  }
  static __device__ __forceinline__ void vec(const double* p, double (&v)[4]) {
    const double2 f = __ldcg((const double2*)p), g = __ldcg((const double2*)p + 1);
    v[0] = f.x; v[1] = f.y; v[2] = g.x; v[3] = g.y;
  }
};

// Four consecutive values as float (fp32 paths: no fp64 conversions).
template <typename T>
__device__ __forceinline__ void ld4f_row(const T* p, float (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 f = __ldg((const float4*)p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (float)__ldg(p + q);
  }
}
template <typename T>
__device__ __forceinline__ void ld4f_vec(const T* p, float (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 f = __ldcg((const float4*)p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (float)__ldcg(p + q);
  }
}

// Row dot products a_row . x by one warp (result on every lane).  Lanes
// take four consecutive columns at a time with 16-byte loads, several
// steps in flight, so that a warp streams its row at HBM speed; rows start
// on 64-element boundaries, x is checked for 16-byte alignment.
template <typename A0, typename X>
__device__ double row_dot_d(const A0* row, const X* x, int n, int lane) {
  double acc = 0.0;
  const int n4 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) ? (n & ~3) : 0;
#pragma unroll 4
  for (int j = lane * 4; j < n4; j += 128) {
    double av[4], xv[4];
    Ld4<A0>::row(row + j, av);
    Ld4<X>::vec(x + j, xv);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = __fma_rn(av[q], xv[q], acc);
  }
  for (int j = n4 + lane; j < n; j += 32) acc = __fma_rn(AV<A0>::ld(row + j), (double)__ldcg(x + j), acc);
  return warp_sum_d(acc);
}
// row_dot_d for NR rows at once (the same sums, row by row): x is loaded
// once for all rows, and the rows' chains and reductions are independent,
// so one warp keeps more loads and fp64 work in flight.  (The dd product
// keeps one row per warp: it is bound by fp64 throughput, not latency.)
template <typename A0, typename X, int NR>
__device__ void rows_dot_d(const A0* const (&row)[NR], const X* x, int n, int lane, double (&out)[NR]) {
  double acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0.0;
  const int n4 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) ? (n & ~3) : 0;
  if constexpr (sizeof(A0) == 4 && sizeof(X) == 4) {
    // fp32 matrix and vector: widened by integer instructions (the fp64
    // pipe then only does the fused multiply-adds); a step with a subnormal,
    // infinite or NaN operand on any lane takes the hardware conversion.
    // The step loop is warp-uniform (the vote needs every lane): lanes past
    // n4 in the last step load nothing and add zeros.  Two accumulators per
    // row (columns 0, 2 and 1, 3 of each step) keep four independent fp64
    // chains per warp in flight.
    double acc2[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc2[r] = 0.0;
#pragma unroll 2
    for (int j0 = 0; j0 < n4; j0 += 128) {
      const int j = j0 + lane * 4;
      const bool in = j < n4;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 xf = in ? __ldcg((const float4*)(x + j)) : z4;
      float4 af[NR];
      bool sp = widen_special4(xf);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        af[r] = in ? __ldg((const float4*)(row[r] + j)) : z4;
        sp |= widen_special4(af[r]);
      }
      if (__any_sync(0xffffffffu, sp)) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          acc[r] = __fma_rn((double)af[r].x, (double)xf.x, acc[r]);
          acc2[r] = __fma_rn((double)af[r].y, (double)xf.y, acc2[r]);
          acc[r] = __fma_rn((double)af[r].z, (double)xf.z, acc[r]);
          acc2[r] = __fma_rn((double)af[r].w, (double)xf.w, acc2[r]);
        }
      } else {
        const double x0 = widen_normal(xf.x), x1 = widen_normal(xf.y), x2 = widen_normal(xf.z),
                     x3 = widen_normal(xf.w);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          acc[r] = __fma_rn(widen_normal(af[r].x), x0, acc[r]);
          acc2[r] = __fma_rn(widen_normal(af[r].y), x1, acc2[r]);
          acc[r] = __fma_rn(widen_normal(af[r].z), x2, acc[r]);
          acc2[r] = __fma_rn(widen_normal(af[r].w), x3, acc2[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = __dadd_rn(acc[r], acc2[r]);
  } else {
#pragma unroll 2
    for (int j = lane * 4; j < n4; j += 128) {
      double xv[4];
      Ld4<X>::vec(x + j, xv);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double av[4];
        Ld4<A0>::row(row[r] + j, av);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r] = __fma_rn(av[q], xv[q], acc[r]);
      }
    }
  }
  for (int j = n4 + lane; j < n; j += 32) {
    const double xj = (double)__ldcg(x + j);
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = __fma_rn(AV<A0>::ld(row[r] + j), xj, acc[r]);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) out[r] = warp_sum_d(acc[r]);
}
// Compensated (twice-working-precision) dot product, result as dd.
template <typename A0, typename X>
__device__ dd_t row_dot_dd(const A0* row, const X* x, int n, int lane) {
  double s = 0.0, c = 0.0;
  const int n4 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) ? (n & ~3) : 0;
#pragma unroll 2
  for (int j = lane * 4; j < n4; j += 128) {
    double av[4], xv[4];
    Ld4<A0>::row(row + j, av);
    Ld4<X>::vec(x + j, xv);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const dd_t p = two_prod(av[q], xv[q]);
      const dd_t t = two_sum_ord(s, p.hi);
      s = t.hi;
      c = __dadd_rn(c, __dadd_rn(t.lo, p.lo));
    }
  }
  for (int j = n4 + lane; j < n; j += 32) {
    const dd_t p = two_prod(AV<A0>::ld(row + j), (double)__ldcg(x + j));
    const dd_t t = two_sum_ord(s, p.hi);
    s = t.hi;
    c = __dadd_rn(c, __dadd_rn(t.lo, p.lo));
  }
  dd_t v = fast_two_sum(s, c);
  return warp_sum_dd(v);
}

// Reduce NV per-CTA values (each already reduced within the CTA and held by
// thread 0) across the grid.  op[i]: 0 = sum, 1 = NaN-propagating max.
template <int NV>
__device__ bool grid_reduce(Cx& cx, const RefineArgs& a, double (&v)[NV], const int (&op)[NV]) {
  PhaseTimer pt(cx, 5);
  __shared__ double s_res[kRedW];
  double* buf = a.red + (size_t)cx.redbuf * cx.G * kRedW;
  cx.redbuf ^= 1;
  if (cx.tid == 0)
    for (int i = 0; i < NV; ++i) buf[cx.cta * kRedW + i] = v[i];
  if (!grid_barrier(a.bar, a.err, cx.G)) return false;
  if (cx.warp == 0) {
    for (int i = 0; i < NV; ++i) {
      double acc = op[i] ? 0.0 : 0.0;
      for (int c = cx.lane; c < cx.G; c += 32) {
        double q = __ldcg(buf + c * kRedW + i);
        acc = op[i] ? nanmax(acc, q) : __dadd_rn(acc, q);
      }
      acc = op[i] ? warp_nanmax_d(acc) : warp_sum_d(acc);
      if (cx.lane == 0) s_res[i] = acc;
    }
  }
  __syncthreads();
  for (int i = 0; i < NV; ++i) v[i] = s_res[i];
  __syncthreads();
  return true;
}

// CTA-level reduction of one value per thread (thread 0 gets the result).
static __device__ double cta_reduce(double v, int op, int tid) {
  __shared__ double s_w[kRefThreads / 32];
  v = op ? warp_nanmax_d(v) : warp_sum_d(v);
  if ((tid & 31) == 0) s_w[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid == 0) {
    r = s_w[0];
    for (int i = 1; i < kRefThreads / 32; ++i) r = op ? nanmax(r, s_w[i]) : __dadd_rn(r, s_w[i]);
  }
  __syncthreads();
  return r;
}

// ----------------------------------------------------- triangular solves
//
// Block substitution with inverted diagonal blocks.  Block b of the forward
// solve computes z_b = c_b - sum_{j<b} L_bj y_j, then y_b = inv(L_bb) z_b
// rounded to the storage format; the backward solve runs the same way from
// the last block up with U.  The inverses come from inv.cu, in the
// arithmetic format of the solve.
//
// Thread (r, seg) of the CTA owning block b handles row r and the 16
// columns seg*16 .. seg*16+15 of every 64x64 tile of that row block.  As
// the blocks it depends on become available, the CTA accumulates their
// tiles (tile loads and payload loads issued one dependency ahead), so when
// the last one arrives only that tile, a 4-lane reduction, the 64x64
// product with the inverse and another 4-lane reduction remain on the
// critical path.
//
// Hand-off between CTAs: each solved value is published as 64-bit words
// carrying 32 payload bits and the 32-bit epoch of the solve.  A 64-bit
// aligned store or load is single-copy atomic, so a consumer that sees the
// current epoch in a word also sees that word's payload: no flag, fence or
// second round trip is needed.  Epochs grow by one per triangular solve and
// the payload buffer is zeroed whenever the epoch counter restarts.

// N consecutive factor values of one row (N in {4, 8, 16}), widened.  The
// first value's column is a multiple of N and rows start on 64-element
// boundaries, so the N values are aligned to N * sizeof(F) bytes.
__device__ __forceinline__ float h16_to_f(unsigned short b, __half*) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ float h16_to_f(unsigned short b, __nv_bfloat16*) { return __uint_as_float((unsigned)b << 16); }

template <typename F, int N> struct SegLd;
template <int N> struct SegLd<float, N> {
  template <typename Lt>
  static __device__ __forceinline__ void ld(const float* p, Lt (&v)[N]) {
#pragma unroll
    for (int m = 0; m < N / 4; ++m) {
      const float4 f = __ldg((const float4*)p + m);
      v[4 * m] = (Lt)f.x; v[4 * m + 1] = (Lt)f.y; v[4 * m + 2] = (Lt)f.z; v[4 * m + 3] = (Lt)f.w;
    }
  }
};
template <int N> struct SegLd<double, N> {
  template <typename Lt>
  static __device__ __forceinline__ void ld(const double* p, Lt (&v)[N]) {
#pragma unroll
    for (int m = 0; m < N / 2; ++m) {
      const double2 f = __ldg((const double2*)p + m);
      v[2 * m] = (Lt)f.x; v[2 * m + 1] = (Lt)f.y;
    }
  }
};
// 16-bit formats: each 32-bit word holds two values, the lower address in
// the low half
template <typename H, int N> struct SegLdH {
  template <typename Lt>
  static __device__ __forceinline__ void ld(const H* p, Lt (&v)[N]) {
    unsigned w[N / 2];
    if (N >= 8) {
#pragma unroll
      for (int m = 0; m < N / 8; ++m) {
        const uint4 u = __ldg((const uint4*)p + m);
        w[4 * m] = u.x; w[4 * m + 1] = u.y; w[4 * m + 2] = u.z; w[4 * m + 3] = u.w;
      }
    } else {
      const uint2 u = __ldg((const uint2*)p);
      w[0] = u.x; w[1] = u.y;
    }
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      v[2 * k] = (Lt)h16_to_f((unsigned short)(w[k] & 0xffffu), (H*)nullptr);
      v[2 * k + 1] = (Lt)h16_to_f((unsigned short)(w[k] >> 16), (H*)nullptr);
    }
  }
};
template <int N> struct SegLd<__half, N> : SegLdH<__half, N> {};
template <int N> struct SegLd<__nv_bfloat16, N> : SegLdH<__nv_bfloat16, N> {};

// N consecutive factor values of one row, widened; zero outside the matrix.
template <typename F, typename Lt, int N>
__device__ __forceinline__ void load_seg(const F* LU, int ldf, int n, int row, int col, Lt (&v)[N]) {
  if (row < n && col + N <= n) {
    SegLd<F, N>::ld(LU + (size_t)row * ldf + col, v);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k)
      v[k] = (row < n && col + k < n) ? (Lt)to_f(LU[(size_t)row * ldf + col + k]) : (Lt)0;
  }
}

// Accumulator policies.  V: value type of the solve; A: running sum of
// products (fin() turns it into a V); L: factor element after widening;
// I: inverse element; kW: 32-bit payload words per value.  wsub(w, acc) is
// T(w - sum), the block's result before it is rounded to its storage format.
// Vectors live in double arrays (fp32 solves store floats in them, so that
// they never touch the scarce fp64 pipe; dd solves use a high and a low
// array).
// fp32 sums are compensated (ff_t, Dot2): their result is the accurately
// rounded fp32 value of the sum, which is the model of an fp32 sum that the
// solves follow (an accurate sum rounded once to the arithmetic precision),
// at a few fp32 instructions per term instead of fp64 work.
struct AccF {
  using V = float;
  using A = ff_t;
  using L = float;
  using I = float;
  static constexpr int kW = 1;
  static __device__ __forceinline__ V zero() { return 0.0f; }
  static __device__ __forceinline__ V load(const double* hi, const double*, int i) {
    return __ldcg((const float*)hi + i);
  }
  static __device__ __forceinline__ void save(double* hi, double*, int i, V v) { ((float*)hi)[i] = v; }
  static __device__ __forceinline__ void put(double* hi, double*, int i, double h, double) {
    ((float*)hi)[i] = (float)h;
  }
  static __device__ __forceinline__ double get(const double* hi, const double*, int i) {
    return (double)((const float*)hi)[i];
  }
  static __device__ __forceinline__ A azero() { return ff_t{0.0f, 0.0f}; }
  static __device__ __forceinline__ A merge(A a, A b) { return ff_merge(a, b); }
  static __device__ __forceinline__ A ax(A a, int m) { return ff_shfl_xor(a, m); }
  static __device__ __forceinline__ A fma(L l, V y, A acc) { return ff_fma(l, y, acc); }
  static __device__ __forceinline__ A ifma(I x, V z, A acc) { return ff_fma(x, z, acc); }
  static __device__ __forceinline__ V fin(A acc) { return ff_fin(acc); }
  static __device__ __forceinline__ V wsub(V w, A acc) { return ff_sub_from(w, acc); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ V store(V v, int fmt) { return round_f(v, fmt); }
  static __device__ __forceinline__ V sx(V v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  static __device__ __forceinline__ I inv(const RefineArgs& a, size_t o) { return __ldg(a.inv32 + o); }
  // 16 consecutive scaled-block values of one row (zero outside the matrix)
  using Tm = float;
  template <int N>
  static __device__ __forceinline__ void tile(const RefineArgs& a, int n, int row, int col, Tm (&v)[N]) {
    load_seg<float, float, N>(a.M32, a.ldf, n, row, col, v);
  }
  static __device__ __forceinline__ const Tm* mat(const RefineArgs& a) { return a.M32; }
  static __device__ __forceinline__ A tfma(Tm m, V y, A acc) { return ff_fma(m, y, acc); }
  static __device__ __forceinline__ unsigned word(V v, int) { return __float_as_uint(v); }
  static __device__ __forceinline__ V unword(const unsigned* w) { return __uint_as_float(w[0]); }
};
struct AccD {
  using V = double;
  using A = double;
  using L = double;
  using I = double;
  static constexpr int kW = 2;
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V load(const double* hi, const double*, int i) { return __ldcg(hi + i); }
  static __device__ __forceinline__ void save(double* hi, double*, int i, V v) { hi[i] = v; }
  static __device__ __forceinline__ void put(double* hi, double*, int i, double h, double) { hi[i] = h; }
  static __device__ __forceinline__ double get(const double* hi, const double*, int i) { return hi[i]; }
  static __device__ __forceinline__ A azero() { return 0.0; }
  static __device__ __forceinline__ A merge(A a, A b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ A ax(A a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
  static __device__ __forceinline__ A fma(L l, V y, A acc) { return __fma_rn(l, y, acc); }
  static __device__ __forceinline__ A ifma(I x, V z, A acc) { return __fma_rn(x, z, acc); }
  static __device__ __forceinline__ V fin(A acc) { return acc; }
  static __device__ __forceinline__ V wsub(V w, A acc) { return __dsub_rn(w, acc); }
  static __device__ __forceinline__ V add(V a, V b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ V store(V v, int) { return v; }
  static __device__ __forceinline__ V sx(V v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  static __device__ __forceinline__ I inv(const RefineArgs& a, size_t o) { return __ldg(a.inv_hi + o); }
  using Tm = double;
  template <int N>
  static __device__ __forceinline__ void tile(const RefineArgs& a, int n, int row, int col, Tm (&v)[N]) {
    load_seg<double, double, N>(a.M64, a.ldf, n, row, col, v);
  }
  static __device__ __forceinline__ const Tm* mat(const RefineArgs& a) { return a.M64; }
  static __device__ __forceinline__ A tfma(Tm m, V y, A acc) { return __fma_rn(m, y, acc); }
  static __device__ __forceinline__ unsigned word(V v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return k == 0 ? (unsigned)b : (unsigned)(b >> 32);
  }
  static __device__ __forceinline__ V unword(const unsigned* w) {
    return __longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0]));
  }
};
// Double-double sums of products are accumulated with compensation: each
// product is split exactly (TwoProduct) and its low-order parts kept apart,
// the running high word is updated by TwoSum and the rounding errors are
// summed in a second word (the scheme of Ogita, Rump and Oishi's Dot2,
// extended by the low words of the dd operands).  About 11 fp64 operations
// per term instead of 26 for a dd multiply and an accurate dd add, with an
// error of order n u^2 times the sum of |terms|, as for sums in dd.
struct DDAcc {
  double s, c;
};
struct AccDD {
  using V = dd_t;
  using A = DDAcc;
  using L = double;
  using I = dd_t;
  static constexpr int kW = 4;
  static __device__ __forceinline__ V zero() { return dd_t{0.0, 0.0}; }
  static __device__ __forceinline__ V load(const double* hi, const double* lo, int i) {
    return dd_t{__ldcg(hi + i), __ldcg(lo + i)};
  }
  static __device__ __forceinline__ void save(double* hi, double* lo, int i, V v) { hi[i] = v.hi; lo[i] = v.lo; }
  static __device__ __forceinline__ void put(double* hi, double* lo, int i, double h, double l) {
    hi[i] = h;
    lo[i] = l;
  }
  static __device__ __forceinline__ double get(const double* hi, const double* lo, int i) {
    return __dadd_rn(hi[i], lo[i]);
  }
  static __device__ __forceinline__ A azero() { return DDAcc{0.0, 0.0}; }
  // two partial sums: TwoSum of the running words, errors added (exact
  // error-free step, so every lane of a butterfly gets the same result)
  static __device__ __forceinline__ A merge(A a, A b) {
    const dd_t t = two_sum(a.s, b.s);
    return DDAcc{t.hi, __dadd_rn(__dadd_rn(a.c, b.c), t.lo)};
  }
  static __device__ __forceinline__ A ax(A a, int m) {
    return DDAcc{__shfl_xor_sync(0xffffffffu, a.s, m), __shfl_xor_sync(0xffffffffu, a.c, m)};
  }
  static __device__ __forceinline__ A fma(L l, V y, A acc) {
    const dd_t p = two_prod(l, y.hi);
    const double pl = __fma_rn(l, y.lo, p.lo);
    const dd_t t = two_sum_ord(acc.s, p.hi);
    return DDAcc{t.hi, __dadd_rn(acc.c, __dadd_rn(t.lo, pl))};
  }
  static __device__ __forceinline__ A ifma(I x, V z, A acc) {
    const dd_t p = two_prod(x.hi, z.hi);
    const double pl = __fma_rn(x.hi, z.lo, __fma_rn(x.lo, z.hi, p.lo));
    const dd_t t = two_sum_ord(acc.s, p.hi);
    return DDAcc{t.hi, __dadd_rn(acc.c, __dadd_rn(t.lo, pl))};
  }
  static __device__ __forceinline__ V fin(A acc) { return two_sum(acc.s, acc.c); }
  static __device__ __forceinline__ V wsub(V w, A acc) { return dd_sub(w, fin(acc)); }
  static __device__ __forceinline__ V add(V a, V b) { return dd_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return dd_sub(a, b); }
  static __device__ __forceinline__ V store(V v, int) { return v; }
  static __device__ __forceinline__ V sx(V v, int m) { return dd_shfl_xor(v, m); }
  static __device__ __forceinline__ I inv(const RefineArgs& a, size_t o) {
    return dd_t{__ldg(a.inv_hi + o), __ldg(a.inv_lo + o)};
  }
  using Tm = dd_t;
  template <int N>
  static __device__ __forceinline__ void tile(const RefineArgs& a, int n, int row, int col, Tm (&v)[N]) {
    double h[N], l[N];
    load_seg<double, double, N>(a.Mdh, a.ldf, n, row, col, h);
    load_seg<double, double, N>(a.Mdl, a.ldf, n, row, col, l);
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = dd_t{h[k], l[k]};
  }
  static __device__ __forceinline__ A tfma(Tm m, V y, A acc) { return ifma(m, y, acc); }
  static __device__ __forceinline__ unsigned word(V v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(k < 2 ? v.hi : v.lo);
    return (k & 1) ? (unsigned)(b >> 32) : (unsigned)b;
  }
  static __device__ __forceinline__ V unword(const unsigned* w) {
    return dd_t{__longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0])),
                __longlong_as_double((long long)(((unsigned long long)w[3] << 32) | w[2]))};
  }
};

static_assert(kRefThreads == 4 * kBlk, "substitution thread layout");

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Distributed shared memory: the address of `p` (this CTA's shared memory)
// in cluster peer `rank`, a relaxed store there, and a relaxed load of this
// CTA's own copy that observes such stores.
__device__ __forceinline__ unsigned peer_addr(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_peer_u64(unsigned addr, unsigned long long v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_inbox_u64(const unsigned long long* p) {
  unsigned long long v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return v;
}
// Cluster-wide barrier of all threads (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Tag of an inbox word: the solve's epoch and the block's round (block /
// number of teams), bit 31 clear so that it never equals the all-ones fill
// of a fresh inbox.
__device__ __forceinline__ unsigned inbox_tag(unsigned epoch, int round) {
  return ((epoch << 8) | ((unsigned)round & 0xffu)) & 0x7fffffffu;
}

// Payload words of one block held by one lane: values lane and lane + 32.
template <int W>
struct LLRaw {
  unsigned long long w[2][W];
};

template <int W>
__device__ __forceinline__ void ll_issue(const unsigned long long* blk, int lane, LLRaw<W>& r) {
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int k = 0; k < W; ++k) r.w[m][k] = ld_relaxed_u64(blk + (size_t)(lane + 32 * m) * W + k);
}

template <int W>
__device__ __forceinline__ bool ll_ready(const LLRaw<W>& r, unsigned epoch) {
  bool ok = true;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int k = 0; k < W; ++k) ok &= (unsigned)(r.w[m][k] >> 32) == epoch;
  return __all_sync(0xffffffffu, ok);
}

// Complete the payload of block `blk` whose loads were issued into r: poll
// until every word carries `epoch`, then stage the 64 values for the warp.
// Bounded like every device wait (MSIR_ERR_TIMEOUT, or another block's
// error).
template <typename ACC>
__device__ __forceinline__ bool ll_complete(const unsigned long long* blk, unsigned epoch, int lane,
                                            LLRaw<ACC::kW>& r, typename ACC::V* stage, int* err,
                                            int where) {
  constexpr int W = ACC::kW;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (!ll_ready<W>(r, epoch)) {
    if ((++spins & 255u) == 0u) {
      int bad = 0;
      if (lane == 0) {
        if (t0 == 0) t0 = gtimer();
        if (ld_volatile_i32(err) != 0) bad = 1;
        else if (gtimer() - t0 > kWaitTimeoutNs) bad = 2;
      }
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad == 2) {
        // diagnostics: the first word still missing and the epoch it holds
        int idx = -1;
        unsigned tag = 0;
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
          for (int k = 0; k < W; ++k)
            if (idx < 0 && (unsigned)(r.w[m][k] >> 32) != epoch) {
              idx = (lane + 32 * m) * W + k;
              tag = (unsigned)(r.w[m][k] >> 32);
            }
        const unsigned mk = __ballot_sync(0xffffffffu, idx >= 0);
        const int src = mk ? __ffs(mk) - 1 : 0;
        idx = __shfl_sync(0xffffffffu, idx, src);
        tag = __shfl_sync(0xffffffffu, tag, src);
        if (lane == 0) record_timeout(err, 2, where, (int)epoch, (idx << 20) | (int)(tag & 0xfffffu));
      }
      if (bad) return false;
    }
    ll_issue<W>(blk, lane, r);
  }
  __syncwarp();  // the previous block's staged values have been consumed
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    unsigned p[W];
#pragma unroll
    for (int k = 0; k < W; ++k) p[k] = (unsigned)r.w[m][k];
    stage[lane + 32 * m] = ACC::unword(p);
  }
  __syncwarp();
  return true;
}

// ll_complete for a block that a cluster peer writes into this CTA's inbox
// slot: poll shared memory (no L2 round trip) until every word carries
// `tag`, then stage the values.  Bounded like every device wait.
template <typename ACC>
__device__ __forceinline__ bool ib_complete(const unsigned long long* slot, unsigned tag, int lane,
                                            typename ACC::V* stage, int* err, int where) {
  constexpr int W = ACC::kW;
  LLRaw<W> r;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (true) {
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int k = 0; k < W; ++k) r.w[m][k] = ld_inbox_u64(slot + (size_t)(lane + 32 * m) * W + k);
    if (ll_ready<W>(r, tag)) break;
    if ((++spins & 1023u) == 0u) {
      int bad = 0;
      if (lane == 0) {
        if (t0 == 0) t0 = gtimer();
        if (ld_volatile_i32(err) != 0) bad = 1;
        else if (gtimer() - t0 > kWaitTimeoutNs) bad = 2;
      }
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad == 2 && lane == 0) record_timeout(err, 2, where, (int)tag, -1);
      if (bad) return false;
    }
  }
  __syncwarp();  // the previous block's staged values have been consumed
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    unsigned p[W];
#pragma unroll
    for (int k = 0; k < W; ++k) p[k] = (unsigned)r.w[m][k];
    stage[lane + 32 * m] = ACC::unword(p);
  }
  __syncwarp();
  return true;
}

// The factor storage type F of the refinement code is a template parameter
// of the single-system kernels (one instantiation per u_f); FAny stands for
// "the format in RefineArgs::f_fmt", read at run time, so that the batched
// engine, whose systems change u_f as they escalate, needs one
// instantiation.  Only the scaled-block construction reads the factors.
struct FAny {};
template <typename F>
__device__ __forceinline__ int factor_fmt(const RefineArgs&) {
  return Fmt<F>::code;
}
template <>
__device__ __forceinline__ int factor_fmt<FAny>(const RefineArgs& a) {
  return a.f_fmt;
}
template <typename F>
__device__ __forceinline__ double factor_at(const RefineArgs& a, size_t i) {
  return (double)to_f(((const F*)a.LU)[i]);
}
template <>
__device__ __forceinline__ double factor_at<FAny>(const RefineArgs& a, size_t i) {
  switch (a.f_fmt) {
    case MSIR_FP16: return (double)to_f(((const __half*)a.LU)[i]);
    case MSIR_BF16: return (double)to_f(((const __nv_bfloat16*)a.LU)[i]);
    case MSIR_FP32: return (double)((const float*)a.LU)[i];
    default: return ((const double*)a.LU)[i];
  }
}

// Scaled off-diagonal blocks M_bj = D_b^{-1} F_bj (j != b; L below the
// diagonal blocks, U above), formed by all CTAs of the grid once per
// factorisation and precision, the first time a solve needs them.  One
// 64x64 tile per step: the inverse of the diagonal block and the factor
// block are staged in shared memory (half the inner dimension at a time);
// thread (i, g) forms row i, columns
// 16g .. 16g+15 of the product, 64 terms each.  fp32/fp64: fp64 inverse,
// fp64 sums, stored as fp64 and rounded to fp32.  dd: dd inverse, sums
// compensated as in the substitutions (Dot2 with the inverse's low word).
template <typename F>
__device__ __noinline__ bool build_scaled(Cx& cx, const RefineArgs& a, bool dd) {
  // staging of half the inner dimension at a time: inverse columns k0..k0+31
  // (high, low words) and factor rows k0..k0+31; the sums keep k order
  constexpr int KH = kBlk / 2;
  double* Xh = (double*)cx.ssm;       // 64 x (KH + 1)
  double* Xl = Xh + kBlk * (KH + 1);  // 64 x (KH + 1)
  double* Fb = Xl + kBlk * (KH + 1);  // KH x kScLd
  const int n = cx.n, nb = cx.nblk, ld = a.ldf;
  const int i = cx.tid >> 2, cg = cx.tid & 3;
  for (int t = cx.cta; t < nb * nb; t += cx.G) {
    const int b = t / nb, j = t % nb;
    if (b == j) continue;
    const bool lower = j < b;
    const size_t ib = ((size_t)(lower ? 0 : 1) * nb + b) * kBlk * kBlk;
    const int r0 = b * kBlk, c0 = j * kBlk;
    const int row = r0 + i;
    double sh[16], sc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) sh[q] = sc[q] = 0.0;
    for (int k0 = 0; k0 < kBlk; k0 += KH) {
      __syncthreads();  // the previous staging is no longer read
      for (int e = cx.tid; e < kBlk * KH; e += kRefThreads) {
        const int rr = e / KH, kk = e % KH;
        Xh[rr * (KH + 1) + kk] = __ldg(a.inv_hi + ib + (size_t)rr * kBlk + k0 + kk);
        if (dd) Xl[rr * (KH + 1) + kk] = __ldg(a.inv_lo + ib + (size_t)rr * kBlk + k0 + kk);
      }
      for (int e = cx.tid; e < KH * kBlk; e += kRefThreads) {
        const int kk = e / kBlk, cc = e % kBlk;
        const int frow = r0 + k0 + kk, col = c0 + cc;
        Fb[kk * kScLd + cc] = (frow < n && col < n) ? factor_at<F>(a, (size_t)frow * ld + col) : 0.0;
      }
      __syncthreads();
      if (!dd) {
        for (int kk = 0; kk < KH; ++kk) {
          const double x = Xh[i * (KH + 1) + kk];
#pragma unroll
          for (int q = 0; q < 16; ++q) sh[q] = __fma_rn(x, Fb[kk * kScLd + cg * 16 + q], sh[q]);
        }
      } else {
        for (int kk = 0; kk < KH; ++kk) {
          const double xh = Xh[i * (KH + 1) + kk], xl = Xl[i * (KH + 1) + kk];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const double f = Fb[kk * kScLd + cg * 16 + q];
            const dd_t p = two_prod(xh, f);
            const double pl = __fma_rn(xl, f, p.lo);
            const dd_t u = two_sum_ord(sh[q], p.hi);
            sh[q] = u.hi;
            sc[q] = __dadd_rn(sc[q], __dadd_rn(u.lo, pl));
          }
        }
      }
    }
    if (row < n) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int col = c0 + cg * 16 + q;
        if (col >= n) continue;
        if (!dd) {
          a.M64[(size_t)row * ld + col] = sh[q];
          a.M32[(size_t)row * ld + col] = __double2float_rn(sh[q]);
        } else {
          const dd_t v = two_sum(sh[q], sc[q]);
          a.Mdh[(size_t)row * ld + col] = v.hi;
          a.Mdl[(size_t)row * ld + col] = v.lo;
        }
      }
    }
  }
  return grid_barrier(a.bar, a.err, cx.G);
}

// 16-byte asynchronous copy global -> shared (L2 only) with zero fill past
// `bytes` (0..16); groups of them are committed and waited for per thread.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Depth of the ring of scaled-block tiles that fp32 / fp64 substitutions
// stream through shared memory (the scaled-block staging area, idle during
// the solves); a member's tile is R x 64 values.
constexpr int kTileRing = 3;

// One triangular solve (LOWER: L y = c, unit diagonal; else U z = y) over
// all blocks of this CTA's team, with the block rows scaled beforehand:
// y_b = w_b - sum_j M_bj y_j, w_b = inv(D_b) c_b (the backward solve the
// same with U).
//
// Teams: K CTAs (K in {1, 2, 4, 8}) share each 64-row block, member m
// taking rows m*64/K .. (m+1)*64/K - 1; teams own blocks t, t + T, t + 2T,
// ... (T = floor(G / K) teams; CTAs beyond K*T idle).  Each row is handled
// by TPR adjacent threads with 64/TPR columns of every tile each (TPR = 4,
// or 8 and 16 for K = 4 and 8 so that at least 4 warps work); the other
// warps only take part in the barriers.  Members need no exchange: each has all it
// needs for its rows (w from all of c_b, the tiles' rows, the published y).
// w_b is formed before the block's dependencies arrive, so the dependency
// chain carries one tile product and a 4-lane sum per block.  The backward
// solve takes y_b from the forward solve's published words (epoch - 1),
// because its rows may have been solved by other members.
//
// Not inlined: its register-heavy loop then does not raise the pressure of
// the rest of the kernel (the call costs a few register saves per solve).
template <typename F, typename ACC, bool LOWER, int K>
__device__ __noinline__ bool trsv_team(Cx& cx, const RefineArgs& a, int store_fmt, unsigned epoch) {
  using V = typename ACC::V;
  using I = typename ACC::I;
  using Tm = typename ACC::Tm;
  constexpr int W = ACC::kW;
  constexpr int R = kBlk / K;               // rows per member
  // threads per row: 4, or more so that a member keeps at least 4 warps
  // busy (one per SM sub-partition; each has its own fp64 unit)
  constexpr int TPR = R * 4 >= 128 ? 4 : 128 / R;
  constexpr int NC = kBlk / TPR;            // columns per thread and tile
  constexpr int NACT = R * TPR;             // working threads (whole warps)
  static_assert(NACT % 32 == 0 && NACT <= kRefThreads && NC >= 4, "team shape");
  V* s_stage = (V*)cx.tsm;                  // per warp: 64 staged values
  const int n = cx.n;
  const bool act = cx.tid < NACT;
  const int r = act ? cx.tid / TPR : 0, seg = cx.tid % TPR;
  V* stage = s_stage + cx.warp * kBlk;
  const int tri = LOWER ? 0 : 1;
  const double* in_hi = a.c_hi;  // forward solve input (backward: published y)
  const double* in_lo = a.c_lo;
  double* out_hi = LOWER ? a.y_hi : a.z_hi;
  double* out_lo = LOWER ? a.y_lo : a.z_lo;
  // hand-off words: [direction][block][64][W] (direction 0 forward, 1 backward)
  const size_t llblk = (size_t)kBlk * kLLWords;
  unsigned long long* ll_y = a.ll + (size_t)tri * cx.nblk * llblk;
  const unsigned long long* ll_fwd = a.ll;
  const int T = cx.G / K;
  const int team = cx.cta / K, member = cx.cta % K;
  const int nmine = team < T && team < cx.nblk ? (cx.nblk - 1 - team) / T + 1 : 0;
  // Clusters (cx.C > 1, K | C): the C / K teams of a cluster own
  // consecutive blocks of each round, and a team takes the blocks of the
  // teams before it in its cluster (forward; after it, backward) from its
  // inbox, where their owners write them through distributed shared memory,
  // instead of from the L2 hand-off words.  Every block is also published to
  // L2 for the other clusters.
  const bool clus = cx.C > 1 && K <= cx.C;
  const int TPC = clus ? cx.C / K : 1;  // teams per cluster
  const int tpos = team % TPC;          // this team's position in its cluster
  for (int q = 0; q < nmine; ++q) {
    const int b = LOWER ? team + q * T : team + (nmine - 1 - q) * T;
    const int r0 = b * kBlk;
    const int nr = min(kBlk, n - r0);
    const int rr = member * R + r;  // row within the block
    const int row = r0 + rr;
    const unsigned itag = inbox_tag(epoch, b / T);
    // dependencies taken from the inbox: forward b - tpos .. b - 1, backward
    // b + 1 .. b + TPC - 1 - tpos (the same round, this cluster)
    const int ib_lo = LOWER ? b - tpos : b + 1;
    const int ib_hi = LOWER ? b - 1 : b + (TPC - 1 - tpos);
    auto from_inbox = [&](int j) { return clus && j >= ib_lo && j <= ib_hi; };
    auto inbox_slot = [&](int j) {  // the source team's position
      return cx.inbox + (size_t)(tpos + (j - b)) * kBlk * W;
    };
    unsigned long long* ts = a.tsv ? a.tsv + ((LOWER ? 0 : 1) * (size_t)cx.nblk + b) * 4 : nullptr;
    if (ts && cx.tid == 0 && member == 0) ts[0] = gtimer();
    bool ok = true;  // a failed wait ends the warp's work; the CTA leaves together below
    // w_r = (row rr of inv(D_b)) c_b
    typename ACC::A wa = ACC::azero();
    if (act) {
      const V* cs;
      if (LOWER) {
        V cv[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const int kk = seg * NC + k;
          cv[k] = kk < nr ? ACC::load(in_hi, in_lo, r0 + kk) : ACC::zero();
        }
        const size_t inv_row = (((size_t)tri * cx.nblk + b) * kBlk + rr) * kBlk + seg * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) wa = ACC::ifma(ACC::inv(a, inv_row + k), cv[k], wa);
      } else {
        LLRaw<W> py;
        ll_issue<W>(ll_fwd + (size_t)b * llblk, cx.lane, py);
        ok = ll_complete<ACC>(ll_fwd + (size_t)b * llblk, epoch - 1, cx.lane, py, stage, a.err,
                              (tri << 24) | (1 << 23) | (b << 12) | b);
        cs = stage + seg * NC;
        const size_t inv_row = (((size_t)tri * cx.nblk + b) * kBlk + rr) * kBlk + seg * NC;
        if (ok) {
#pragma unroll
          for (int k = 0; k < NC; ++k) wa = ACC::ifma(ACC::inv(a, inv_row + k), cs[k], wa);
        }
      }
#pragma unroll
      for (int m = 1; m < TPR; m <<= 1) wa = ACC::merge(wa, ACC::ax(wa, m));
    }
    const V wr = ACC::fin(wa);
    // dependencies in the order they become available
    const int ndep = LOWER ? b : cx.nblk - 1 - b;
    // two interleaved partial sums (even and odd columns), merged at the
    // end: the tile product on the dependency chain is half as deep
    typename ACC::A acc = ACC::azero(), acc2 = ACC::azero();
    // fp32/fp64 tiles of at most a sixth of the staging area stream through a
    // ring in shared memory; wider ones (fp64 without teams) and dd tiles
    // are loaded into registers
    constexpr bool kRing = W <= 2 && (size_t)R * kBlk * sizeof(Tm) * kTileRing <= (size_t)kScaledSmem;
    if (ok && ndep > 0 && act) {
      if constexpr (kRing) {
        // fp32/fp64: the tiles stream through a ring in shared memory,
        // kTileRing - 1 dependencies ahead (asynchronous copies; each thread
        // copies and later reads only its own chunks, so no barrier), and the
        // hand-off words are loaded one dependency ahead
        constexpr int EPC = 16 / (int)sizeof(Tm);  // values per 16-byte chunk
        constexpr int NCH = NC / EPC;              // chunks per thread and tile
        Tm* ring = (Tm*)cx.ssm;                    // [kTileRing][NCH][NACT][EPC]
        const Tm* Mat = ACC::mat(a);
        auto issue = [&](int t) {
          if (t < ndep) {
            const int jt = LOWER ? t : cx.nblk - 1 - t;
            Tm* slot = ring + (size_t)(t % kTileRing) * NCH * NACT * EPC;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
              const int col = jt * kBlk + seg * NC + c * EPC;
              const int valid = row < n ? max(0, min(EPC, n - col)) : 0;
              const Tm* src = Mat + (valid > 0 ? (size_t)row * a.ldf + col : 0);
              cp_async16(slot + ((size_t)c * NACT + cx.tid) * EPC, src, valid * (int)sizeof(Tm));
            }
          }
          cp_async_commit();
        };
#pragma unroll
        for (int t = 0; t < kTileRing - 1; ++t) issue(t);
        LLRaw<W> pc, pn;
        int jb = LOWER ? 0 : cx.nblk - 1;
        if (!from_inbox(jb)) ll_issue<W>(ll_y + (size_t)jb * llblk, cx.lane, pc);
        for (int t = 0; t < ndep; ++t) {
          const int jn = LOWER ? jb + 1 : jb - 1;
          const bool more = t + 1 < ndep;
          issue(t + kTileRing - 1);
          if (more && !from_inbox(jn)) ll_issue<W>(ll_y + (size_t)jn * llblk, cx.lane, pn);
          cp_async_wait<kTileRing - 1>();  // this thread's copies of tile t are done
          Tm tc[NC];
          const Tm* slot = ring + (size_t)(t % kTileRing) * NCH * NACT * EPC;
#pragma unroll
          for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int e = 0; e < EPC; ++e) tc[c * EPC + e] = slot[((size_t)c * NACT + cx.tid) * EPC + e];
          const int where = (tri << 24) | (b << 12) | jb;
          if (!(from_inbox(jb) ? ib_complete<ACC>(inbox_slot(jb), itag, cx.lane, stage, a.err, where | (1 << 22))
                               : ll_complete<ACC>(ll_y + (size_t)jb * llblk, epoch, cx.lane, pc, stage, a.err, where))) {
            ok = false;
            break;
          }
          if (ts && !more && cx.tid == 0 && member == 0) ts[3] = gtimer();
          const V* ys = stage + seg * NC;
#pragma unroll
          for (int k = 0; k < NC; k += 2) {
            acc = ACC::tfma(tc[k], ys[k], acc);
            acc2 = ACC::tfma(tc[k + 1], ys[k + 1], acc2);
          }
          if (!more) break;
          pc = pn;
          jb = jn;
        }
        cp_async_wait<0>();  // no copy outlives the solve (the ring is reused)
      } else {
        // fp64 without teams: tile and payload loads one dependency ahead
        // (double buffer); dd: the next tile is loaded after the current
        // one is used (its products, not the loads, bound the dd solve)
        constexpr bool kDouble = W <= 2;
        Tm tc[NC], tn[kDouble ? NC : 1];
        LLRaw<W> pc, pn;
        int jb = LOWER ? 0 : cx.nblk - 1;
        ACC::template tile<NC>(a, n, row, jb * kBlk + seg * NC, tc);
        if (!from_inbox(jb)) ll_issue<W>(ll_y + (size_t)jb * llblk, cx.lane, pc);
        for (int t = 0; t < ndep; ++t) {
          const int jn = LOWER ? jb + 1 : jb - 1;
          const bool more = t + 1 < ndep;
          if (kDouble && more) {
            ACC::template tile<NC>(a, n, row, jn * kBlk + seg * NC, *(Tm(*)[NC])tn);
            if (!from_inbox(jn)) ll_issue<W>(ll_y + (size_t)jn * llblk, cx.lane, pn);
          }
          const int where = (tri << 24) | (b << 12) | jb;
          if (!(from_inbox(jb) ? ib_complete<ACC>(inbox_slot(jb), itag, cx.lane, stage, a.err, where | (1 << 22))
                               : ll_complete<ACC>(ll_y + (size_t)jb * llblk, epoch, cx.lane, pc, stage, a.err, where))) {
            ok = false;
            break;
          }
          if (ts && !more && cx.tid == 0 && member == 0) ts[3] = gtimer();
          const V* ys = stage + seg * NC;
#pragma unroll
          for (int k = 0; k < NC; k += 2) {
            acc = ACC::tfma(tc[k], ys[k], acc);
            acc2 = ACC::tfma(tc[k + 1], ys[k + 1], acc2);
          }
          if (!more) break;
          if (kDouble) {
#pragma unroll
            for (int k = 0; k < NC; ++k) tc[k] = tn[kDouble ? k : 0];
            pc = pn;
          } else {
            ACC::template tile<NC>(a, n, row, jn * kBlk + seg * NC, tc);
            if (!from_inbox(jn)) ll_issue<W>(ll_y + (size_t)jn * llblk, cx.lane, pc);
          }
          jb = jn;
        }
      }
    }
    acc = ACC::merge(acc, acc2);
    if (ts && cx.tid == 0 && member == 0) ts[1] = gtimer();
    if (act && ok) {
      // the TPR segments of the row: s_r, then y_r = S(T(w_r - s_r))
#pragma unroll
      for (int m = 1; m < TPR; m <<= 1) acc = ACC::merge(acc, ACC::ax(acc, m));
      V y = ACC::store(ACC::wsub(wr, acc), store_fmt);
      if (rr >= nr) y = ACC::zero();
      // publish: segment k writes payload word k of the row (rows past n as 0)
      if (seg < W)
        st_relaxed_u64(ll_y + (size_t)b * llblk + (size_t)rr * W + seg,
                       ((unsigned long long)epoch << 32) | ACC::word(y, seg));
      if (clus) {
        // and into the inboxes of the cluster's teams that take this block
        // next (their K members each): word k of the row for target CTA c,
        // spread over the row's TPR threads
        const int nteams = LOWER ? min(TPC - 1 - tpos, cx.nblk - 1 - b) : tpos;
        const unsigned long long* dst = cx.inbox + ((size_t)tpos * kBlk + rr) * W;
        for (int e = seg; e < nteams * K * W; e += TPR) {
          const int ci = e / W, k = e % W;
          const int cpos = LOWER ? tpos + 1 + ci / K : tpos - 1 - ci / K;
          st_peer_u64(peer_addr(dst + k, (unsigned)(cpos * K + ci % K)),
                      ((unsigned long long)itag << 32) | ACC::word(y, k));
        }
      }
      if (seg == 0 && rr < nr) ACC::save(out_hi, out_lo, row, y);
    }
    if (ts && cx.tid == 0 && member == 0) ts[2] = gtimer();
    if (__syncthreads_or(!ok)) return false;  // staged values are reused by the next block
  }
  return true;
}

// Team size of a solve in arithmetic ACC: fp32 solves keep one CTA per
// block (their products are cheap; teams need two grid barriers per
// solve).  fp64 and dd solves split each block's rows over K CTAs, which
// shortens the tile product on the dependency chain K-fold (on GB300's
// narrow fp64 pipe it costs more than the hand-off): K = 8 when each team
// then owns at most two blocks, else 4 when each owns at most four, else 2.
// Measured (one GPU, fp64 solves at n = 8192, dd solves at n = 4096): K = 4
// beats K = 2 by 15-20 %; K = 8, whose teams then own 7 or 4 blocks,
// gains nothing more.
template <typename ACC>
__device__ __forceinline__ int team_size(const Cx& cx) {
  if (ACC::kW == 1) return 1;
  int k;
  if (cx.team_k > 0) {
    k = cx.team_k <= cx.G ? cx.team_k : 1;
  } else {
    const int half = (cx.nblk + 1) / 2, quarter = (cx.nblk + 3) / 4;
    k = cx.G / 8 >= half ? 8 : (cx.G / 4 >= quarter ? 4 : (cx.G >= 2 ? 2 : 1));
  }
  return cx.C > 1 ? min(k, cx.C) : k;  // a team stays inside one cluster
}

template <typename F, typename ACC, bool LOWER>
__device__ __forceinline__ bool trsv(Cx& cx, const RefineArgs& a, int store_fmt) {
  const unsigned epoch = ++cx.epoch;
  const int K = team_size<ACC>(cx);
  if (ACC::kW > 1 && K == 8) return trsv_team<F, ACC, LOWER, 8>(cx, a, store_fmt, epoch);
  if (ACC::kW > 1 && K == 4) return trsv_team<F, ACC, LOWER, 4>(cx, a, store_fmt, epoch);
  if (ACC::kW > 1 && K == 2) return trsv_team<F, ACC, LOWER, 2>(cx, a, store_fmt, epoch);
  return trsv_team<F, ACC, LOWER, 1>(cx, a, store_fmt, epoch);
}

// M^{-1} applied to the right-hand side already placed in c (permuted
// order, scaled by R, rounded to the storage format): forward then backward
// substitution.  Result in z (natural order, before the S*mu scaling).
template <typename F, typename ACC>
__device__ bool msolve(Cx& cx, const RefineArgs& a, int store_fmt) {
  // scaled blocks of the current factors in this precision, once
  const unsigned need = ACC::kW == 4 ? 2u : 1u;
  if (!(cx.mready & need)) {
    if (!build_scaled<F>(cx, a, need == 2u)) return false;
    cx.mready |= need;
  }
  // Rows of block b are prepared (c) and consumed (z) by CTA b mod G.  A
  // team of K > 1 CTAs spreads them over other CTAs, so c must be visible
  // grid-wide before the forward solve and z after the backward solve.
  const bool team = team_size<ACC>(cx) > 1;
  if (team && !grid_barrier(a.bar, a.err, cx.G)) return false;
  {
    PhaseTimer pt(cx, 1);
    if (!trsv<F, ACC, true>(cx, a, store_fmt)) return false;
  }
  PhaseTimer pt(cx, 2);
  if (!trsv<F, ACC, false>(cx, a, store_fmt)) return false;
  return !team || grid_barrier(a.bar, a.err, cx.G);
}

template <typename F>
__device__ bool msolve_arith(Cx& cx, const RefineArgs& a, int arith, int store_fmt) {
  if (arith == MSIR_FP32) return msolve<F, AccF>(cx, a, store_fmt);
  if (arith == MSIR_FP64) return msolve<F, AccD>(cx, a, store_fmt);
  return msolve<F, AccDD>(cx, a, store_fmt);
}

// right-hand side element of a substitution in precision `arith`
__device__ __forceinline__ void put_c(const RefineArgs& a, int arith, int i, double h, double l) {
  if (arith == MSIR_FP32) AccF::put(a.c_hi, a.c_lo, i, h, l);
  else if (arith == MSIR_FP64) AccD::put(a.c_hi, a.c_lo, i, h, l);
  else AccDD::put(a.c_hi, a.c_lo, i, h, l);
}
// solution element (z) of a substitution in precision `arith`, as a double
__device__ __forceinline__ double get_z(const RefineArgs& a, int arith, int i) {
  if (arith == MSIR_FP32) return AccF::get(a.z_hi, a.z_lo, i);
  if (arith == MSIR_FP64) return AccD::get(a.z_hi, a.z_lo, i);
  return AccDD::get(a.z_hi, a.z_lo, i);
}

// iterate over the rows of my blocks
#define FOR_MY_ROWS(cx, i)                                                          \
  for (int _b = (cx).cta; _b < (cx).nblk; _b += (cx).G)                               \
    for (int i = _b * kBlk + (cx).tid; i < min((_b + 1) * kBlk, (cx).n); i += kRefThreads)

// Squeezed factors of B = mu R A S (Sec. 2.1.2's cited scaling): A x = c is
// solved as B y = mu R c, x = S y; mu scales the right-hand side before it
// is rounded to the solve's storage format, which keeps it (and y) inside
// the bf16 / fp16 range when A's entries are far from 1.
static __device__ __forceinline__ double rscale(const RefineArgs& a, int row) {
  return a.Rsc ? a.Rsc[row] * a.mu : 1.0;
}
static __device__ __forceinline__ double cscale(const RefineArgs& a, int col) {
  return a.Ssc ? a.Ssc[col] : 1.0;
}

// ------------------------------------------------------------ residual

// r_p[i] = b[perm[i]] - A[perm[i]] x in ur; rows are spread over every warp
// of the grid (the fp64 work needs all SMs).  Returns (via grid reduction)
// s = ||r||_inf and ||x||_inf, and, with an exact solution given (MSIR_CONV_TRUE),
// ferr = ||x - x_ref||_inf / ||x_ref||_inf.  The caller has made x complete
// (barrier).
template <typename A0>
__device__ __noinline__ bool residual(Cx& cx, const RefineArgs& a, const double* x, int ur, double& s,
                         double& xnorm, double* ferr = nullptr) {
  PhaseTimer pt(cx, 0);
  const A0* A = (const A0*)a.A;
  double mr = 0.0, mx = 0.0;
  const int nw = cx.G * (kRefThreads / 32);
  for (int i = cx.cta * (kRefThreads / 32) + cx.warp; i < cx.n; i += nw) {
    const int ar = a.perm[i];
    const A0* row = A + (size_t)ar * a.lda;
    if (ur == MSIR_DD) {
      const dd_t ax = row_dot_dd<A0>(row, x, cx.n, cx.lane);
      const dd_t r = dd_sub(dd_t{a.b[ar], 0.0}, ax);
      if (cx.lane == 0) { a.r_hi[i] = r.hi; a.r_lo[i] = r.lo; }
      mr = nanmax(mr, fabs(r.hi));
    } else {
      const double ax = row_dot_d<A0>(row, x, cx.n, cx.lane);
      const double r = __dsub_rn(a.b[ar], ax);
      if (cx.lane == 0) { a.r_hi[i] = r; a.r_lo[i] = 0.0; }
      mr = nanmax(mr, fabs(r));
    }
  }
  double mf = 0.0, mref = 0.0;
  for (int i = cx.cta * kRefThreads + cx.tid; i < cx.n; i += cx.G * kRefThreads) {
    const double xi = __ldcg(x + i);
    mx = nanmax(mx, fabs(xi));
    if (a.xref) {
      const double ri = __ldg(a.xref + i);
      mf = nanmax(mf, fabs(__dsub_rn(xi, ri)));
      mref = nanmax(mref, fabs(ri));
    }
  }
  mr = cta_reduce(mr, 1, cx.tid);
  mx = cta_reduce(mx, 1, cx.tid);
  if (a.xref) {
    mf = cta_reduce(mf, 1, cx.tid);
    mref = cta_reduce(mref, 1, cx.tid);
    double v[4] = {mr, mx, mf, mref};
    const int op[4] = {1, 1, 1, 1};
    if (!grid_reduce<4>(cx, a, v, op)) return false;
    s = v[0];
    xnorm = v[1];
    if (ferr) *ferr = v[3] > 0.0 ? v[2] / v[3] : v[2];
    return true;
  }
  double v[2] = {mr, mx};
  const int op[2] = {1, 1};
  if (!grid_reduce<2>(cx, a, v, op)) return false;
  s = v[0];
  xnorm = v[1];
  if (ferr) *ferr = 0.0;
  return true;
}

// fl_u(r_p[i] / s), division in u_r
static __device__ __forceinline__ double scaled_r(const RefineArgs& a, int i, double s, int ur, int u) {
  if (ur == MSIR_DD) {
    const dd_t q = dd_div_d(dd_t{__ldcg(a.r_hi + i), __ldcg(a.r_lo + i)}, s);
    return urnd(q.hi, u);
  }
  return urnd(__ddiv_rn(__ldcg(a.r_hi + i), s), u);
}

// --------------------------------------------------------------- GMRES

struct GmresOut {
  int k;
  bool nonfinite;
};

// Working-precision arithmetic for the GMRES vectors and the Givens /
// least-squares scalars (U = float for u = fp32, double for u = fp64).
template <typename U> struct UA;
template <> struct UA<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float wsum(float v) { return warp_sum_f(v); }
  static __device__ __forceinline__ float rnd(double v) { return __double2float_rn(v); }
};
template <> struct UA<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double wsum(double v) { return warp_sum_d(v); }
  static __device__ __forceinline__ double rnd(double v) { return v; }
};

// Operator t = A v (rows perm[i]) in the operator precision, scaled by R,
// placed in c.  op = FP32: compensated fp32 sums (the accurately rounded
// fp32 value of each row's sum), rows of my blocks (no barrier needed before
// the substitution); FP64 / DD: rows over every warp of the grid, followed
// by a grid barrier.
template <typename A0, typename U>
__device__ __noinline__ bool apply_A(Cx& cx, const RefineArgs& a, const U* v, int op) {
  PhaseTimer pt(cx, 4);
  const A0* A = (const A0*)a.A;
  if (op == MSIR_FP32) {
    // a warp's 8 rows together: v is loaded once per column and the eight
    // rows' loads and sums are independent, so their latencies overlap
    for (int b = cx.cta; b < cx.nblk; b += cx.G) {
      const int i0 = b * kBlk + cx.warp * 8;
      if (i0 >= cx.n) continue;
      const A0* rows[8];
      ff_t acc[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int i = min(i0 + rr, cx.n - 1);  // rows past n repeat the last one, never stored
        rows[rr] = A + (size_t)a.perm[i] * a.lda;
        acc[rr] = ff_t{0.0f, 0.0f};
      }
      // four consecutive columns per lane and step, 16-byte loads
      const int n4 = ((reinterpret_cast<uintptr_t>(v) & 15) == 0) ? (cx.n & ~3) : 0;
      // software pipeline: the next step's 8 rows x 4 columns and v are
      // loaded into registers while this step's compensated sums run
      {
        int j = cx.lane * 4;
        float an[8][4], vn[4];
        if (j < n4) {
          ld4f_vec<U>(v + j, vn);
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) ld4f_row<A0>(rows[rr] + j, an[rr]);
        }
        for (; j < n4; j += 128) {
          float ac[8][4], vc[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) vc[q] = vn[q];
#pragma unroll
          for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) ac[rr][q] = an[rr][q];
          if (j + 128 < n4) {
            ld4f_vec<U>(v + j + 128, vn);
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) ld4f_row<A0>(rows[rr] + j + 128, an[rr]);
          }
#pragma unroll
          for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[rr] = ff_fma(ac[rr][q], vc[q], acc[rr]);
        }
      }
      for (int j = n4 + cx.lane; j < cx.n; j += 32) {
        const float vj = (float)__ldcg(v + j);
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) acc[rr] = ff_fma((float)__ldg(rows[rr] + j), vj, acc[rr]);
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) acc[rr] = ff_merge(acc[rr], ff_shfl_xor(acc[rr], m));
      if (cx.lane < 8 && i0 + cx.lane < cx.n) {
        float mine = ff_fin(acc[0]);
#pragma unroll
        for (int rr = 1; rr < 8; ++rr)
          if (cx.lane == rr) mine = ff_fin(acc[rr]);
        const int ar = a.perm[i0 + cx.lane];
        const float R = (float)rscale(a, ar);
        ((float*)a.c_hi)[i0 + cx.lane] = __fmul_rn(mine, R);
      }
    }
    __syncthreads();
    return true;
  }
  const int nw = cx.G * (kRefThreads / 32);
  if (op == MSIR_DD) {
    for (int i = cx.cta * (kRefThreads / 32) + cx.warp; i < cx.n; i += nw) {
      const int ar = a.perm[i];
      const dd_t tt = row_dot_dd<A0, U>(A + (size_t)ar * a.lda, v, cx.n, cx.lane);
      if (cx.lane == 0) {
        const double R = rscale(a, ar);
        a.c_hi[i] = tt.hi * R;
        a.c_lo[i] = tt.lo * R;
      }
    }
    return grid_barrier(a.bar, a.err, cx.G);
  }
  // fp64: two rows per warp at a time (rows i and i + nw); a missing second
  // row repeats the first and is not stored
  for (int i = cx.cta * (kRefThreads / 32) + cx.warp; i < cx.n; i += 2 * nw) {
    const int i2 = i + nw < cx.n ? i + nw : i;
    const int ar[2] = {a.perm[i], a.perm[i2]};
    const A0* const rows[2] = {A + (size_t)ar[0] * a.lda, A + (size_t)ar[1] * a.lda};
    double acc[2];
    rows_dot_d<A0, U, 2>(rows, v, cx.n, cx.lane, acc);
    if (cx.lane == 0) {
      a.c_hi[i] = acc[0] * rscale(a, ar[0]);
      if (i2 != i) a.c_hi[i2] = acc[1] * rscale(a, ar[1]);
    }
  }
  return grid_barrier(a.bar, a.err, cx.G);
}

// GMRES's vector work (Gram-Schmidt, norms, basis updates) uses a flat
// partition: CTA c owns the contiguous rows [c*chunk, (c+1)*chunk) with
// chunk = ceil(n / G), so every CTA shares it (the substitutions' block
// partition leaves all but n/64 CTAs without rows).  Grid barriers separate
// the phases that hand rows between the two partitions.
__device__ __forceinline__ void flat_rows(const Cx& cx, int& r0, int& r1) {
  const int chunk = (cx.n + cx.G - 1) / cx.G;
  r0 = min(cx.n, cx.cta * chunk);
  r1 = min(cx.n, r0 + chunk);
}

// out_i = fl_u(z_i * S_i * mu), flat rows (after the substitution's rows
// are visible grid-wide)
template <typename U>
__device__ bool finish_solve(Cx& cx, const RefineArgs& a, U* out, int arith) {
  if (!grid_barrier(a.bar, a.err, cx.G)) return false;
  int r0, r1;
  flat_rows(cx, r0, r1);
  for (int i = r0 + cx.tid; i < r1; i += kRefThreads) out[i] = UA<U>::rnd(get_z(a, arith, i) * cscale(a, i));
  __syncthreads();
  return true;
}

// Two-stage grid reduction of the (k+1) Gram-Schmidt partial sums; the
// result (rounded to u) lands in s_h[0..k].
template <typename U>
__device__ bool cgs_reduce(Cx& cx, const RefineArgs& a, int kp1, U* s_h) {
  PhaseTimer pt(cx, 3);
  if (!grid_barrier(a.bar, a.err, cx.G)) return false;
  for (int j = cx.cta * 8 + cx.warp; j < kp1; j += cx.G * 8) {
    double acc = 0.0;
    for (int c = cx.lane; c < cx.G; c += 32) acc = __dadd_rn(acc, __ldcg(a.hred + (size_t)c * (a.kcap + 1) + j));
    acc = warp_sum_d(acc);
    if (cx.lane == 0) a.hvec[j] = (double)UA<U>::rnd(acc);
  }
  if (!grid_barrier(a.bar, a.err, cx.G)) return false;
  for (int j = cx.tid; j < kp1; j += kRefThreads) s_h[j] = (U)__ldcg(a.hvec + j);
  __syncthreads();
  return true;
}

// partial sums p_j = sum over my rows of V_j[i] * w[i], j = 0..k, then
// summed over the CTAs in fp64 and rounded to u (the oracle's reading of
// "inner products in u": an accurate sum rounded once).  u = fp64: fp64
// sums.  u = fp32: compensated fp32 sums (Dot2: every product's and
// addition's rounding error kept in a second word), passed on as the fp64
// value s + c; fp64 arithmetic on fp32 data spends most of its time
// widening operands on GB300's narrow fp64 pipe.
//
// The phase is bound by load latency, not bandwidth: each thread takes
// kVec consecutive basis vectors (one 16-byte load per row; the basis is
// row-major with ldv a multiple of 32) and loads kChunk rows ahead of the
// sums, so a CTA keeps about 50 KB of loads in flight.
template <typename U>
__device__ __noinline__ void cgs_partials(Cx& cx, const RefineArgs& a, const U* V, const U* w, int kp1) {
  PhaseTimer pt(cx, 3);
  constexpr int kVec = 16 / (int)sizeof(U);
  constexpr int kChunk = 12;
  using Vec = typename std::conditional<sizeof(U) == 4, float4, double2>::type;
  int r0, r1;
  flat_rows(cx, r0, r1);
  const int nq = (kp1 + kVec - 1) / kVec;
  for (int jq = cx.tid; jq < nq; jq += kRefThreads) {
    const int j0 = jq * kVec;
    // columns j0 .. j0 + kVec - 1 (those past k are summed and not stored)
    ff_t af[kVec];
    double ad[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) {
      af[e] = ff_t{0.0f, 0.0f};
      ad[e] = 0.0;
    }
    for (int i0 = r0; i0 < r1; i0 += kChunk) {
      U vv[kChunk][kVec], wv[kChunk];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
        const int i = i0 + c;
        if (i < r1) {
          const Vec t = __ldcg((const Vec*)(V + (size_t)i * a.ldv + j0));
          const U* tp = (const U*)&t;
#pragma unroll
          for (int e = 0; e < kVec; ++e) vv[c][e] = tp[e];
          wv[c] = __ldcg(w + i);
        } else {
#pragma unroll
          for (int e = 0; e < kVec; ++e) vv[c][e] = (U)0;
          wv[c] = (U)0;
        }
      }
#pragma unroll
      for (int c = 0; c < kChunk; ++c)
#pragma unroll
        for (int e = 0; e < kVec; ++e) {
          if constexpr (sizeof(U) == 4) af[e] = ff_fma(vv[c][e], wv[c], af[e]);
          else ad[e] = __fma_rn(vv[c][e], wv[c], ad[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < kVec; ++e) {
      if (j0 + e >= kp1) break;
      a.hred[(size_t)cx.cta * (a.kcap + 1) + j0 + e] =
          sizeof(U) == 4 ? __dadd_rn((double)af[e].s, (double)af[e].c) : ad[e];
    }
  }
}

// sum_j V_j[i] c_j for the rows i0 .. i0+kRows-1 (those below r1) by one
// warp: lane l sums the columns 4l .. 4l+3 (fp64: 2l, 2l+1) of every
// 128-column (64) step, in order, with 16-byte loads two steps ahead, then a
// butterfly over the lanes.  The rows' loads and reductions are
// independent, so their latencies overlap.  Lane q < kRows returns row
// i0+q's sum as a compensated pair (u = fp32: Dot2 in fp32, the pair's sum
// is the value; u = fp64: an fp64 sum in .s, .c = 0).
constexpr int kRows = 8;
struct RowSum {
  double s, c;
};
template <typename U>
__device__ __forceinline__ RowSum basis_rows_dot(const RefineArgs& a, const U* V, int i0, int r1, int kp1,
                                                 const U* c, int lane) {
  constexpr int kVec = 16 / (int)sizeof(U);
  constexpr int kStep = 32 * kVec;
  using Vec = typename std::conditional<sizeof(U) == 4, float4, double2>::type;
  ff_t af[kRows];
  double ad[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    af[q] = ff_t{0.0f, 0.0f};
    ad[q] = 0.0;
  }
  const int nr = min(kRows, r1 - i0);
#pragma unroll 2
  for (int j0 = lane * kVec; j0 < kp1; j0 += kStep) {
    U vv[kRows][kVec], cj[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) cj[e] = j0 + e < kp1 ? c[j0 + e] : (U)0;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      if (q < nr) {
        const Vec t = __ldcg((const Vec*)(V + (size_t)(i0 + q) * a.ldv + j0));
        const U* tp = (const U*)&t;
#pragma unroll
        for (int e = 0; e < kVec; ++e) vv[q][e] = j0 + e < kp1 ? tp[e] : (U)0;  // columns past k may hold anything
      } else {
#pragma unroll
        for (int e = 0; e < kVec; ++e) vv[q][e] = (U)0;
      }
    }
#pragma unroll
    for (int q = 0; q < kRows; ++q)
#pragma unroll
      for (int e = 0; e < kVec; ++e) {
        if constexpr (sizeof(U) == 4) af[q] = ff_fma(vv[q][e], cj[e], af[q]);
        else ad[q] = __fma_rn(vv[q][e], cj[e], ad[q]);
      }
  }
  RowSum mine{0.0, 0.0};
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    if constexpr (sizeof(U) == 4) {
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) af[q] = ff_merge(af[q], ff_shfl_xor(af[q], m));
      if (lane == q) mine = RowSum{(double)af[q].s, (double)af[q].c};
    } else {
      const double t = warp_sum_d(ad[q]);
      if (lane == q) mine.s = t;
    }
  }
  return mine;
}

// w_i = fl_u(w_i - sum_j V_j[i] h_j) with the difference taken from the
// accurate sum (fp32: w - (s + c) by ff_sub_from); flat rows, kRows rows
// per warp at a time
template <typename U>
__device__ __noinline__ void cgs_update(Cx& cx, const RefineArgs& a, const U* V, U* w, int kp1, const U* s_h) {
  PhaseTimer pt(cx, 3);
  int r0, r1;
  flat_rows(cx, r0, r1);
  for (int i0 = r0 + cx.warp * kRows; i0 < r1; i0 += (kRefThreads / 32) * kRows) {
    const RowSum acc = basis_rows_dot<U>(a, V, i0, r1, kp1, s_h, cx.lane);
    const int i = i0 + cx.lane;
    if (cx.lane < kRows && i < r1) {
      if constexpr (sizeof(U) == 4)
        w[i] = ff_sub_from(w[i], ff_t{(float)acc.s, (float)acc.c});
      else
        w[i] = UA<U>::rnd(__dsub_rn((double)w[i], acc.s));
    }
  }
  __syncthreads();
}

// d_i = fl_u(sum_j V_j[i] y_j) over the flat rows (the GMRES correction)
template <typename U>
__device__ __noinline__ void basis_combine(Cx& cx, const RefineArgs& a, const U* V, int kdone, const U* y) {
  int f0, f1;
  flat_rows(cx, f0, f1);
  for (int i0 = f0 + cx.warp * kRows; i0 < f1; i0 += (kRefThreads / 32) * kRows) {
    const RowSum acc = basis_rows_dot<U>(a, V, i0, f1, kdone, y, cx.lane);
    const int i = i0 + cx.lane;
    if (cx.lane < kRows && i < f1)
      a.d[i] = sizeof(U) == 4 ? (double)ff_fin(ff_t{(float)acc.s, (float)acc.c}) : (double)UA<U>::rnd(acc.s);
  }
}

template <typename U>
__device__ bool grid_sum_sq(Cx& cx, const RefineArgs& a, const U* w, double& out) {
  double ss = 0.0;
  int r0, r1;
  flat_rows(cx, r0, r1);
  for (int i = r0 + cx.tid; i < r1; i += kRefThreads) {
    const double wv = (double)w[i];
    ss = __fma_rn(wv, wv, ss);
  }
  double v[1] = {cta_reduce(ss, 0, cx.tid)};
  const int opr[1] = {0};
  if (!grid_reduce<1>(cx, a, v, opr)) return false;
  out = v[0];
  return true;
}

template <typename A0, typename F, typename U>
__device__ bool gmres(Cx& cx, const RefineArgs& a, double s, int ur, int u, int op, double tau,
                      unsigned char* gsm, GmresOut& out) {
  using M = UA<U>;
  __shared__ double s_bc[1];
  const int kcap = a.kcap;
  U* sm_cs = (U*)gsm;
  U* sm_sn = sm_cs + kcap + 1;
  U* sm_g = sm_sn + kcap + 1;   // kcap + 2
  U* s_h = sm_g + kcap + 2;     // 2 (kcap + 1)
  U* V = (U*)a.V;
  U* vk = (U*)a.vk;
  U* w = (U*)a.w;
  out.k = 0;
  out.nonfinite = false;
  // w0 = fl_u(M^{-1} r~) with the substitutions in op
  for (int b = cx.cta; b < cx.nblk; b += cx.G)
    for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads)
      put_c(a, op, i, scaled_r(a, i, s, ur, u) * rscale(a, a.perm[i]), 0.0);
  __syncthreads();
  if (!msolve_arith<F>(cx, a, op, op)) return false;
  if (!finish_solve<U>(cx, a, w, op)) return false;
  double ss;
  if (!grid_sum_sq<U>(cx, a, w, ss)) return false;
  const U beta = M::sqrt_(M::rnd(ss));
  if (!isfinite((double)beta)) { out.nonfinite = true; return true; }
  int f0, f1;
  flat_rows(cx, f0, f1);
  if (beta == (U)0) {
    for (int i = f0 + cx.tid; i < f1; i += kRefThreads) a.d[i] = 0.0;
    return grid_barrier(a.bar, a.err, cx.G);  // d is read by the block partition
  }
  for (int i = f0 + cx.tid; i < f1; i += kRefThreads) {
    const U v = M::div(w[i], beta);
    V[(size_t)i * a.ldv] = v;
    vk[i] = v;
  }
  if (cx.tid == 0) sm_g[0] = beta;
  __syncthreads();
  int kdone = 0;
  for (int k = 0; k < kcap; ++k) {
    // full V_k needed by the matrix-vector product
    if (!grid_barrier(a.bar, a.err, cx.G)) return false;
    if (!apply_A<A0, U>(cx, a, vk, op)) return false;
    if (!msolve_arith<F>(cx, a, op, op)) return false;
    if (!finish_solve<U>(cx, a, w, op)) return false;
    // classical Gram-Schmidt, twice
    cgs_partials<U>(cx, a, V, w, k + 1);
    if (!cgs_reduce<U>(cx, a, k + 1, s_h)) return false;
    cgs_update<U>(cx, a, V, w, k + 1, s_h);
    for (int j = cx.tid; j <= k; j += kRefThreads) s_h[kcap + 1 + j] = s_h[j];
    __syncthreads();
    cgs_partials<U>(cx, a, V, w, k + 1);
    if (!cgs_reduce<U>(cx, a, k + 1, s_h)) return false;
    cgs_update<U>(cx, a, V, w, k + 1, s_h);
    for (int j = cx.tid; j <= k; j += kRefThreads) s_h[j] = M::add(s_h[kcap + 1 + j], s_h[j]);
    __syncthreads();
    double ww;
    if (!grid_sum_sq<U>(cx, a, w, ww)) return false;
    const U hk1 = M::sqrt_(M::rnd(ww));
    // Givens rotations (every CTA computes the same numbers)
    unsigned long long tg0 = (cx.cta == 0 && cx.tid == 0) ? gtimer() : 0;
    // the entry carried from one rotation to the next stays in a register
    U carry = (U)0;
    if constexpr (sizeof(U) == 8) {
      // fp64: the four products of a rotation on lanes 0-3 of warp 0 (lane
      // q: cs x0, sn x1, -sn x0, cs x1), then lanes 0 and 2 add their pairs:
      // two fp64 instructions on the chain per rotation instead of six
      if (cx.warp == 0) {
        const int q = cx.lane & 3;
        carry = s_h[0];
        for (int i = 0; i < k; ++i) {
          const U cs = sm_cs[i], sn = sm_sn[i], x1 = s_h[i + 1];
          const U ml = q == 1 ? sn : (q == 2 ? -sn : cs);
          const U p = M::mul(ml, (q & 1) ? x1 : carry);
          const U t = M::add(p, __shfl_down_sync(0xffffffffu, p, 1));
          if (cx.lane == 0) s_h[i] = t;
          carry = __shfl_sync(0xffffffffu, t, 2);
        }
      }
    } else if (cx.tid == 0) {
      // the operands of four rotations are loaded ahead of their use
      carry = s_h[0];
      int i = 0;
      for (; i + 4 <= k; i += 4) {
        U cs[4], sn[4], x1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          cs[q] = sm_cs[i + q];
          sn[q] = sm_sn[i + q];
          x1[q] = s_h[i + q + 1];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const U x0 = carry;
          s_h[i + q] = M::add(M::mul(cs[q], x0), M::mul(sn[q], x1[q]));
          carry = M::add(M::mul(-sn[q], x0), M::mul(cs[q], x1[q]));
        }
      }
      for (; i < k; ++i) {
        const U x0 = carry, x1 = s_h[i + 1];
        s_h[i] = M::add(M::mul(sm_cs[i], x0), M::mul(sm_sn[i], x1));
        carry = M::add(M::mul(-sm_sn[i], x0), M::mul(sm_cs[i], x1));
      }
    }
    if (cx.tid == 0) {
      s_h[k] = carry;
      const U f = s_h[k], g = hk1;
      U c, sn, r;
      if (g == (U)0) {
        c = (U)1; sn = (U)0; r = f;
      } else {
        r = M::sqrt_(M::add(M::mul(f, f), M::mul(g, g)));
        c = M::div(f, r);
        sn = M::div(g, r);
      }
      sm_cs[k] = c;
      sm_sn[k] = sn;
      s_h[k] = r;
      const U gk = sm_g[k];
      sm_g[k] = M::mul(c, gk);
      sm_g[k + 1] = M::mul(-sn, gk);
      s_bc[0] = fabs((double)sm_g[k + 1]) / (double)beta;
    }
    __syncthreads();
    if (cx.cta == 0) {
      double* Hk = a.H + (size_t)k * (kcap + 1);
      for (int i = cx.tid; i <= k; i += kRefThreads) Hk[i] = (double)s_h[i];
    }
    if (cx.cta == 0 && cx.tid == 0) cx.t_ns[6] += gtimer() - tg0;
    const double relres = s_bc[0];
    kdone = k + 1;
    if (hk1 != (U)0 && isfinite((double)hk1)) {
      for (int i = f0 + cx.tid; i < f1; i += kRefThreads) {
        const U v = M::div(w[i], hk1);
        V[(size_t)i * a.ldv + k + 1] = v;
        vk[i] = v;
      }
    }
    __syncthreads();
    if (!isfinite(relres) || relres <= tau || hk1 == (U)0) break;
  }
  // y from the rotated Hessenberg matrix (CTA 0), then d = fl_u(V y)
  if (cx.cta == 0 && cx.tid == 0) {
    for (int i = kdone - 1; i >= 0; --i) {
      U acc = sm_g[i];
      for (int j = i + 1; j < kdone; ++j)
        acc = M::sub(acc, M::mul((U)a.H[(size_t)j * (kcap + 1) + i], (U)a.yv[j]));
      a.yv[i] = (double)M::div(acc, (U)a.H[(size_t)i * (kcap + 1) + i]);
    }
  }
  if (!grid_barrier(a.bar, a.err, cx.G)) return false;
  for (int j = cx.tid; j < kdone; j += kRefThreads) s_h[j] = (U)__ldcg(a.yv + j);
  __syncthreads();
  basis_combine<U>(cx, a, V, kdone, s_h);
  out.k = kdone;
  return grid_barrier(a.bar, a.err, cx.G);  // d is read by the block partition
}

// -------------------------------------------------------------- kernel

// (cta: the block's index in the solve's grid; block 0 writes the report)
static __device__ void rep_new_stage(const RefineArgs& a, RefState& S, int cta) {
  if (cta == 0 && threadIdx.x == 0 && S.nstages < MSIR_MAX_STAGES) {
    msir_stage& g = a.rep->stage[S.nstages];
    g.uf = S.uf;
    g.u = S.u;
    g.ur = S.ur;
    g.alg = S.alg;
    g.steps = 0;
    g.nonfinite = 0;
  }
  S.nstages++;
}

// Algorithm 4's stopping logic after one completed step (mirrors Sec. 2.1.1
// with the readings listed in the library documentation).  Thread 0 only.
// Returns 0 continue, 1 converged, 2 switch (reset = phi > phi_0).
static __device__ int ctl_step(RefState& S, const RefineArgs& a, double s, double dnorm, double xnorm,
                               double nbe, double ferr, int kg, int* reset) {
  const double delta = s * dnorm;
  const double z = xnorm > 0.0 ? delta / xnorm : __longlong_as_double(0x7ff0000000000000ll);
  const double v = isfinite(S.delta_prev) ? delta / S.delta_prev : 0.0;
  S.rho_max = fmax(S.rho_max, v);
  const double phi =
      S.rho_max < 1.0 ? z / (1.0 - S.rho_max) : __longlong_as_double(0x7ff0000000000000ll);
  S.phi = phi;
  if (!S.have_phi0) { S.phi0 = phi; S.have_phi0 = 1; }
  S.delta_prev = delta;
  const double gamma = a.gamma > 0.0 ? a.gamma : sqrt((double)a.n);
  const double uu0 = unit_roundoff(a.u0);
  const double thr = gamma * uu0;
  bool conv = phi >= 0.0 && phi <= thr;
  if (a.conv == MSIR_CONV_COMBINED) conv = conv && nbe <= 2.0 * uu0;
  if (a.conv == MSIR_CONV_TRUE) conv = ferr <= uu0 && nbe <= uu0;
  *reset = 0;
  if (conv) return 1;
  const bool trig = z <= unit_roundoff(S.u) || v >= a.rho_thresh || S.it >= a.i_max ||
                    (S.alg != MSIR_ALG_SIR && kg >= 0 && (double)kg >= a.kmax);
  if (trig) {
    *reset = phi > S.phi0 ? 1 : 0;
    return 2;
  }
  return 0;
}

// Algorithm 4 after the factorisation (the MSIR mode of the refinement
// kernel): x0, then SIR / SGMRES-IR / GMRES-IR steps with the stopping
// logic, until convergence, a stage that needs a finer u_f (S.phase =
// PH_NEED_ESC) or the end.  Run by every CTA of a cooperative launch, or by
// one CTA alone (cx.G = 1) in the batched engine.  S, s_act, s_reset and
// s_alg live in shared memory.  Returns false if a device wait failed.
template <typename A0, typename F>
__device__ __forceinline__ bool refine_msir(Cx& cx, const RefineArgs& a, RefState& S, unsigned char* gsm, int& s_act,
                            int& s_reset, int& s_alg) {
  bool ok = true;
  const int ff = factor_fmt<F>(a);
  const int arith_f = ff == MSIR_FP64 ? MSIR_FP64 : MSIR_FP32;
  double s = S.s, xnorm = 0.0, nbe = S.nbe;
  if (S.phase == PH_START) {
    if (a.normb == 0.0) {
      FOR_MY_ROWS(cx, i) { a.x[i] = 0.0; a.xbest[i] = 0.0; }
      if (cx.tid == 0) { S.cged = 1; S.status = MSIR_OK; S.phase = PH_DONE; S.nbe = 0.0; S.s = 0.0; }
      __syncthreads();
      return true;  // b = 0: x = 0, converged
    }
    // x0 = fl_u(fl_u(||b||) M_f^{-1} fl_u(b / ||b||)) with the u_f model
    for (int b = cx.cta; b < cx.nblk; b += cx.G)
      for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads) {
        const int pr = a.perm[i];
        const double bt = urnd(__ddiv_rn(a.b[pr], a.normb), S.u);
        put_c(a, arith_f, i, round_to(bt * rscale(a, pr), S.uf), 0.0);
      }
    __syncthreads();
    ok = msolve_arith<F>(cx, a, arith_f, S.uf);
    if (!ok) return false;
    {
      const double nb_u = urnd(a.normb, S.u);
      double mx = 0.0;
      FOR_MY_ROWS(cx, i) {
        const double d0 = urnd(get_z(a, arith_f, i) * cscale(a, i), S.u);
        const double x0 = urnd(nb_u * d0, S.u);
        a.x0[i] = x0;
        mx = nanmax(mx, fabs(x0));
      }
      mx = cta_reduce(mx, 1, cx.tid);
      double v[1] = {mx};
      const int op[1] = {1};
      if (!(ok = grid_reduce<1>(cx, a, v, op))) return false;
      const bool bad = !isfinite(v[0]);
      FOR_MY_ROWS(cx, i) {
        if (bad) a.x0[i] = 0.0;
        a.x[i] = a.x0[i];
        a.xbest[i] = a.x0[i];
      }
    }
    if (!(ok = grid_barrier(a.bar, a.err, cx.G))) return false;
    if (!(ok = residual<A0>(cx, a, a.x, S.ur, s, xnorm))) return false;
    nbe = s / (a.normA * xnorm + a.normb);
    if (cx.tid == 0) {
      S.best_nbe = nbe;
      S.alg = MSIR_ALG_SIR;
      S.it = 0;
      S.rho_max = 0.0;
      S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
      S.phase = PH_ESCALATED + 10;  // running
      rep_new_stage(a, S, cx.cta);
    }
    __syncthreads();
  } else if (S.phase == PH_ESCALATED) {
    if (!(ok = grid_barrier(a.bar, a.err, cx.G))) return false;
    if (!(ok = residual<A0>(cx, a, a.x, S.ur, s, xnorm))) return false;
    nbe = s / (a.normA * xnorm + a.normb);
    if (cx.tid == 0) {
      if (nbe < S.best_nbe) S.best_nbe = nbe;
      S.alg = MSIR_ALG_SIR;
      S.it = 0;
      S.rho_max = 0.0;
      S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
      S.phase = PH_ESCALATED + 10;
      rep_new_stage(a, S, cx.cta);
    }
    __syncthreads();
    if (nbe <= S.best_nbe) FOR_MY_ROWS(cx, i) a.xbest[i] = a.x[i];
  }

  while (true) {
    if (s == 0.0) {
      if (cx.tid == 0) { S.cged = 1; S.status = MSIR_OK; }
      break;
    }
    if (!isfinite(s)) break;
    const int u = S.u, ur = S.ur;
    int kg = -1;
    bool nonfinite = false;
    if (S.alg == MSIR_ALG_SIR) {
      for (int b = cx.cta; b < cx.nblk; b += cx.G)
        for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads) {
          const double rt = scaled_r(a, i, s, ur, u);
          put_c(a, arith_f, i, round_to(rt * rscale(a, a.perm[i]), S.uf), 0.0);
        }
      __syncthreads();
      if (!(ok = msolve_arith<F>(cx, a, arith_f, S.uf))) break;
      FOR_MY_ROWS(cx, i) a.d[i] = urnd(get_z(a, arith_f, i) * cscale(a, i), u);
      __syncthreads();
    } else {
      const int op = S.alg == MSIR_ALG_SGMRES ? u : square_of(u);
      const double tau = a.tau > 0.0 ? a.tau : (u == MSIR_FP32 ? 1e-6 : 1e-10);
      GmresOut go;
      if (u == MSIR_FP32) {
        if (!(ok = gmres<A0, F, float>(cx, a, s, ur, u, op, tau, gsm, go))) break;
      } else {
        if (!(ok = gmres<A0, F, double>(cx, a, s, ur, u, op, tau, gsm, go))) break;
      }
      kg = go.k;
      nonfinite = go.nonfinite;
    }
    // tentative update x_{i+1} = fl_u(x_i + fl_u(fl_u(s) d)) and the norms
    double md = 0.0, mx = 0.0;
    const double su = urnd(s, u);
    FOR_MY_ROWS(cx, i) {
      const double dv = nonfinite ? 0.0 : a.d[i];
      const double xv = a.x[i];
      a.xn[i] = urnd(xv + urnd(su * dv, u), u);
      md = nanmax(md, fabs(dv));
      mx = nanmax(mx, fabs(xv));
    }
    md = cta_reduce(md, 1, cx.tid);
    mx = cta_reduce(mx, 1, cx.tid);
    {
      double v[2] = {md, mx};
      const int op[2] = {1, 1};
      if (!(ok = grid_reduce<2>(cx, a, v, op))) break;
      md = v[0];
      mx = v[1];
    }
    if (nonfinite || !isfinite(md)) {
      // Inf/NaN correction: no update, the step is not counted, next stage
      if (cx.tid == 0) {
        if (cx.cta == 0 && S.nstages >= 1 && S.nstages <= MSIR_MAX_STAGES)
          a.rep->stage[S.nstages - 1].nonfinite = 1;
        if (S.alg == MSIR_ALG_GMRES) {
          S.phase = PH_NEED_ESC;
        } else {
          S.alg += 1;
          S.it = 0;
          S.rho_max = 0.0;
          S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
          rep_new_stage(a, S, cx.cta);
        }
      }
      __syncthreads();
      if (S.phase == PH_NEED_ESC) break;
      continue;
    }
    const double s_old = s, xnorm_old = mx;
    FOR_MY_ROWS(cx, i) a.x[i] = a.xn[i];
    if (!(ok = grid_barrier(a.bar, a.err, cx.G))) break;
    double ferr = 0.0;
    if (!(ok = residual<A0>(cx, a, a.x, ur, s, xnorm, &ferr))) break;
    nbe = s / (a.normA * xnorm + a.normb);
    const bool better = nbe < S.best_nbe;
    // every thread has read S before thread 0 updates it (shared memory)
    __syncthreads();
    if (better) FOR_MY_ROWS(cx, i) a.xbest[i] = a.x[i];
    if (cx.tid == 0) {
      if (better) S.best_nbe = nbe;
      S.it += 1;
      S.total_steps += 1;
      if (kg >= 0) S.total_gmres += kg;
      if (cx.cta == 0 && S.nstages >= 1 && S.nstages <= MSIR_MAX_STAGES) {
        msir_stage& g = a.rep->stage[S.nstages - 1];
        if (kg >= 0 && g.steps < MSIR_MAX_STEPS) g.gmres_iters[g.steps] = kg;
        g.steps += 1;
      }
      int rs = 0;
      s_act = ctl_step(S, a, s_old, md, xnorm_old, nbe, ferr, kg, &rs);
      s_reset = rs;
      s_alg = S.alg;
      S.nbe = nbe;
    }
    __syncthreads();
    // decisions below use s_act/s_reset/s_alg: thread 0 changes S.alg
    // inside this branch while other warps may not have reached it yet
    if (s_act == 1) {
      if (cx.tid == 0) { S.cged = 1; S.status = MSIR_OK; }
      break;
    }
    if (s_act == 2) {
      const bool reset = s_reset != 0;
      if (reset) FOR_MY_ROWS(cx, i) a.x[i] = a.x0[i];
      if (s_alg == MSIR_ALG_GMRES) {
        if (cx.tid == 0) S.phase = PH_NEED_ESC;
        __syncthreads();
        break;
      }
      if (cx.tid == 0) {
        S.alg += 1;
        S.it = 0;
        S.rho_max = 0.0;
        S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
        rep_new_stage(a, S, cx.cta);
      }
      __syncthreads();
      if (reset) {
        if (!(ok = grid_barrier(a.bar, a.err, cx.G))) break;
        if (!(ok = residual<A0>(cx, a, a.x, ur, s, xnorm))) break;
        nbe = s / (a.normA * xnorm + a.normb);
        const bool b2 = nbe < S.best_nbe;
        if (b2) FOR_MY_ROWS(cx, i) a.xbest[i] = a.x[i];
        __syncthreads();
        if (cx.tid == 0 && b2) S.best_nbe = nbe;
        __syncthreads();
      }
    }
  }
  if (cx.tid == 0) {
    S.s = s;
    S.nbe = nbe;
    if (S.phase != PH_NEED_ESC) S.phase = PH_DONE;
  }
  __syncthreads();
  if (ok && S.phase == PH_DONE && !S.cged) {
    // not converged: return the iterate of smallest nbe
    FOR_MY_ROWS(cx, i) a.x[i] = a.xbest[i];
    if (cx.tid == 0) { S.status = MSIR_NOT_CONVERGED; S.nbe = S.best_nbe; }
  }
  return ok;
}

template <typename A0, typename F>
// One CTA per SM.  (Two per SM, with 128 registers per thread, let
// concurrent systems share SMs, but measured slower: spinning and fp64 work
// of one system then slow the other's.)
__global__ void __launch_bounds__(kRefThreads, 1) refine_kernel(RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* gsm = smem_raw + kTrsvSmem + kScaledSmem + kInboxSmem;  // GMRES scalars
  __shared__ RefState S;
  __shared__ int s_act, s_reset, s_alg;

  Cx cx;
  cx.tsm = smem_raw;
  cx.ssm = smem_raw + kTrsvSmem;
  cx.G = gridDim.x;
  cx.cta = blockIdx.x;
  cx.tid = threadIdx.x;
  cx.lane = threadIdx.x & 31;
  cx.warp = threadIdx.x >> 5;
  cx.n = a.n;
  cx.nblk = (a.n + kBlk - 1) / kBlk;
  cx.team_k = a.team_k;
  cx.redbuf = 0;
  cx.inbox = (unsigned long long*)(smem_raw + kTrsvSmem + kScaledSmem);
  cx.C = 1;
  if (a.cluster > 1) {
    // the inbox starts all ones (a tag no hand-off uses); peers write into
    // it only after every CTA of the cluster has filled its own
    for (int i = cx.tid; i < kInboxSmem / 8; i += kRefThreads) cx.inbox[i] = ~0ull;
    unsigned rank, nrank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nrank));
    // the block-to-team mapping assumes rank = block index mod cluster size
    if ((int)nrank == a.cluster && (int)rank == cx.cta % a.cluster && a.cluster <= kMaxCluster) cx.C = a.cluster;
    cluster_sync_all();
  }
  if (cx.tid == 0) S = *a.st;
  __syncthreads();
  cx.epoch = S.epoch;
  cx.mready = S.mready;
  cx.t_ns = S.t_ns;
  bool ok = true;
  if (a.mode == MODE_RESIDUAL) {
    double s = 0.0, xn = 0.0;
    ok = grid_barrier(a.bar, a.err, cx.G) && residual<A0>(cx, a, a.x, a.ap_arith, s, xn);
    if (ok && cx.cta == 0 && cx.tid == 0) *a.res_s = s;
  } else if (a.mode == MODE_APPLY) {
    for (int b = cx.cta; b < cx.nblk; b += cx.G)
      for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads) {
        const int pr = a.perm[i];
        const double v = a.ap_in[pr] * rscale(a, pr);
        put_c(a, a.ap_arith, i, a.ap_arith == MSIR_DD ? v : round_to(v, a.ap_store), 0.0);
      }
    __syncthreads();
    ok = msolve_arith<F>(cx, a, a.ap_arith, a.ap_store);
    if (ok) FOR_MY_ROWS(cx, i) a.ap_out[i] = get_z(a, a.ap_arith, i) * cscale(a, i);
  } else {
    ok = refine_msir<A0, F>(cx, a, S, gsm, s_act, s_reset, s_alg);
  }
  __syncthreads();
  if (!ok && cx.tid == 0) { S.phase = PH_ERROR; S.status = MSIR_ERR_TIMEOUT; }
  if (cx.tid == 0) {
    S.epoch = cx.epoch;
    S.mready = cx.mready;
  }
  __syncthreads();
  if (cx.cta == 0 && cx.tid == 0) *a.st = S;
  // no CTA leaves while a cluster peer may still write into its inbox (every
  // wait before this point is bounded, so every peer arrives)
  if (a.cluster > 1) cluster_sync_all();
}

// Entry point of one instantiation (defined in refine_<a>_<f>.cu).
template <typename A0, typename F> void* refine_entry();

}  // namespace msir
