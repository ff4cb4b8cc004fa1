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
// it depends on publish their flag (epoch counter, release/acquire), then
// one warp solves the 64x64 diagonal block by substitution and publishes.
// Grid barriers are used only where a full vector is needed (matrix-vector
// products) or a global reduction (norms, Gram-Schmidt coefficients).  The
// stage controller is replicated in every CTA: all CTAs compute the same
// decisions from the same reduced values, so control flow stays uniform.
// All waits are bounded (MSIR_ERR_TIMEOUT).
#pragma once

#include "common.cuh"
#include "refine.h"

namespace msir {

// ----------------------------------------------------------- helpers

struct Cx {
  int G, cta, tid, lane, warp, n, nblk;
  unsigned epoch;
  int redbuf;
  unsigned long long* t_ns;  // per-phase timers (CTA 0, thread 0), shared memory
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

// Row dot products a_row . x, one warp, result on every lane.
template <typename A0>
__device__ double row_dot_d(const A0* row, const double* x, int n, int lane) {
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = __fma_rn(AV<A0>::ld(row + j), __ldcg(x + j), acc);
  return warp_sum_d(acc);
}
// Compensated (twice-working-precision) dot product, result as dd.
template <typename A0>
__device__ dd_t row_dot_dd(const A0* row, const double* x, int n, int lane) {
  double s = 0.0, c = 0.0;
  for (int j = lane; j < n; j += 32) {
    dd_t p = two_prod(AV<A0>::ld(row + j), __ldcg(x + j));
    dd_t t = two_sum(s, p.hi);
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

// Accumulator policies of the substitutions.  V: accumulator, L: factor
// element after widening, storage of the vectors: float for AccF (so that
// fp32 solves never touch the scarce fp64 pipe), double for AccD, a pair of
// double arrays (high, low words) for AccDD.
struct AccF {
  using V = float;
  using L = float;
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
  static __device__ __forceinline__ V fma(L l, V y, V acc) { return __fmaf_rn(l, y, acc); }
  static __device__ __forceinline__ V mul(L l, V y) { return __fmul_rn(l, y); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ V div(V a, L d) { return __fdiv_rn(a, d); }
  static __device__ __forceinline__ V store(V v, int fmt) { return round_f(v, fmt); }
  static __device__ __forceinline__ V wsum(V v) { return warp_sum_f(v); }
  static __device__ __forceinline__ V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
};
struct AccD {
  using V = double;
  using L = double;
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V load(const double* hi, const double*, int i) { return __ldcg(hi + i); }
  static __device__ __forceinline__ void save(double* hi, double*, int i, V v) { hi[i] = v; }
  static __device__ __forceinline__ void put(double* hi, double*, int i, double h, double) { hi[i] = h; }
  static __device__ __forceinline__ double get(const double* hi, const double*, int i) { return hi[i]; }
  static __device__ __forceinline__ V fma(L l, V y, V acc) { return __fma_rn(l, y, acc); }
  static __device__ __forceinline__ V mul(L l, V y) { return __dmul_rn(l, y); }
  static __device__ __forceinline__ V sub(V a, V b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ V div(V a, L d) { return __ddiv_rn(a, d); }
  static __device__ __forceinline__ V store(V v, int) { return v; }
  static __device__ __forceinline__ V wsum(V v) { return warp_sum_d(v); }
  static __device__ __forceinline__ V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
};
struct AccDD {
  using V = dd_t;
  using L = double;
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
  static __device__ __forceinline__ V fma(L l, V y, V acc) { return dd_add(acc, dd_mul_d(y, l)); }
  static __device__ __forceinline__ V mul(L l, V y) { return dd_mul_d(y, l); }
  static __device__ __forceinline__ V sub(V a, V b) { return dd_sub(a, b); }
  static __device__ __forceinline__ V div(V a, L d) { return dd_div_d(a, d); }
  static __device__ __forceinline__ V store(V v, int) { return v; }
  static __device__ __forceinline__ V wsum(V v) { return warp_sum_dd(v); }
  static __device__ __forceinline__ V shfl(V v, int src) {
    return dd_t{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
  }
};

template <typename Lt, typename F>
__device__ __forceinline__ Lt ld_fac(const F* p) {
  return (Lt)to_f(*p);
}

constexpr int kDtLd = kBlk + 1;

// One triangular solve (LOWER: L y = c, unit diagonal; else U z = y) over
// all blocks this CTA owns.
template <typename F, typename ACC, bool LOWER>
__device__ bool trsv(Cx& cx, const RefineArgs& a, int store_fmt, void* Dt_raw) {
  using V = typename ACC::V;
  using Lt = typename ACC::L;
  __shared__ V s_sum[kBlk];
  Lt* Dt = (Lt*)Dt_raw;
  const F* LU = (const F*)a.LU;
  const int ldf = a.ldf, n = cx.n;
  const unsigned epoch = ++cx.epoch;
  const double* in_hi = LOWER ? a.c_hi : a.y_hi;
  const double* in_lo = LOWER ? a.c_lo : a.y_lo;
  const double* src_hi = LOWER ? a.y_hi : a.z_hi;  // solved components read from other blocks
  const double* src_lo = LOWER ? a.y_lo : a.z_lo;
  double* out_hi = LOWER ? a.y_hi : a.z_hi;
  double* out_lo = LOWER ? a.y_lo : a.z_lo;
  const int nmine = cx.cta < cx.nblk ? (cx.nblk - 1 - cx.cta) / cx.G + 1 : 0;
  for (int q = 0; q < nmine; ++q) {
    const int b = LOWER ? cx.cta + q * cx.G : cx.cta + (nmine - 1 - q) * cx.G;
    const int r0 = b * kBlk;
    const int nr = min(kBlk, n - r0);
    unsigned long long* ts = a.tsv ? a.tsv + ((LOWER ? 0 : 1) * (size_t)cx.nblk + b) * 3 : nullptr;
    if (ts && cx.tid == 0) ts[0] = gtimer();
    // diagonal tile, transposed: Dt[m][i] = T[r0+i][r0+m]
    for (int idx = cx.tid; idx < kBlk * kBlk; idx += kRefThreads) {
      const int i = idx / kBlk, m = idx % kBlk;
      Lt v = (Lt)0;
      if (i < nr && m < nr && (LOWER ? m < i : m >= i)) v = ld_fac<Lt>(LU + (size_t)(r0 + i) * ldf + r0 + m);
      if (!LOWER && i == m && i >= nr) v = (Lt)1;  // padding rows of a partial block: identity
      Dt[m * kDtLd + i] = v;
    }
    // off-diagonal products
    V acc[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = ACC::zero();
    const int njb = LOWER ? b : cx.nblk - 1 - b;
    for (int t = 0; t < njb; ++t) {
      const int jb = LOWER ? t : cx.nblk - 1 - t;
      const int c0 = jb * kBlk;
      const int ca = c0 + cx.lane, cb = c0 + 32 + cx.lane;
      // the tile of L (U) does not depend on the flag: load it first
      Lt la[8], lb[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int row = r0 + cx.warp * 8 + rr;
        const F* lr = LU + (size_t)row * ldf;
        la[rr] = (row < n && ca < n) ? ld_fac<Lt>(lr + ca) : (Lt)0;
        lb[rr] = (row < n && cb < n) ? ld_fac<Lt>(lr + cb) : (Lt)0;
      }
      if (!wait_flag(a.flags + (size_t)jb * kFlagStride, epoch, a.err)) return false;
      V y0 = ACC::zero(), y1 = ACC::zero();
      if (ca < n) y0 = ACC::load(src_hi, src_lo, ca);
      if (cb < n) y1 = ACC::load(src_hi, src_lo, cb);
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        acc[rr] = ACC::fma(la[rr], y0, acc[rr]);
        acc[rr] = ACC::fma(lb[rr], y1, acc[rr]);
      }
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      V sm = ACC::wsum(acc[rr]);
      if (cx.lane == 0) s_sum[cx.warp * 8 + rr] = sm;
    }
    __syncthreads();
    if (ts && cx.tid == 0) ts[1] = gtimer();
    if (cx.warp == 0) {
      const int l = cx.lane;
      V z0 = ACC::zero(), z1 = ACC::zero();
      if (l < nr) z0 = ACC::sub(ACC::load(in_hi, in_lo, r0 + l), s_sum[l]);
      if (l + 32 < nr) z1 = ACC::sub(ACC::load(in_hi, in_lo, r0 + 32 + l), s_sum[32 + l]);
      // Fully unrolled: each lane keeps its two rows; rows beyond nr stay 0
      // and are never stored.  y_m is broadcast from lane m mod 32.
      V y0 = ACC::zero(), y1 = ACC::zero();
      if (LOWER) {
#pragma unroll
        for (int m = 0; m < 32; ++m) {
          const V ym = ACC::store(ACC::shfl(z0, m), store_fmt);
          if (l == m) y0 = ym;
          if (l > m) z0 = ACC::sub(z0, ACC::mul(Dt[m * kDtLd + l], ym));
          z1 = ACC::sub(z1, ACC::mul(Dt[m * kDtLd + l + 32], ym));
        }
#pragma unroll
        for (int m = 32; m < 64; ++m) {
          const V ym = ACC::store(ACC::shfl(z1, m - 32), store_fmt);
          if (l == m - 32) y1 = ym;
          if (l + 32 > m) z1 = ACC::sub(z1, ACC::mul(Dt[m * kDtLd + l + 32], ym));
        }
      } else {
#pragma unroll
        for (int m = 63; m >= 32; --m) {
          const V xm = ACC::store(ACC::div(ACC::shfl(z1, m - 32), Dt[m * kDtLd + m]), store_fmt);
          if (l == m - 32) y1 = xm;
          if (l + 32 < m) z1 = ACC::sub(z1, ACC::mul(Dt[m * kDtLd + l + 32], xm));
          z0 = ACC::sub(z0, ACC::mul(Dt[m * kDtLd + l], xm));
        }
#pragma unroll
        for (int m = 31; m >= 0; --m) {
          const V xm = ACC::store(ACC::div(ACC::shfl(z0, m), Dt[m * kDtLd + m]), store_fmt);
          if (l == m) y0 = xm;
          if (l < m) z0 = ACC::sub(z0, ACC::mul(Dt[m * kDtLd + l], xm));
        }
      }
      if (l < nr) ACC::save(out_hi, out_lo, r0 + l, y0);
      if (l + 32 < nr) ACC::save(out_hi, out_lo, r0 + 32 + l, y1);
      __syncwarp();
      if (l == 0) {
        st_release_u32(a.flags + (size_t)b * kFlagStride, epoch);
        if (ts) ts[2] = gtimer();
      }
    }
    __syncthreads();
  }
  return true;
}

// M^{-1} applied to the right-hand side already placed in c (permuted
// order, scaled by R, rounded to the storage format): forward then backward
// substitution.  Result in z (natural order, before the S*mu scaling).
template <typename F, typename ACC>
__device__ bool msolve(Cx& cx, const RefineArgs& a, int store_fmt, void* Dt) {
  {
    PhaseTimer pt(cx, 1);
    if (!trsv<F, ACC, true>(cx, a, store_fmt, Dt)) return false;
  }
  PhaseTimer pt(cx, 2);
  return trsv<F, ACC, false>(cx, a, store_fmt, Dt);
}

template <typename F>
__device__ bool msolve_arith(Cx& cx, const RefineArgs& a, int arith, int store_fmt, void* Dt) {
  if (arith == MSIR_FP32) return msolve<F, AccF>(cx, a, store_fmt, Dt);
  if (arith == MSIR_FP64) return msolve<F, AccD>(cx, a, store_fmt, Dt);
  return msolve<F, AccDD>(cx, a, store_fmt, Dt);
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

static __device__ __forceinline__ double rscale(const RefineArgs& a, int row) {
  return a.Rsc ? a.Rsc[row] : 1.0;
}
static __device__ __forceinline__ double cscale(const RefineArgs& a, int col) {
  return a.Ssc ? a.Ssc[col] * a.mu : 1.0;
}

// ------------------------------------------------------------ residual

// r_p[i] = b[perm[i]] - A[perm[i]] x in ur; rows are spread over every warp
// of the grid (the fp64 work needs all SMs).  Returns (via grid reduction)
// s = ||r||_inf and ||x||_inf.  The caller has made x complete (barrier).
template <typename A0>
__device__ bool residual(Cx& cx, const RefineArgs& a, const double* x, int ur, double& s,
                         double& xnorm) {
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
  for (int i = cx.cta * kRefThreads + cx.tid; i < cx.n; i += cx.G * kRefThreads)
    mx = nanmax(mx, fabs(__ldcg(x + i)));
  mr = cta_reduce(mr, 1, cx.tid);
  mx = cta_reduce(mx, 1, cx.tid);
  double v[2] = {mr, mx};
  const int op[2] = {1, 1};
  if (!grid_reduce<2>(cx, a, v, op)) return false;
  s = v[0];
  xnorm = v[1];
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
// placed in c.  op = FP32: fp32 accumulation, rows of my blocks (no barrier
// needed before the substitution); FP64 / DD: rows over every warp of the
// grid, followed by a grid barrier.
template <typename A0, typename U>
__device__ bool apply_A(Cx& cx, const RefineArgs& a, const U* v, int op) {
  PhaseTimer pt(cx, 4);
  const A0* A = (const A0*)a.A;
  if (op == MSIR_FP32) {
    for (int b = cx.cta; b < cx.nblk; b += cx.G) {
      for (int rr = 0; rr < 8; ++rr) {
        const int i = b * kBlk + cx.warp * 8 + rr;
        if (i >= cx.n) break;
        const int ar = a.perm[i];
        const A0* row = A + (size_t)ar * a.lda;
        float acc = 0.0f;
        for (int j = cx.lane; j < cx.n; j += 32) acc = __fmaf_rn((float)__ldg(row + j), (float)__ldcg(v + j), acc);
        acc = warp_sum_f(acc);
        if (cx.lane == 0) {
          const float R = a.Rsc ? (float)a.Rsc[ar] : 1.0f;
          ((float*)a.c_hi)[i] = __fmul_rn(acc, R);
        }
      }
    }
    __syncthreads();
    return true;
  }
  const int nw = cx.G * (kRefThreads / 32);
  for (int i = cx.cta * (kRefThreads / 32) + cx.warp; i < cx.n; i += nw) {
    const int ar = a.perm[i];
    const A0* row = A + (size_t)ar * a.lda;
    const double R = rscale(a, ar);
    if (op == MSIR_DD) {
      double sh = 0.0, sc = 0.0;
      for (int j = cx.lane; j < cx.n; j += 32) {
        const dd_t p = two_prod((double)__ldg(row + j), (double)__ldcg(v + j));
        const dd_t t = two_sum(sh, p.hi);
        sh = t.hi;
        sc = __dadd_rn(sc, __dadd_rn(t.lo, p.lo));
      }
      const dd_t tt = warp_sum_dd(fast_two_sum(sh, sc));
      if (cx.lane == 0) { a.c_hi[i] = tt.hi * R; a.c_lo[i] = tt.lo * R; }
    } else {
      double acc = 0.0;
      for (int j = cx.lane; j < cx.n; j += 32) acc = __fma_rn((double)__ldg(row + j), (double)__ldcg(v + j), acc);
      acc = warp_sum_d(acc);
      if (cx.lane == 0) a.c_hi[i] = acc * R;
    }
  }
  return grid_barrier(a.bar, a.err, cx.G);
}

// out_i = fl_u(z_i * S_i * mu) for my rows
template <typename U>
__device__ void finish_solve(Cx& cx, const RefineArgs& a, U* out, int arith) {
  FOR_MY_ROWS(cx, i) out[i] = UA<U>::rnd(get_z(a, arith, i) * cscale(a, i));
  __syncthreads();
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

// partial sums p_j = sum over my rows of V_j[i] * w[i], j = 0..k.  Sums are
// accumulated in fp64 (a product of two fp32 values is exact in fp64), then
// rounded to u, as the oracle's reading of "inner products in u" states.
template <typename U>
__device__ void cgs_partials(Cx& cx, const RefineArgs& a, const U* V, const U* w, int kp1) {
  PhaseTimer pt(cx, 3);
  for (int j = cx.warp; j < kp1; j += kRefThreads / 32) {
    const U* Vj = V + (size_t)j * a.ldv;
    double acc = 0.0;
    for (int b = cx.cta; b < cx.nblk; b += cx.G)
      for (int i = b * kBlk + cx.lane; i < min((b + 1) * kBlk, cx.n); i += 32)
        acc = __fma_rn((double)__ldcg(Vj + i), (double)__ldcg(w + i), acc);
    acc = warp_sum_d(acc);
    if (cx.lane == 0) a.hred[(size_t)cx.cta * (a.kcap + 1) + j] = acc;
  }
}

// w_i = fl_u(w_i - sum_j V_j[i] h_j), the sum in fp64
template <typename U>
__device__ void cgs_update(Cx& cx, const RefineArgs& a, const U* V, U* w, int kp1, const U* s_h) {
  PhaseTimer pt(cx, 3);
  FOR_MY_ROWS(cx, i) {
    double acc = 0.0;
    for (int j = 0; j < kp1; ++j) acc = __fma_rn((double)__ldcg(V + (size_t)j * a.ldv + i), (double)s_h[j], acc);
    w[i] = UA<U>::rnd(__dsub_rn((double)w[i], acc));
  }
  __syncthreads();
}

template <typename U>
__device__ bool grid_sum_sq(Cx& cx, const RefineArgs& a, const U* w, double& out) {
  double ss = 0.0;
  FOR_MY_ROWS(cx, i) {
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
                      void* Dt, unsigned char* gsm, GmresOut& out) {
  using M = UA<U>;
  __shared__ double s_bc[1];
  const int kcap = a.kcap;
  U* sm_cs = (U*)gsm;
  U* sm_sn = sm_cs + kcap + 1;
  U* sm_g = sm_sn + kcap + 1;   // kcap + 2
  U* s_h = sm_g + kcap + 2;     // 2 (kcap + 1)
  U* V = (U*)a.V;
  U* w = (U*)a.w;
  out.k = 0;
  out.nonfinite = false;
  // w0 = fl_u(M^{-1} r~) with the substitutions in op
  for (int b = cx.cta; b < cx.nblk; b += cx.G)
    for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads)
      put_c(a, op, i, scaled_r(a, i, s, ur, u) * rscale(a, a.perm[i]), 0.0);
  __syncthreads();
  if (!msolve_arith<F>(cx, a, op, op, Dt)) return false;
  finish_solve<U>(cx, a, w, op);
  double ss;
  if (!grid_sum_sq<U>(cx, a, w, ss)) return false;
  const U beta = M::sqrt_(M::rnd(ss));
  if (!isfinite((double)beta)) { out.nonfinite = true; return true; }
  if (beta == (U)0) {
    FOR_MY_ROWS(cx, i) a.d[i] = 0.0;
    __syncthreads();
    return true;
  }
  FOR_MY_ROWS(cx, i) V[i] = M::div(w[i], beta);
  if (cx.tid == 0) sm_g[0] = beta;
  __syncthreads();
  int kdone = 0;
  for (int k = 0; k < kcap; ++k) {
    // full V_k needed by the matrix-vector product
    if (!grid_barrier(a.bar, a.err, cx.G)) return false;
    if (!apply_A<A0, U>(cx, a, V + (size_t)k * a.ldv, op)) return false;
    if (!msolve_arith<F>(cx, a, op, op, Dt)) return false;
    finish_solve<U>(cx, a, w, op);
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
    if (cx.tid == 0) {
      for (int i = 0; i < k; ++i) {
        const U x0 = s_h[i], x1 = s_h[i + 1];
        s_h[i] = M::add(M::mul(sm_cs[i], x0), M::mul(sm_sn[i], x1));
        s_h[i + 1] = M::add(M::mul(-sm_sn[i], x0), M::mul(sm_cs[i], x1));
      }
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
      if (cx.cta == 0) {
        double* Hk = a.H + (size_t)k * (kcap + 1);
        for (int i = 0; i <= k; ++i) Hk[i] = (double)s_h[i];
      }
    }
    __syncthreads();
    if (cx.cta == 0 && cx.tid == 0) cx.t_ns[6] += gtimer() - tg0;
    const double relres = s_bc[0];
    kdone = k + 1;
    if (hk1 != (U)0 && isfinite((double)hk1)) {
      FOR_MY_ROWS(cx, i) V[(size_t)(k + 1) * a.ldv + i] = M::div(w[i], hk1);
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
  FOR_MY_ROWS(cx, i) {
    double acc = 0.0;
    for (int j = 0; j < kdone; ++j) acc = __fma_rn((double)__ldcg(V + (size_t)j * a.ldv + i), (double)s_h[j], acc);
    a.d[i] = (double)M::rnd(acc);
  }
  __syncthreads();
  out.k = kdone;
  return true;
}

// -------------------------------------------------------------- kernel

static __device__ void rep_new_stage(const RefineArgs& a, RefState& S) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && S.nstages < MSIR_MAX_STAGES) {
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
                               double nbe, int kg, int* reset) {
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

template <typename A0, typename F>
__global__ void __launch_bounds__(kRefThreads, 1) refine_kernel(RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  void* Dt = smem_raw;                                               // kBlk x kDtLd (double)
  unsigned char* gsm = smem_raw + sizeof(double) * kBlk * kDtLd;     // GMRES scalars
  __shared__ RefState S;
  __shared__ int s_act, s_reset;

  Cx cx;
  cx.G = gridDim.x;
  cx.cta = blockIdx.x;
  cx.tid = threadIdx.x;
  cx.lane = threadIdx.x & 31;
  cx.warp = threadIdx.x >> 5;
  cx.n = a.n;
  cx.nblk = (a.n + kBlk - 1) / kBlk;
  cx.redbuf = 0;
  if (cx.tid == 0) S = *a.st;
  __syncthreads();
  cx.epoch = S.epoch;
  cx.t_ns = S.t_ns;
  bool ok = true;
  const int ff = Fmt<F>::code;
  const int arith_f = ff == MSIR_FP64 ? MSIR_FP64 : MSIR_FP32;

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
    ok = msolve_arith<F>(cx, a, a.ap_arith, a.ap_store, Dt);
    if (ok) FOR_MY_ROWS(cx, i) a.ap_out[i] = get_z(a, a.ap_arith, i) * cscale(a, i);
  } else {
    // ------------------------------------------------------------ MSIR
    double s = S.s, xnorm = 0.0, nbe = S.nbe;
    if (S.phase == PH_START) {
      if (a.normb == 0.0) {
        FOR_MY_ROWS(cx, i) { a.x[i] = 0.0; a.xbest[i] = 0.0; }
        if (cx.tid == 0) { S.cged = 1; S.status = MSIR_OK; S.phase = PH_DONE; S.nbe = 0.0; S.s = 0.0; }
        __syncthreads();
        goto finish;
      }
      // x0 = fl_u(fl_u(||b||) M_f^{-1} fl_u(b / ||b||)) with the u_f model
      for (int b = cx.cta; b < cx.nblk; b += cx.G)
        for (int i = b * kBlk + cx.tid; i < min((b + 1) * kBlk, cx.n); i += kRefThreads) {
          const int pr = a.perm[i];
          const double bt = urnd(__ddiv_rn(a.b[pr], a.normb), S.u);
          put_c(a, arith_f, i, round_to(bt * rscale(a, pr), S.uf), 0.0);
        }
      __syncthreads();
      ok = msolve_arith<F>(cx, a, arith_f, S.uf, Dt);
      if (!ok) goto finish;
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
        if (!(ok = grid_reduce<1>(cx, a, v, op))) goto finish;
        const bool bad = !isfinite(v[0]);
        FOR_MY_ROWS(cx, i) {
          if (bad) a.x0[i] = 0.0;
          a.x[i] = a.x0[i];
          a.xbest[i] = a.x0[i];
        }
      }
      if (!(ok = grid_barrier(a.bar, a.err, cx.G))) goto finish;
      if (!(ok = residual<A0>(cx, a, a.x, S.ur, s, xnorm))) goto finish;
      nbe = s / (a.normA * xnorm + a.normb);
      if (cx.tid == 0) {
        S.best_nbe = nbe;
        S.alg = MSIR_ALG_SIR;
        S.it = 0;
        S.rho_max = 0.0;
        S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
        S.phase = PH_ESCALATED + 10;  // running
        rep_new_stage(a, S);
      }
      __syncthreads();
    } else if (S.phase == PH_ESCALATED) {
      if (!(ok = grid_barrier(a.bar, a.err, cx.G))) goto finish;
      if (!(ok = residual<A0>(cx, a, a.x, S.ur, s, xnorm))) goto finish;
      nbe = s / (a.normA * xnorm + a.normb);
      if (cx.tid == 0) {
        if (nbe < S.best_nbe) S.best_nbe = nbe;
        S.alg = MSIR_ALG_SIR;
        S.it = 0;
        S.rho_max = 0.0;
        S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
        S.phase = PH_ESCALATED + 10;
        rep_new_stage(a, S);
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
        if (!(ok = msolve_arith<F>(cx, a, arith_f, S.uf, Dt))) break;
        FOR_MY_ROWS(cx, i) a.d[i] = urnd(get_z(a, arith_f, i) * cscale(a, i), u);
        __syncthreads();
      } else {
        const int op = S.alg == MSIR_ALG_SGMRES ? u : square_of(u);
        const double tau = a.tau > 0.0 ? a.tau : (u == MSIR_FP32 ? 1e-6 : 1e-10);
        GmresOut go;
        if (u == MSIR_FP32) {
          if (!(ok = gmres<A0, F, float>(cx, a, s, ur, u, op, tau, Dt, gsm, go))) break;
        } else {
          if (!(ok = gmres<A0, F, double>(cx, a, s, ur, u, op, tau, Dt, gsm, go))) break;
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
            rep_new_stage(a, S);
          }
        }
        __syncthreads();
        if (S.phase == PH_NEED_ESC) break;
        continue;
      }
      const double s_old = s, xnorm_old = mx;
      FOR_MY_ROWS(cx, i) a.x[i] = a.xn[i];
      if (!(ok = grid_barrier(a.bar, a.err, cx.G))) break;
      if (!(ok = residual<A0>(cx, a, a.x, ur, s, xnorm))) break;
      nbe = s / (a.normA * xnorm + a.normb);
      const bool better = nbe < S.best_nbe;
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
        s_act = ctl_step(S, a, s_old, md, xnorm_old, nbe, kg, &rs);
        s_reset = rs;
        S.nbe = nbe;
      }
      __syncthreads();
      if (s_act == 1) {
        if (cx.tid == 0) { S.cged = 1; S.status = MSIR_OK; }
        break;
      }
      if (s_act == 2) {
        const bool reset = s_reset != 0;
        if (reset) FOR_MY_ROWS(cx, i) a.x[i] = a.x0[i];
        if (S.alg == MSIR_ALG_GMRES) {
          if (cx.tid == 0) S.phase = PH_NEED_ESC;
          __syncthreads();
          break;
        }
        if (cx.tid == 0) {
          S.alg += 1;
          S.it = 0;
          S.rho_max = 0.0;
          S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
          rep_new_stage(a, S);
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
  }
finish:
  __syncthreads();
  if (!ok && cx.tid == 0) { S.phase = PH_ERROR; S.status = MSIR_ERR_TIMEOUT; }
  if (cx.tid == 0) S.epoch = cx.epoch;
  __syncthreads();
  if (cx.cta == 0 && cx.tid == 0) *a.st = S;
}

// Entry point of one instantiation (defined in refine_<a>_<f>.cu).
template <typename A0, typename F> void* refine_entry();

}  // namespace msir
