// Inverses of the 64x64 diagonal blocks of packed LU factors (device code
// shared by the inverse kernel and the batched engine).
//
// The inverse X = B^{-1} of one diagonal block is formed in double-double
// by substitution on the columns of the identity: row i of X follows from
// row i of B X = I once the rows it depends on are known (first to last for
// the unit lower L, last to first for U).  Thread (c, part) accumulates a
// quarter of the terms of column c with a compensated sum (TwoProduct
// terms, TwoSum on the running sum, errors summed apart, as in Ogita, Rump
// and Oishi's Dot2), and the four quarters are combined with the accurate
// dd addition.  The relative accuracy is about kappa(B) 2^-100, so rounding
// the result once gives the correctly rounded fp32 and fp64 inverses except
// within that distance of a rounding boundary.
//
// Outputs, each [2][nblk][64][64] row-major (triangle 0 = L, 1 = U), zero
// outside the n - 64 b rows and columns of a ragged last block:
//   inv32  fp32 rounding of the dd inverse (one rounding of hi + lo)
//   inv_hi, inv_lo  the dd inverse (hi = its fp64 rounding)
#pragma once

#include "common.cuh"

namespace msir {

constexpr int kIB = 64;
constexpr int kInvThreads = 256;  // 64 columns x 4 partial sums
constexpr int kXld = kIB + 1;
constexpr size_t kInvSmem = sizeof(double) * 3 * kIB * kXld;

// fp32 value nearest to hi + lo (normalised dd): fl32(hi) unless hi is an
// exact tie between two fp32 neighbours, in which case lo decides.
__device__ __forceinline__ float dd_to_f32(double hi, double lo) {
  const float r = __double2float_rn(hi);
  const double rd = (double)r;
  const double d = hi - rd;  // exact
  if (d == 0.0 || lo == 0.0 || !isfinite(rd)) return r;
  const float o = nextafterf(r, d > 0.0 ? INFINITY : -INFINITY);
  if ((double)o - rd != 2.0 * d) return r;  // not a tie
  return ((lo > 0.0) == (d > 0.0)) ? o : r;
}

// One diagonal block b of triangle `lower` (L if true, else U), by one
// block of kInvThreads threads; sm_inv holds kInvSmem bytes.
template <typename F>
__device__ void inv_diag_block(const F* __restrict__ LU, int ldf, int n, int nblk, int b, bool lower,
                               float* inv32, double* inv_hi, double* inv_lo, double* sm_inv) {
  double* B = sm_inv;            // the diagonal block, identity-padded
  double* Xh = B + kIB * kXld;   // inverse, high words
  double* Xl = Xh + kIB * kXld;  // inverse, low words
  const int r0 = b * kIB;
  const int nr = min(kIB, n - r0);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kIB * kIB; idx += kInvThreads) {
    const int i = idx / kIB, k = idx % kIB;
    double v = 0.0;
    if (i < nr && k < nr) {
      if (lower ? k < i : k >= i) v = (double)to_f(LU[(size_t)(r0 + i) * ldf + r0 + k]);
      else if (k == i) v = 1.0;  // unit diagonal of L
    } else if (i == k) {
      v = 1.0;
    }
    B[i * kXld + k] = v;
    Xh[i * kXld + k] = 0.0;
    Xl[i * kXld + k] = 0.0;
  }
  __syncthreads();
  const int c = tid >> 2, part = tid & 3;
  for (int step = 0; step < kIB; ++step) {
    const int i = lower ? step : kIB - 1 - step;
    const bool active = lower ? c <= i : c >= i;
    // sum over the known rows k of B[i][k] X[k][c]; X[k][c] = 0 outside
    // the triangle, so only k in [c, i) (L) or (i, c] (U) contribute
    double sh = 0.0, sl = 0.0;
    if (active) {
      const int k0 = lower ? c : i + 1;
      const int k1 = lower ? i : c + 1;
      for (int k = k0 + part; k < k1; k += 4) {
        const double bik = B[i * kXld + k];
        const dd_t p = two_prod(bik, Xh[k * kXld + c]);
        const double pl = __fma_rn(bik, Xl[k * kXld + c], p.lo);
        const dd_t t = two_sum(sh, p.hi);
        sh = t.hi;
        sl = __dadd_rn(sl, __dadd_rn(t.lo, pl));
      }
    }
    dd_t s = two_sum(sh, sl);
    s = dd_add(s, dd_shfl_xor(s, 1));
    s = dd_add(s, dd_shfl_xor(s, 2));
    if (active && part == 0) {
      dd_t x = dd_sub(dd_t{i == c ? 1.0 : 0.0, 0.0}, s);
      if (!lower) x = dd_div_d(x, B[i * kXld + i]);
      Xh[i * kXld + c] = x.hi;
      Xl[i * kXld + c] = x.lo;
    }
    __syncthreads();
  }
  const size_t base = ((size_t)(lower ? 0 : 1) * nblk + b) * kIB * kIB;
  for (int idx = tid; idx < kIB * kIB; idx += kInvThreads) {
    const int i = idx / kIB, k = idx % kIB;
    double h = Xh[i * kXld + k], l = Xl[i * kXld + k];
    if (i >= nr || k >= nr) h = l = 0.0;
    inv_hi[base + idx] = h;
    inv_lo[base + idx] = l;
    inv32[base + idx] = dd_to_f32(h, l);
  }
}

}  // namespace msir
