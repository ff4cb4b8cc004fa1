// LU factorisation by one thread block, for the batched engine's small
// systems (n <= kCtaLuMax): Algorithm 4's first step, A = LU by blocked
// right-looking GEPP in u_f (Sec. 1), with the rounding points of the
// library's multi-kernel LU:
//
//  * the matrix is held in u_f storage between steps;
//  * a panel of nb columns is widened to the arithmetic precision T (fp32
//    for u_f <= fp32, fp64 for u_f = fp64) and factored column by column:
//    pivot = largest |a_ij| (ties to the smallest row, NaN never chosen
//    unless every candidate is NaN), full panel rows swapped, the column
//    below divided by the pivot, the trailing panel columns updated with a
//    rounded product and a rounded difference; a zero pivot is recorded and
//    skipped; the panel is stored back in u_f;
//  * interchanges reach the other columns of the outer block, U12 =
//    L11^{-1} A12 by forward substitution in T (rounded product, rounded
//    difference, ascending), stored in u_f;
//  * trailing updates: per element a fused multiply-add chain in T over the
//    K products in ascending order from zero, then one rounded difference
//    and the u_f store.  Two-level blocking: panels of nb inside outer
//    blocks of nbo columns.
//
// For u_f = fp32 / fp64 this is the oracle's model operation for operation.
// The bf16 / fp16 outer update (K = nbo), which the multi-kernel LU runs on
// the tensor cores with fp32 accumulation in an order the hardware does not
// fix, is here the ascending fp32 chain.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace msir {

constexpr int kCtaLuMax = 512;    // largest n the batched engine factors in one block
constexpr int kCtaLuThreads = 256;

template <typename T> struct TArith;
template <> struct TArith<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct TArith<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// arithmetic precision of a u_f factorisation
template <typename F>
using LuT = typename std::conditional<std::is_same<F, double>::value, double, float>::type;

template <typename F>
__device__ __forceinline__ F lu_store(LuT<F> v) {
  if constexpr (std::is_same<F, double>::value) return v;
  else return from_t<F>(v);
}

// bytes of shared memory cta_lu needs: the largest of its three uses of
// the same space, a panel of width nb (row stride nb + 1) over up to
// kCtaLuMax rows, the substitution's L11 and column chunk (two 64 x 65
// tiles) and the update's L21 and U12 tiles (32 x 65 and 64 x 33)
template <typename F>
constexpr size_t cta_lu_smem(int nb) {
  const size_t panel = (size_t)kCtaLuMax * (nb + 1);
  const size_t trsm = (size_t)2 * 64 * 65;
  const size_t upd = (size_t)32 * 65 + 64 * 33;
  const size_t m = panel > trsm ? panel : trsm;
  return (m > upd ? m : upd) * sizeof(LuT<F>);
}

// Argmax of |P[r][j]| over rows r in [j, m) (NaN counts as -1, ties go to
// the smaller row), by the whole block; returns the row on every thread.
template <typename T>
__device__ int cta_pivot(const T* P, int ldp, int j, int m, double* s_val, int* s_idx) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double bv = -2.0;
  int bi = m;
  for (int r = j + tid; r < m; r += kCtaLuThreads) {
    double a = fabs((double)P[r * ldp + j]);
    if (isnan(a)) a = -1.0;
    if (a > bv || (a == bv && r < bi)) { bv = a; bi = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if (lane == 0) { s_val[warp] = bv; s_idx[warp] = bi; }
  __syncthreads();
  if (tid == 0) {
    double v = s_val[0];
    int i = s_idx[0];
    for (int w = 1; w < kCtaLuThreads / 32; ++w)
      if (s_val[w] > v || (s_val[w] == v && s_idx[w] < i)) { v = s_val[w]; i = s_idx[w]; }
    s_idx[0] = i;
  }
  __syncthreads();
  const int p = s_idx[0];
  __syncthreads();  // s_idx is reused by the next column
  return p;
}

// Factor the panel A[kk.., kk..kk+w) (m = n - kk rows); ipiv gets global rows.
template <typename F>
__device__ void cta_panel(F* A, int lda, int n, int kk, int w, int* ipiv, int& info, int& nonfinite,
                          LuT<F>* P, double* s_val, int* s_idx) {
  using T = LuT<F>;
  using X = TArith<T>;
  const int m = n - kk, ldp = w + 1, tid = threadIdx.x;
  for (int e = tid; e < m * w; e += kCtaLuThreads) {
    const int r = e / w, c = e % w;
    P[r * ldp + c] = (T)to_f(A[(size_t)(kk + r) * lda + kk + c]);
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    const int p = cta_pivot<T>(P, ldp, j, m, s_val, s_idx);
    if (tid == 0) ipiv[kk + j] = kk + p;
    if (p != j && tid < w) {
      const T t = P[j * ldp + tid];
      P[j * ldp + tid] = P[p * ldp + tid];
      P[p * ldp + tid] = t;
    }
    __syncthreads();
    const T piv = P[j * ldp + j];
    if (piv != (T)0) {
      for (int r = j + 1 + tid; r < m; r += kCtaLuThreads) {
        const T l = X::div(P[r * ldp + j], piv);
        P[r * ldp + j] = l;
        for (int c = j + 1; c < w; ++c) P[r * ldp + c] = X::sub(P[r * ldp + c], X::mul(l, P[j * ldp + c]));
      }
    } else if (tid == 0 && info == 0) {
      info = kk + j + 1;
    }
    __syncthreads();
  }
  int bad = 0;
  for (int e = tid; e < m * w; e += kCtaLuThreads) {
    const int r = e / w, c = e % w;
    const F v = lu_store<F>(P[r * ldp + c]);
    bad |= !isfinite((double)to_f(v));
    A[(size_t)(kk + r) * lda + kk + c] = v;
  }
  if (__syncthreads_or(bad) && tid == 0) nonfinite = 1;
}

// Interchanges of rows r0 .. r0+w-1 (ipiv) applied to columns [c0, c1).
template <typename F>
__device__ void cta_swap_cols(F* A, int lda, const int* ipiv, int r0, int w, int c0, int c1) {
  for (int c = c0 + threadIdx.x; c < c1; c += kCtaLuThreads)
    for (int j = r0; j < r0 + w; ++j) {
      const int p = ipiv[j];
      if (p != j) {
        const F t = A[(size_t)j * lda + c];
        A[(size_t)j * lda + c] = A[(size_t)p * lda + c];
        A[(size_t)p * lda + c] = t;
      }
    }
  __syncthreads();
}

// U12 = L11^{-1} A12 for rows r0 .. r0+w-1 (w <= 64), columns [c0, c1), in T
// with the stored unit lower L11; stored in u_f.  Chunks of 64 columns are
// held in shared memory; step m updates every row below m of the chunk in
// parallel (each element keeps the ascending order of its terms).
template <typename F>
__device__ void cta_trsm(F* A, int lda, int r0, int w, int c0, int c1, int& nonfinite, LuT<F>* sm) {
  using T = LuT<F>;
  using X = TArith<T>;
  if (c1 <= c0) return;
  constexpr int CW = 64, LD = 65;
  T* Ls = sm;            // w x w, stride 65
  T* Xs = sm + 64 * LD;  // w x CW, stride 65
  const int tid = threadIdx.x;
  for (int e = tid; e < w * w; e += kCtaLuThreads) {
    const int i = e / w, k = e % w;
    Ls[i * LD + k] = (T)to_f(A[(size_t)(r0 + i) * lda + r0 + k]);
  }
  int bad = 0;
  for (int cb = c0; cb < c1; cb += CW) {
    const int cw = min(CW, c1 - cb);
    for (int e = tid; e < w * cw; e += kCtaLuThreads) {
      const int i = e / cw, j = e % cw;
      Xs[i * LD + j] = (T)to_f(A[(size_t)(r0 + i) * lda + cb + j]);
    }
    __syncthreads();
    for (int m = 0; m + 1 < w; ++m) {
      for (int e = tid; e < (w - 1 - m) * cw; e += kCtaLuThreads) {
        const int i = m + 1 + e / cw, j = e % cw;
        Xs[i * LD + j] = X::sub(Xs[i * LD + j], X::mul(Ls[i * LD + m], Xs[m * LD + j]));
      }
      __syncthreads();
    }
    for (int e = tid; e < w * cw; e += kCtaLuThreads) {
      const int i = e / cw, j = e % cw;
      const F v = lu_store<F>(Xs[i * LD + j]);
      bad |= !isfinite((double)to_f(v));
      A[(size_t)(r0 + i) * lda + cb + j] = v;
    }
    __syncthreads();
  }
  if (__syncthreads_or(bad) && tid == 0) nonfinite = 1;
}

// C = A[r0+K.., c0..c1) <- fl_f(fl_T(C - L21 U12)), K = w products per
// element as an ascending fused multiply-add chain in T.  Tiles of 32 x 32
// elements, L21 and U12 staged in shared memory; thread t takes rows
// (t / 8) and columns 4 (t % 8) .. 4 (t % 8) + 3 of the tile.
template <typename F>
__device__ void cta_update(F* A, int lda, int n, int r0, int w, int c0, int c1, int& nonfinite,
                           LuT<F>* sm) {
  using T = LuT<F>;
  using X = TArith<T>;
  const int rb = r0 + w;
  if (c1 <= c0 || rb >= n) return;
  T* Ls = sm;               // 32 x 65
  T* Us = sm + 32 * 65;     // 64 x 33
  const int tid = threadIdx.x, tr = tid >> 3, tc = (tid & 7) * 4;
  int bad = 0;
  for (int i0 = rb; i0 < n; i0 += 32)
    for (int j0 = c0; j0 < c1; j0 += 32) {
      __syncthreads();  // the previous tile's operands are no longer read
      for (int e = tid; e < 32 * w; e += kCtaLuThreads) {
        const int i = e / w, k = e % w;
        Ls[i * 65 + k] = i0 + i < n ? (T)to_f(A[(size_t)(i0 + i) * lda + r0 + k]) : (T)0;
      }
      for (int e = tid; e < w * 32; e += kCtaLuThreads) {
        const int k = e / 32, j = e % 32;
        Us[k * 33 + j] = j0 + j < c1 ? (T)to_f(A[(size_t)(r0 + k) * lda + j0 + j]) : (T)0;
      }
      __syncthreads();
      const int i = i0 + tr;
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
      for (int k = 0; k < w; ++k) {
        const T l = Ls[tr * 65 + k];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = X::fma(l, Us[k * 33 + tc + q], acc[q]);
      }
      if (i < n) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = j0 + tc + q;
          if (j < c1) {
            F* pc = A + (size_t)i * lda + j;
            const F v = lu_store<F>(X::sub((T)to_f(*pc), acc[q]));
            bad |= !isfinite((double)to_f(v));
            *pc = v;
          }
        }
      }
    }
  if (__syncthreads_or(bad) && threadIdx.x == 0) nonfinite = 1;
}

// The whole factorisation.  ipiv: LAPACK-style global rows (0-based).
// info: 1-based first zero pivot (0: none); nonfinite: a stored value is
// Inf or NaN.  Every thread of the block calls it; smem holds
// cta_lu_smem<F>(nb) bytes.
template <typename F>
__device__ void cta_lu(F* A, int lda, int n, int nb, int nbo, int* ipiv, int* info_out, int* nonfinite_out,
                       unsigned char* smem) {
  using T = LuT<F>;
  __shared__ double s_val[kCtaLuThreads / 32];
  __shared__ int s_idx[kCtaLuThreads / 32];
  __shared__ int s_info, s_nonfinite;
  T* P = (T*)smem;
  if (threadIdx.x == 0) { s_info = 0; s_nonfinite = 0; }
  __syncthreads();
  int& info = s_info;
  int& nonfinite = s_nonfinite;
  for (int k = 0; k < n; k += nbo) {
    const int W = min(nbo, n - k);
    for (int kk = k; kk < k + W; kk += nb) {
      const int w = min(nb, k + W - kk);
      cta_panel<F>(A, lda, n, kk, w, ipiv, info, nonfinite, P, s_val, s_idx);
      __syncthreads();
      cta_swap_cols<F>(A, lda, ipiv, kk, w, k, kk);
      cta_swap_cols<F>(A, lda, ipiv, kk, w, kk + w, k + W);
      cta_trsm<F>(A, lda, kk, w, kk + w, k + W, nonfinite, P);
      __syncthreads();
      cta_update<F>(A, lda, n, kk, w, kk + w, k + W, nonfinite, P);
      __syncthreads();
    }
    cta_swap_cols<F>(A, lda, ipiv, k, W, 0, k);
    cta_swap_cols<F>(A, lda, ipiv, k, W, k + W, n);
    cta_trsm<F>(A, lda, k, W, k + W, n, nonfinite, P);
    __syncthreads();
    cta_update<F>(A, lda, n, k, W, k + W, n, nonfinite, P);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *info_out = s_info;
    *nonfinite_out = s_nonfinite;
  }
  __syncthreads();
}

}  // namespace msir
