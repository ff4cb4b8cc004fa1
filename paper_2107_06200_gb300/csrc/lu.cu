// Blocked right-looking GEPP in the factorisation precision u_f
// (Algorithm 4, first step; partial pivoting as in Sec. 1).
//
// The matrix lives in device memory in its storage format F (bf16, fp16,
// fp32 or fp64), row-major with leading dimension lda.  Arithmetic of the
// panel and of the triangular solves is carried out in T = fp32 (fp64 when
// F is fp64), with every product and every difference explicitly rounded,
// so those steps are bit-for-bit reproducible; values are rounded back to F
// when they are stored.  Two-level blocking: outer blocks of W = nbo
// columns, factored as panels of nb columns.
//
//   lu_outer_panel      one thread-block cluster factors an (n-k) x W outer
//                       block: for each nb-column panel, the pivot search,
//                       interchange, scaling and rank-1 updates run with the
//                       panel in shared memory; pivot candidates and the
//                       pivot row are pushed to every CTA of the cluster
//                       through distributed shared memory, so each column
//                       costs one cluster barrier.  The inner interchanges,
//                       substitution and update of the outer block follow.
//   lu_outer_swap_trsm  applies the outer block's interchanges to the other
//                       columns, forms U12 = L11^{-1} A12 by substitution and
//                       (for the tensor-core update) writes U12^T.
//   lu_update_simt      A22 <- fl_F(fl_T(A22 - L21 U12)) for fp32/fp64
//                       factors (the bf16/fp16 update is in lu_tc.cu).
#include <cooperative_groups.h>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace msir {

template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T sub_rn(T a, T b);
template <> __device__ __forceinline__ float sub_rn<float>(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ double sub_rn<double>(double a, double b) { return __dsub_rn(a, b); }
template <typename T> __device__ __forceinline__ T div_rn(T a, T b);
template <> __device__ __forceinline__ float div_rn<float>(float a, float b) { return __fdiv_rn(a, b); }
template <> __device__ __forceinline__ double div_rn<double>(double a, double b) { return __ddiv_rn(a, b); }
template <typename T> __device__ __forceinline__ T fma_rn(T a, T b, T c);
template <> __device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename F> __device__ __forceinline__ F store_rn(typename Fmt<F>::T v);
template <> __device__ __forceinline__ __half store_rn<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_rn<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ float store_rn<float>(float v) { return v; }
template <> __device__ __forceinline__ double store_rn<double>(double v) { return v; }

// Panel width limit per arithmetic precision (also the register arrays).
template <typename T> struct PanelNB { static constexpr int v = 32; };
template <> struct PanelNB<double> { static constexpr int v = 16; };

// Pivot order: larger |a| first; NaN (mapped to -1) only if nothing else;
// equal magnitudes -> smaller row index.  Compared in the panel's own
// arithmetic precision (fp64 instructions are scarce on this GPU).
template <typename T>
__device__ __forceinline__ bool better(T av, int ai, T bv, int bi) {
  return av > bv || (av == bv && ai < bi);
}
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(ov, oi, v, i)) { v = ov; i = oi; }
  }
}
// The same order for float by two warp reductions: v is -2 (no candidate),
// -1 (NaN) or a non-negative float, whose bits order like its values, so
// the key 0 / 1 / bits + 2 is monotone in v; the smallest index among the
// lanes holding the largest key wins.
__device__ __forceinline__ void warp_argmax(float& v, int& i) {
  const unsigned key = v == -2.f ? 0u : v == -1.f ? 1u : __float_as_uint(v) + 2u;
  const unsigned mk = __reduce_max_sync(0xffffffffu, key);
  i = __reduce_min_sync(0xffffffffu, key == mk ? i : INT_MAX);
  v = mk == 0u ? -2.f : mk == 1u ? -1.f : __uint_as_float(mk - 2u);
}

// ------------------------------------------------------------------ panel

// Optional section timers (rank 0, thread 0): 0 column loop, 1 cluster
// barrier of the column loop, 2 pivot search + push, 3 rank-1 update,
// 4 panel store + permutation maps, 5 inner interchanges + substitution,
// 6 inner update, 7 panel load.
// They add up in shared memory and reach a.tdbg once, at the kernel's end,
// so that the measurement keeps global-memory round trips off the loop.
#define PT_BEGIN(id) unsigned long long _t##id = (a.tdbg && rank == 0 && tid == 0) ? gtimer() : 0
#define PT_END(id) \
  if (a.tdbg && rank == 0 && tid == 0) s_tacc[id] += gtimer() - _t##id

template <typename F>
__global__ void __launch_bounds__(kPanelThreads, 1) lu_outer_panel(PanelArgs a) {
  using T = typename Fmt<F>::T;
  constexpr int NBM = PanelNB<T>::v;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kPanelThreads / 32;
  F* A = (F*)a.A;
  const int lda = a.lda, n = a.n, k = a.k, W = a.W, nb = a.nb;
  const int ldp = nb + 1;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = (T*)smem_raw;                                        // R_cap x ldp
  T* cand_row = P + (size_t)a.R_cap * ldp;                    // [2][16][NBM]
  T* jrow = cand_row + 2 * 16 * NBM;                          // [2][NBM]
  T* L11t = jrow + 2 * NBM;                                   // NBM x NBM, transposed
  T* U12 = L11t + NBM * NBM;                                  // NBM x W
  T* cand_v = U12 + (size_t)NBM * W;                          // [2][16]
  size_t off = sizeof(T) * ((size_t)a.R_cap * ldp + 2 * 16 * NBM + 2 * NBM + NBM * NBM +
                            (size_t)NBM * W + 32);
  off = (off + 7) & ~(size_t)7;
  int* cand_i = (int*)(smem_raw + off);                       // [2][16]
  int* s_piv = cand_i + 32;                                   // [NBM]
  int* mpos = s_piv + NBM;                                    // inner map positions [2*NBM]
  int* mval = mpos + 2 * NBM;                                 // inner map sources
  int* opos = mval + 2 * NBM;                                 // outer map (rank 0) [2*W]
  int* oval = opos + 2 * W;
  __shared__ T s_wv[NW];
  __shared__ int s_wi[NW];
  __shared__ int s_cnt, s_ocnt, s_nf;
  __shared__ unsigned long long s_tacc[8];

  if (tid == 0) { s_ocnt = W; s_nf = 0; }
  if (tid < 8) s_tacc[tid] = 0;
  for (int s = tid; s < W; s += blockDim.x) { opos[s] = s; oval[s] = s; }
  __syncthreads();

  for (int kk = k; kk < k + W; kk += nb) {
    const int w = min(nb, k + W - kk);
    const int m = n - kk;
    const int R = (m + C - 1) / C;
    const int my0 = rank * R;
    const int nloc = max(0, min(m, my0 + R) - my0);

    PT_BEGIN(7);
    for (int li = tid; li < nloc; li += blockDim.x) {
      const F* src = A + (size_t)(kk + my0 + li) * lda + kk;
      F v[NBM];
#pragma unroll
      for (int c = 0; c < NBM; ++c) v[c] = c < w ? src[c] : F(0);
#pragma unroll
      for (int c = 0; c < NBM; ++c)
        if (c < w) P[li * ldp + c] = (T)to_f(v[c]);
    }
    __syncthreads();
    PT_END(7);

    PT_BEGIN(0);
    for (int j = 0; j < w; ++j) {
      const int buf = j & 1;
      PT_BEGIN(2);
      // local pivot candidate among my rows with panel index >= j
      T bv = (T)-2;
      int bi = INT_MAX;
      for (int li = tid; li < nloc; li += blockDim.x) {
        const int gi = my0 + li;
        if (gi >= j) {
          T av = fabs(P[li * ldp + j]);
          if (isnan(av)) av = (T)-1;
          if (better(av, gi, bv, bi)) { bv = av; bi = gi; }
        }
      }
      warp_argmax(bv, bi);
      if (lane == 0) { s_wv[warp] = bv; s_wi[warp] = bi; }
      __syncthreads();
      const int ownj = j / R;
      if (warp == 0) {
        T v = lane < NW ? s_wv[lane] : (T)-2;
        int i = lane < NW ? s_wi[lane] : INT_MAX;
        warp_argmax(v, i);
        // push (value, index) and the candidate row to every CTA
        if (lane < C) {
          cl.map_shared_rank(cand_v, lane)[buf * 16 + rank] = v;
          cl.map_shared_rank(cand_i, lane)[buf * 16 + rank] = i;
        }
        // lane c sends column c of the candidate row (w <= 32)
        if (lane < w) {
          const T val = i != INT_MAX ? P[(i - my0) * ldp + lane] : (T)0;
          for (int d = 0; d < C; ++d) cl.map_shared_rank(cand_row, d)[(buf * 16 + rank) * NBM + lane] = val;
        }
      } else if (warp == 1 && ownj == rank) {
        if (lane < w) {
          const T val = P[(j - my0) * ldp + lane];
          for (int d = 0; d < C; ++d) cl.map_shared_rank(jrow, d)[buf * NBM + lane] = val;
        }
      }
      PT_END(2);
      PT_BEGIN(1);
      cl.sync();
      PT_END(1);
      // every warp reduces the C candidates (lane q reads rank q's)
      T pv = lane < C ? cand_v[buf * 16 + lane] : (T)-2;
      int p = lane < C ? cand_i[buf * 16 + lane] : INT_MAX;
      warp_argmax(pv, p);
      const int ownp = p / R;
      const T* prow = cand_row + (buf * 16 + ownp) * NBM;
      const T* jr = jrow + buf * NBM;
      if (tid < w) {
        if (ownj == rank) P[(j - my0) * ldp + tid] = prow[tid];
        if (p != j && ownp == rank) P[(p - my0) * ldp + tid] = jr[tid];
      }
      if (tid == 0) s_piv[j] = p;
      __syncthreads();
      PT_BEGIN(3);
      const T piv = prow[j];
      if (piv != (T)0) {
        // pivot row and each updated row staged in registers, so that the
        // loads of a row are not ordered behind its stores.  Columns go in
        // chunks of 8: a chunk left of column j+1 is skipped (a uniform
        // branch), one right of it runs unpredicated.
        for (int li = tid; li < nloc; li += blockDim.x) {
          const int gi = my0 + li;
          if (gi > j) {
            T* row = P + li * ldp;
            const T l = div_rn(row[j], piv);
            if (w == NBM) {
#pragma unroll
              for (int c0 = 0; c0 < NBM; c0 += 8) {
                if (c0 + 7 <= j) continue;
                T rv[8], pv[8];
                if (c0 > j) {
#pragma unroll
                  for (int q = 0; q < 8; ++q) {
                    rv[q] = row[c0 + q];
                    pv[q] = prow[c0 + q];
                  }
#pragma unroll
                  for (int q = 0; q < 8; ++q) rv[q] = sub_rn(rv[q], mul_rn(l, pv[q]));
#pragma unroll
                  for (int q = 0; q < 8; ++q) row[c0 + q] = rv[q];
                } else {
#pragma unroll
                  for (int q = 0; q < 8; ++q)
                    if (c0 + q > j) {
                      rv[q] = row[c0 + q];
                      pv[q] = prow[c0 + q];
                    }
#pragma unroll
                  for (int q = 0; q < 8; ++q)
                    if (c0 + q > j) rv[q] = sub_rn(rv[q], mul_rn(l, pv[q]));
#pragma unroll
                  for (int q = 0; q < 8; ++q)
                    if (c0 + q > j) row[c0 + q] = rv[q];
                }
              }
            } else {
              T rv[NBM];
#pragma unroll
              for (int c = 1; c < NBM; ++c)
                if (c > j && c < w) rv[c] = row[c];
#pragma unroll
              for (int c = 1; c < NBM; ++c)
                if (c > j && c < w) rv[c] = sub_rn(rv[c], mul_rn(l, prow[c]));
#pragma unroll
              for (int c = 1; c < NBM; ++c)
                if (c > j && c < w) row[c] = rv[c];
            }
            row[j] = l;
          }
        }
      } else if (rank == 0 && tid == 0) {
        atomicCAS(a.info, 0, kk + j + 1);
      }
      // no barrier here: the next column's scan reads only this thread's own
      // rows, its pushes read rows after the next barrier, and the candidate
      // buffers alternate, so a slower thread's update never meets them
      PT_END(3);
    }
    __syncthreads();
    PT_END(0);

    // round the panel to F in place, store it, and record its pivots
    PT_BEGIN(4);
    int nf = 0;
    // full-width panels are written with 16-byte stores (a row segment of
    // NBM values starts on a 16-byte boundary: kk is a multiple of nb and
    // lda of 64); the last, narrower panel of a block element by element
    constexpr int kPer16 = 16 / (int)sizeof(F);
    for (int li = tid; li < nloc; li += blockDim.x) {
      F* dst = A + (size_t)(kk + my0 + li) * lda + kk;
      if (w == NBM) {
#pragma unroll
        for (int c0 = 0; c0 < NBM; c0 += kPer16) {
          unsigned char bytes[16];
#pragma unroll
          for (int q = 0; q < kPer16; ++q) {
            const F v = store_rn<F>(P[li * ldp + c0 + q]);
            memcpy(bytes + q * sizeof(F), &v, sizeof(F));
            P[li * ldp + c0 + q] = (T)to_f(v);
            if (!isfinite(to_f(v))) nf = 1;
          }
          uint4 pk;
          memcpy(&pk, bytes, 16);
          *reinterpret_cast<uint4*>(dst + c0) = pk;
        }
      } else {
        for (int c = 0; c < w; ++c) {
          const F v = store_rn<F>(P[li * ldp + c]);
          dst[c] = v;
          P[li * ldp + c] = (T)to_f(v);
          if (!isfinite(to_f(v))) nf = 1;
        }
      }
    }
    if (nf) s_nf = 1;
    if (rank == 0 && tid < w) a.ipiv[kk + tid] = kk + s_piv[tid];

    // composite permutation of this panel's interchanges (positions
    // relative to kk; positions < w are slots 0..w-1), and of the outer
    // block's (relative to k, kept by rank 0).  Built by warp 0.
    if (warp == 0) {
      if (lane == 0) s_cnt = w;
      for (int s = lane; s < 2 * NBM; s += 32) { mpos[s] = s < w ? s : -1; mval[s] = s < w ? s : -1; }
      __syncwarp();
      for (int j = 0; j < w; ++j) {
        const int q = s_piv[j];
        int sq;
        if (q < w) {
          sq = q;
        } else {
          const int cnt = s_cnt;
          unsigned hit = __ballot_sync(0xffffffffu, lane + w < cnt && mpos[lane + w] == q);
          if (hit) {
            sq = w + __ffs(hit) - 1;
          } else {
            sq = cnt;
            if (lane == 0) { mpos[cnt] = q; mval[cnt] = q; s_cnt = cnt + 1; }
          }
          __syncwarp();
        }
        if (lane == 0 && sq != j) {
          const int t = mval[j];
          mval[j] = mval[sq];
          mval[sq] = t;
        }
        __syncwarp();
      }
    } else if (warp == 1 && rank == 0) {
      // the outer block's map, built beside warp 0's inner map
      {
        const int base = kk - k;
        for (int j = 0; j < w; ++j) {
          const int pa = base + j, pb = base + s_piv[j];
          int sb;
          if (pb < W) {
            sb = pb;
          } else {
            const int cnt = s_ocnt;
            int found = -1;
            for (int s0 = W; s0 < cnt; s0 += 32) {
              unsigned hit = __ballot_sync(0xffffffffu, s0 + lane < cnt && opos[s0 + lane] == pb);
              if (hit) { found = s0 + __ffs(hit) - 1; break; }
            }
            if (found < 0) {
              found = cnt;
              if (lane == 0) { opos[cnt] = pb; oval[cnt] = pb; s_ocnt = cnt + 1; }
            }
            sb = found;
            __syncwarp();
          }
          if (lane == 0 && sb != pa) {
            const int t = oval[pa];
            oval[pa] = oval[sb];
            oval[sb] = t;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    cl.sync();  // panel values visible to the whole cluster
    PT_END(4);
    PT_BEGIN(5);

    // inner interchanges on [k, kk) and [kk+w, k+W), then U12 = L11^{-1} A12
    // for [kk+w, k+W): one warp per column
    const int nleft = kk - k, nright = k + W - kk - w;
    if (nright > 0) {
      for (int idx = tid; idx < w * w; idx += blockDim.x) {
        const int i = idx / w, c = idx % w;  // L11t[c][i] = L[i][c]
        L11t[c * NBM + i] = (T)to_f(A[(size_t)(kk + i) * lda + kk + c]);
      }
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int g = rank * NW + warp; g < nleft + nright; g += C * NW) {
      const int c = g < nleft ? k + g : kk + w + (g - nleft);
      // slots lane and lane + 32
      T v0 = (T)0, v1 = (T)0;
      if (lane < cnt) v0 = (T)to_f(A[(size_t)(kk + mval[lane]) * lda + c]);
      if (lane + 32 < cnt) v1 = (T)to_f(A[(size_t)(kk + mval[lane + 32]) * lda + c]);
      __syncwarp();
      if (lane >= w && lane < cnt) A[(size_t)(kk + mpos[lane]) * lda + c] = store_rn<F>(v0);
      if (lane + 32 >= w && lane + 32 < cnt) A[(size_t)(kk + mpos[lane + 32]) * lda + c] = store_rn<F>(v1);
      if (g < nleft) {
        if (lane < w) A[(size_t)(kk + lane) * lda + c] = store_rn<F>(v0);
      } else {
        T x = v0;  // row `lane` of the column
        for (int mm = 0; mm < w - 1; ++mm) {
          const T xm = __shfl_sync(0xffffffffu, x, mm);
          if (lane > mm && lane < w) x = sub_rn(x, mul_rn(L11t[mm * NBM + lane], xm));
        }
        if (lane < w) {
          const F v = store_rn<F>(x);
          A[(size_t)(kk + lane) * lda + c] = v;
          if (!isfinite(to_f(v))) s_nf = 1;
        }
      }
    }
    cl.sync();
    PT_END(5);
    PT_BEGIN(6);

    // inner update of my panel rows below the diagonal block:
    // A[kk+gi][kk+w+c] <- fl(A - sum_mm L[gi][mm] U12[mm][c]), L from P, the
    // sum an ascending fused multiply-add chain from zero per element.
    // Register tiles of 4 rows x CW columns per thread (CW = 4, or 2 for
    // fp64; a warp covers 8 CW rows x 16 columns): 4 + CW shared-memory
    // loads per 4 CW multiply-adds.
    if (nright > 0) {
      for (int idx = tid; idx < w * nright; idx += blockDim.x) {
        const int i = idx / nright, c = idx % nright;
        U12[i * W + c] = (T)to_f(A[(size_t)(kk + i) * lda + kk + w + c]);
      }
      __syncthreads();
      const int lfirst = max(0, w - my0);  // first local row with gi >= w
      const int nrow = nloc - lfirst;
      constexpr int CW = sizeof(T) == 8 ? 2 : 4;
      constexpr int CG = 16 / CW;              // column groups of a warp
      constexpr int WR = 32 / CG * 4;          // rows of a warp tile
      const int tiles_r = (nrow + WR - 1) / WR, tiles_c = (nright + 15) / 16;
      const int ri = lane / CG, ci = lane % CG;
      for (int t = warp; t < tiles_r * tiles_c; t += NW) {
        const int r0 = lfirst + (t / tiles_c) * WR + ri * 4;
        const int c0 = (t % tiles_c) * 16 + ci * CW;
        int lr[4], uc[CW];
#pragma unroll
        for (int r = 0; r < 4; ++r) lr[r] = min(r0 + r, nloc - 1) * ldp;  // rows past nloc: not stored
#pragma unroll
        for (int q = 0; q < CW; ++q) uc[q] = min(c0 + q, nright - 1);     // columns past nright: not stored
        T acc[4][CW];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < CW; ++q) acc[r][q] = (T)0;
#pragma unroll 4
        for (int mm = 0; mm < w; ++mm) {
          T l[4], u[CW];
#pragma unroll
          for (int r = 0; r < 4; ++r) l[r] = P[lr[r] + mm];
#pragma unroll
          for (int q = 0; q < CW; ++q) u[q] = U12[mm * W + uc[q]];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < CW; ++q) acc[r][q] = fma_rn(l[r], u[q], acc[r][q]);
        }
        // C read and written as one CW-value vector per row (8 or 16 bytes)
        // when kk + w is a multiple of CW (rows start on 128-byte boundaries
        // and c0 is a multiple of CW, so the vector is then aligned)
        using Vec = typename std::conditional<sizeof(F) * CW == 8, uint2, uint4>::type;
        const bool vec_ok = ((kk + w) % CW) == 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (r0 + r >= nloc) continue;
          F* dst = A + (size_t)(kk + my0 + r0 + r) * lda + kk + w + c0;
          if (vec_ok && c0 + CW <= nright) {
            Vec raw = *reinterpret_cast<const Vec*>(dst);
            F* e = reinterpret_cast<F*>(&raw);
#pragma unroll
            for (int q = 0; q < CW; ++q) e[q] = store_rn<F>(sub_rn((T)to_f(e[q]), acc[r][q]));
            *reinterpret_cast<Vec*>(dst) = raw;
          } else {
#pragma unroll
            for (int q = 0; q < CW; ++q)
              if (c0 + q < nright) dst[q] = store_rn<F>(sub_rn((T)to_f(dst[q]), acc[r][q]));
          }
        }
      }
    }
    cl.sync();
    PT_END(6);
  }

  if (s_nf) atomicExch(a.nonfinite, 1);
  if (a.tdbg && rank == 0 && tid < 8) a.tdbg[tid] += s_tacc[tid];
  if (rank == 0) {
    const int oc = s_ocnt;
    for (int s = tid; s < oc; s += blockDim.x) {
      a.map_pos[s] = opos[s];
      a.map_val[s] = oval[s];
    }
    if (tid == 0) *a.map_cnt = oc;
  }
}

// ------------------------------------------------- outer swaps and TRSM

template <typename F>
__global__ void __launch_bounds__(256) lu_outer_swap_trsm(SwapTrsmArgs a) {
  using T = typename Fmt<F>::T;
  F* A = (F*)a.A;
  const int lda = a.lda, k = a.k, W = a.W;
  const int cnt = *a.map_cnt;
  const int nleft = a.do_left ? k : 0, nright = a.c_end - a.c_begin;
  const int tiles_left = (nleft + 31) / 32;
  const int tiles_right = nright > 0 ? (nright + 31) / 32 : 0;
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldL = W + (sizeof(F) == 2 ? 2 : 1);  // padded: rows of L fall in different banks
  T* X = (T*)smem_raw;                       // W x 32
  F* L = (F*)(X + (size_t)W * 32);           // W x ldL (only when right tiles exist)
  F* E = L + (size_t)W * ldL;                // (cnt - W) x 32 displaced rows
  size_t off = sizeof(T) * (size_t)W * 32 + sizeof(F) * ((size_t)W * ldL + (size_t)W * 32);
  off = (off + 15) & ~(size_t)15;
  int* pos = (int*)(smem_raw + off);
  int* val = pos + 2 * W;
  __shared__ int s_nf;
  if (tid == 0) s_nf = 0;
  for (int s = tid; s < cnt; s += blockDim.x) { pos[s] = a.map_pos[s]; val[s] = a.map_val[s]; }
  bool need_L = false;
  for (int t = blockIdx.x; t < tiles_left + tiles_right; t += gridDim.x)
    if (t >= tiles_left) need_L = true;
  if (need_L) {
    for (int idx = tid; idx < W * W; idx += blockDim.x) {
      const int i = idx / W, c = idx % W;
      L[i * ldL + c] = A[(size_t)(k + i) * lda + k + c];
    }
  }
  __syncthreads();

  for (int t = blockIdx.x; t < tiles_left + tiles_right; t += gridDim.x) {
    const bool right = t >= tiles_left;
    const int c0 = right ? a.c_begin + (t - tiles_left) * 32 : t * 32;
    const int cend = right ? a.c_end : k;
    // gather sources
    for (int idx = tid; idx < cnt * 32; idx += blockDim.x) {
      const int s = idx / 32, cc = idx % 32, c = c0 + cc;
      if (c < cend) {
        F v = A[(size_t)(k + val[s]) * lda + c];
        if (s < W) X[s * 32 + cc] = (T)to_f(v);
        else E[(s - W) * 32 + cc] = v;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < (cnt - W) * 32; idx += blockDim.x) {
      const int s = W + idx / 32, cc = idx % 32, c = c0 + cc;
      if (c < cend) A[(size_t)(k + pos[s]) * lda + c] = E[(s - W) * 32 + cc];
    }
    if (right) {
      for (int mm = 0; mm < W - 1; ++mm) {
        const int rows = W - 1 - mm;
        for (int idx = tid; idx < rows * 32; idx += blockDim.x) {
          const int i = mm + 1 + idx / 32, cc = idx % 32;
          X[i * 32 + cc] = sub_rn(X[i * 32 + cc], mul_rn((T)to_f(L[i * ldL + mm]), X[mm * 32 + cc]));
        }
        __syncthreads();
      }
    }
    int nf = 0;
    for (int idx = tid; idx < W * 32; idx += blockDim.x) {
      const int s = idx / 32, cc = idx % 32, c = c0 + cc;
      if (c < cend) {
        F v = store_rn<F>(X[s * 32 + cc]);
        A[(size_t)(k + s) * lda + c] = v;
        if (right && !isfinite(to_f(v))) nf = 1;
      }
    }
    if (right && a.Ut != nullptr) {
      F* Ut = (F*)a.Ut;
      for (int idx = tid; idx < W * 32; idx += blockDim.x) {
        const int cc = idx / W, s = idx % W, c = c0 + cc;
        if (c < cend) Ut[(size_t)(c - k - W) * a.ldut + s] = store_rn<F>(X[s * 32 + cc]);
      }
    }
    if (nf) s_nf = 1;
    __syncthreads();
  }
  if (s_nf) atomicExch(a.nonfinite, 1);
}

// ------------------------------------------------------- SIMT update

template <typename F>
__global__ void __launch_bounds__(256) lu_update_simt(UpdateArgs a) {
  using T = typename Fmt<F>::T;
  F* A = (F*)a.A;
  const int lda = a.lda, k = a.k, W = a.W;
  const int r0 = k + W, M = a.n - r0;
  const int c0 = a.c_begin, NC = a.c_end - a.c_begin;
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tm = blockIdx.y * BM, tn = blockIdx.x * BN;
  const int ty = tid / 16, tx = tid % 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int kc = 0; kc < W; kc += BK) {
    for (int idx = tid; idx < BM * BK; idx += 256) {
      const int i = idx / BK, kq = idx % BK;
      const int row = tm + i, kk = kc + kq;
      As[kq][i] = (row < M && kk < W) ? (T)to_f(A[(size_t)(r0 + row) * lda + k + kk]) : (T)0;
    }
    for (int idx = tid; idx < BK * BN; idx += 256) {
      const int kq = idx / BN, j = idx % BN;
      const int col = tn + j, kk = kc + kq;
      Bs[kq][j] = (col < NC && kk < W) ? (T)to_f(A[(size_t)(k + kk) * lda + c0 + col]) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < BK; ++kq) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kq][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kq][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma_rn(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = tm + ty * 4 + i;
    if (row >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = tn + tx * 4 + j;
      if (col >= NC) continue;
      F* p = A + (size_t)(r0 + row) * lda + c0 + col;
      *p = store_rn<F>(sub_rn((T)to_f(*p), acc[i][j]));
    }
  }
}

// ------------------------------------------------------------ launchers

size_t panel_smem_bytes(int fmt, int R_cap, int nb, int W) {
  const size_t ts = fmt == MSIR_FP64 ? 8 : 4;
  const int NBM = fmt == MSIR_FP64 ? 16 : 32;
  size_t b = ts * ((size_t)R_cap * (nb + 1) + 2 * 16 * NBM + 2 * NBM + NBM * NBM + (size_t)NBM * W + 32);
  b = (b + 7) & ~(size_t)7;
  b += 32 * sizeof(int) + NBM * sizeof(int) + 4 * NBM * sizeof(int) + 4 * (size_t)W * sizeof(int);
  return b;
}

size_t swap_trsm_smem_bytes(int fmt, int W) {
  const size_t ts = fmt == MSIR_FP64 ? 8 : 4;
  const size_t fs = fmt == MSIR_FP64 ? 8 : fmt == MSIR_FP32 ? 4 : 2;
  const size_t ldL = W + (fs == 2 ? 2 : 1);
  size_t off = ts * (size_t)W * 32 + fs * ((size_t)W * ldL + (size_t)W * 32);
  off = (off + 15) & ~(size_t)15;
  return off + 4 * (size_t)W * sizeof(int);
}

template <typename F>
static cudaError_t launch_panel_t(const PanelArgs& a, int C, cudaStream_t st) {
  size_t smem = panel_smem_bytes(Fmt<F>::code, a.R_cap, a.nb, a.W);
  cudaError_t e = cudaFuncSetAttribute(lu_outer_panel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(lu_outer_panel<F>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lu_outer_panel<F>, a);
}

cudaError_t launch_panel(int fmt, const PanelArgs& a, int C, cudaStream_t st) {
  switch (fmt) {
    case MSIR_FP16: return launch_panel_t<__half>(a, C, st);
    case MSIR_BF16: return launch_panel_t<__nv_bfloat16>(a, C, st);
    case MSIR_FP32: return launch_panel_t<float>(a, C, st);
    case MSIR_FP64: return launch_panel_t<double>(a, C, st);
  }
  return cudaErrorInvalidValue;
}

template <typename F>
static cudaError_t launch_swap_trsm_t(const SwapTrsmArgs& a, int grid, cudaStream_t st) {
  size_t smem = swap_trsm_smem_bytes(Fmt<F>::code, a.W);
  cudaError_t e = cudaFuncSetAttribute(lu_outer_swap_trsm<F>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lu_outer_swap_trsm<F><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_swap_trsm(int fmt, const SwapTrsmArgs& a, int grid, cudaStream_t st) {
  switch (fmt) {
    case MSIR_FP16: return launch_swap_trsm_t<__half>(a, grid, st);
    case MSIR_BF16: return launch_swap_trsm_t<__nv_bfloat16>(a, grid, st);
    case MSIR_FP32: return launch_swap_trsm_t<float>(a, grid, st);
    case MSIR_FP64: return launch_swap_trsm_t<double>(a, grid, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_update_simt(int fmt, const UpdateArgs& a, cudaStream_t st) {
  const int M = a.n - a.k - a.W, NC = a.c_end - a.c_begin;
  if (M <= 0 || NC <= 0) return cudaSuccess;
  dim3 grid((NC + 63) / 64, (M + 63) / 64);
  switch (fmt) {
    case MSIR_FP16: lu_update_simt<__half><<<grid, 256, 0, st>>>(a); break;
    case MSIR_BF16: lu_update_simt<__nv_bfloat16><<<grid, 256, 0, st>>>(a); break;
    case MSIR_FP32: lu_update_simt<float><<<grid, 256, 0, st>>>(a); break;
    case MSIR_FP64: lu_update_simt<double><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace msir
