// The batched engine: one persistent launch solves a whole batch of small
// systems (n <= kBatchMaxN).  Each thread block takes the next system from
// a work counter and runs all of Algorithm 4 on it alone: ingest
// (A_u = fl_u0(A), b_u, norms), the LU in u_f (lu_cta.cuh), the factor
// check with the squeezed retry (Sec. 2.1.2), the inverses of the diagonal
// blocks, and the refinement (refine_msir with a grid of one block: the
// same SIR / SGMRES-IR / GMRES-IR steps, stopping logic and substitutions
// as the single-system kernel).  When a stage asks for a finer u_f
// (Algorithm 4's escalation) the block refactors at the next precision and
// goes on, without returning to the host; the stage machines of the
// systems diverge freely.  Every device wait is bounded as in the
// single-system kernel.
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "batched.h"
#include "inv_impl.cuh"
#include "lu_cta.cuh"
#include "refine_impl.cuh"

namespace msir {

constexpr int kBatchThreads = kRefThreads;
static_assert(kBatchThreads == kCtaLuThreads && kBatchThreads == kInvThreads, "one block shape");

__device__ __forceinline__ int next_uf_d(int f) {
  if (f == MSIR_BF16 || f == MSIR_FP16) return MSIR_FP32;
  if (f == MSIR_FP32) return MSIR_FP64;
  return 0;
}
__device__ __forceinline__ int level_of(int f) {
  if (f == MSIR_FP16 || f == MSIR_BF16) return 0;
  return f == MSIR_FP32 ? 1 : 2;
}

// The per-format device functions are kept out of line: the kernel calls
// each through one switch instead of inlining four copies.  The refinement
// reads the factor format at run time (FAny): one instantiation.
template <typename A0>
__device__ __noinline__ bool batch_refine(Cx& cx, const RefineArgs& a, RefState& S, unsigned char* gsm,
                                          int& s_act, int& s_reset, int& s_alg) {
  return refine_msir<A0, FAny>(cx, a, S, gsm, s_act, s_reset, s_alg);
}
template <typename F>
__device__ __noinline__ void batch_lu(void* A, int lda, int n, int nb, int nbo, int* ipiv, int* info,
                                      int* nonfinite, unsigned char* smem) {
  cta_lu<F>((F*)A, lda, n, nb, nbo, ipiv, info, nonfinite, smem);
}
template <typename F>
__device__ __noinline__ void batch_inv(const void* LU, int ldf, int n, float* inv32, double* inv_hi,
                                       double* inv_lo, unsigned char* smem) {
  const int nblk = (n + kIB - 1) / kIB;
  for (int q = 0; q < 2 * nblk; ++q) {
    inv_diag_block<F>((const F*)LU, ldf, n, nblk, q % nblk, q < nblk, inv32, inv_hi, inv_lo, (double*)smem);
    __syncthreads();
  }
}

__device__ __forceinline__ void batch_lu_fmt(int fmt, void* A, int lda, int n, int nb, int nbo, int* ipiv,
                                             int* info, int* nonfinite, unsigned char* smem) {
  switch (fmt) {
    case MSIR_FP16: batch_lu<__half>(A, lda, n, nb, nbo, ipiv, info, nonfinite, smem); break;
    case MSIR_BF16: batch_lu<__nv_bfloat16>(A, lda, n, nb, nbo, ipiv, info, nonfinite, smem); break;
    case MSIR_FP32: batch_lu<float>(A, lda, n, nb, nbo, ipiv, info, nonfinite, smem); break;
    default: batch_lu<double>(A, lda, n, nb, nbo, ipiv, info, nonfinite, smem); break;
  }
}
__device__ __forceinline__ void batch_inv_fmt(int fmt, const void* LU, int ldf, int n, float* inv32,
                                              double* inv_hi, double* inv_lo, unsigned char* smem) {
  switch (fmt) {
    case MSIR_FP16: batch_inv<__half>(LU, ldf, n, inv32, inv_hi, inv_lo, smem); break;
    case MSIR_BF16: batch_inv<__nv_bfloat16>(LU, ldf, n, inv32, inv_hi, inv_lo, smem); break;
    case MSIR_FP32: batch_inv<float>(LU, ldf, n, inv32, inv_hi, inv_lo, smem); break;
    default: batch_inv<double>(LU, ldf, n, inv32, inv_hi, inv_lo, smem); break;
  }
}

// A_f = fl_f(A_u), or fl_f(mu R_i a_ij S_j) when squeezed (the same
// product order as the single-system path)
template <typename A0>
__device__ void batch_make_factor(int fmt, const A0* Au, int ldu, int n, void* Af, const double* R,
                                  const double* S, double mu) {
  for (int e = threadIdx.x; e < n * n; e += kBatchThreads) {
    const int i = e / n, j = e % n;
    double v = (double)Au[(size_t)i * ldu + j];
    if (R) v = v * R[i] * S[j] * mu;
    const size_t o = (size_t)i * ldu + j;
    switch (fmt) {
      case MSIR_FP16: ((__half*)Af)[o] = from_d<__half>(v); break;
      case MSIR_BF16: ((__nv_bfloat16*)Af)[o] = from_d<__nv_bfloat16>(v); break;
      case MSIR_FP32: ((float*)Af)[o] = from_d<float>(v); break;
      default: ((double*)Af)[o] = v; break;
    }
  }
  __syncthreads();
}

// scale = 2^-e where m = f 2^e, f in [1/2, 1) (1 for m == 0 or non-finite)
__device__ __forceinline__ double batch_pow2_inv(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 1.0;
  int e;
  frexp(m, &e);
  return ldexp(1.0, -e);
}

// Squeezing scalings (Sec. 2.1.2's cited two-sided scaling): R_i from the
// row maxima of |A_u|, S_j from the column maxima of |R A_u|.
template <typename A0>
__device__ void batch_squeeze(const A0* Au, int ldu, int n, double* R, double* S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < n; i += kBatchThreads / 32) {
    double m = 0.0;
    for (int j = lane; j < n; j += 32) m = nanmax(m, fabs((double)Au[(size_t)i * ldu + j]));
    m = warp_nanmax_d(m);
    if (lane == 0) R[i] = batch_pow2_inv(m);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kBatchThreads) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = nanmax(m, fabs((double)Au[(size_t)i * ldu + j] * R[i]));
    S[j] = batch_pow2_inv(m);
  }
  __syncthreads();
}

// permutation of a LAPACK-style ipiv: (P A)[i] = A[perm[i]]
static __device__ void batch_perm(const int* ipiv, int n, int* perm) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int j = 0; j < n; ++j) {
      const int p = ipiv[j];
      if (p != j) {
        const int t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double batch_mu(const BatchArgs& B, int fmt) {
  return fmt == MSIR_FP16 ? B.mu_half : (fmt == MSIR_BF16 ? B.mu_bf16 : B.mu_single);
}

template <typename A0>
__global__ void __launch_bounds__(kBatchThreads, 1) batched_solve_kernel(BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* gsm = smem_raw + kTrsvSmem + kScaledSmem + kInboxSmem;
  __shared__ RefState S;
  __shared__ int s_act, s_reset, s_alg, s_task, s_info, s_nonfinite;
  __shared__ double s_w[kBatchThreads / 32];
  const BatchLayout& L = B.layout;
  char* ws = B.ws + (size_t)blockIdx.x * L.bytes;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // substitution epochs keep growing over the block's systems, so hand-off
  // words of an earlier system never match; the words start at zero
  unsigned epoch = 0;
  {
    unsigned long long* ll = (unsigned long long*)(ws + L.ll);
    const size_t nll = (size_t)4 * ((L.nmax + kBlk - 1) / kBlk) * kBlk * kLLWords;
    for (size_t e = threadIdx.x; e < nll; e += kBatchThreads) ll[e] = 0ull;
  }
  int* iflags = (int*)(ws + L.iflags);
  A0* Au = (A0*)(ws + L.Au);
  double* b_u = (double*)(ws + L.b_u);
  double* rowsum = (double*)(ws + L.rowsum);
  while (true) {
    if (tid == 0) s_task = (int)atomicAdd(B.next, 1u);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= B.count) break;
    const BatchTask T = B.tasks[t];
    const int n = T.n, ldu = L.ldu, u0 = T.u;
    // ---- ingest: A_u = fl_u0(A) row-major, b_u, norms
    for (int e = tid; e < n * n; e += kBatchThreads) {
      const int j = e / n, i = e % n;  // column-major reads, coalesced
      Au[(size_t)i * ldu + j] = (A0)T.A[(size_t)j * n + i];
    }
    for (int i = tid; i < n; i += kBatchThreads) b_u[i] = round_to(T.b[i], u0);
    if (tid < 32) iflags[tid] = 0;
    __syncthreads();
    for (int i = warp; i < n; i += kBatchThreads / 32) {
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s = __dadd_rn(s, fabs((double)Au[(size_t)i * ldu + j]));
      s = warp_sum_d(s);
      if (lane == 0) rowsum[i] = s;
    }
    __syncthreads();
    double ma = 0.0, mb = 0.0;
    for (int i = tid; i < n; i += kBatchThreads) {
      ma = nanmax(ma, rowsum[i]);
      mb = nanmax(mb, fabs(b_u[i]));
    }
    ma = warp_nanmax_d(ma);
    mb = warp_nanmax_d(mb);
    if (lane == 0) s_w[warp] = ma;
    __syncthreads();
    double normA = 0.0;
    for (int w = 0; w < kBatchThreads / 32; ++w) normA = nanmax(normA, s_w[w]);
    __syncthreads();
    if (lane == 0) s_w[warp] = mb;
    __syncthreads();
    double normb = 0.0;
    for (int w = 0; w < kBatchThreads / 32; ++w) normb = nanmax(normb, s_w[w]);
    __syncthreads();
    // ---- controller state and report
    msir_report* rep = B.reps + t;
    for (int e = tid; e < (int)(sizeof(msir_report) / 4); e += kBatchThreads) ((int*)rep)[e] = 0;
    if (tid == 0) {
      memset(&S, 0, sizeof(S));
      S.phase = PH_START;
      S.uf = T.uf;
      S.u = T.u;
      S.ur = T.ur;
      S.delta_prev = __longlong_as_double(0x7ff0000000000000ll);
      S.epoch = epoch;
    }
    __syncthreads();
    // ---- the arguments of refine_msir for this system (grid of one block)
    RefineArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = MODE_SOLVE;
    a.n = n;
    a.a_fmt = u0;
    a.A = Au;
    a.lda = ldu;
    a.b = b_u;
    a.ldf = ldu;
    a.normA = normA;
    a.normb = normb;
    a.x = (double*)(ws + L.x); a.xn = (double*)(ws + L.xn); a.x0 = (double*)(ws + L.x0);
    a.xbest = (double*)(ws + L.xbest);
    a.r_hi = (double*)(ws + L.r_hi); a.r_lo = (double*)(ws + L.r_lo);
    a.c_hi = (double*)(ws + L.c_hi); a.c_lo = (double*)(ws + L.c_lo);
    a.y_hi = (double*)(ws + L.y_hi); a.y_lo = (double*)(ws + L.y_lo);
    a.z_hi = (double*)(ws + L.z_hi); a.z_lo = (double*)(ws + L.z_lo);
    a.d = (double*)(ws + L.d); a.w = (double*)(ws + L.w); a.vk = (double*)(ws + L.vk);
    a.V = (double*)(ws + L.V); a.ldv = L.ldv;
    a.H = (double*)(ws + L.H); a.yv = (double*)(ws + L.yv);
    a.red = (double*)(ws + L.red); a.hred = (double*)(ws + L.hred); a.hvec = (double*)(ws + L.hvec);
    a.ll = (unsigned long long*)(ws + L.ll);
    a.M32 = (float*)(ws + L.M32); a.M64 = (double*)(ws + L.M64);
    a.Mdh = (double*)(ws + L.Mdh); a.Mdl = (double*)(ws + L.Mdl);
    a.bar = (unsigned*)(ws + L.bar);
    a.err = iflags + 2;
    a.rep = rep;
    a.i_max = B.i_max;
    a.rho_thresh = B.rho_thresh;
    a.kmax = fabs(B.kmax_frac) * n;
    a.kcap = max(1, min((int)ceil(fabs(B.kmax_frac) * n), L.kcap));
    a.tau = B.tau;
    a.gamma = B.gamma;
    a.conv = B.conv;
    a.allow_escalation = B.allow_escalation;
    a.u0 = u0;
    a.cluster = 1;
    Cx cx;
    cx.tsm = smem_raw;
    cx.ssm = smem_raw + kTrsvSmem;
    cx.inbox = (unsigned long long*)(smem_raw + kTrsvSmem + kScaledSmem);
    cx.C = 1;
    cx.G = 1;
    cx.cta = 0;
    cx.tid = tid;
    cx.lane = lane;
    cx.warp = warp;
    cx.n = n;
    cx.nblk = (n + kBlk - 1) / kBlk;
    cx.team_k = 0;
    cx.redbuf = 0;
    cx.t_ns = S.t_ns;
    // ---- factor, refine, escalate
    int fmt = T.uf, status = MSIR_OK, nfact = 0, scaled = 0, lu_info = 0, nb_used = 0, nbo_used = 0;
    bool squeeze = false, initial = true, ok = true;
    double t_factor = 0.0, t_refine = 0.0;
    while (true) {
      const int l = level_of(fmt);
      const int tb = B.tune_nb[fmt - 1][batch_bucket(n)], tbo = B.tune_nbo[fmt - 1][batch_bucket(n)];
      int nb = B.nb > 0 ? B.nb : (tb > 0 ? tb : (fmt == MSIR_FP64 ? 16 : 32));
      int nbo = B.nbo > 0 ? B.nbo : (tbo > 0 ? tbo : 64);
      if (fmt == MSIR_FP64 && nb > 16) nb = 16;
      if (nbo % nb) nbo = nb * ((nbo + nb - 1) / nb);
      if (nbo > 64) nbo = 64;
      nb_used = nb;
      nbo_used = nbo;
      void* Fl = ws + L.F[l];
      int* ipiv = (int*)(ws + L.ipiv[l]);
      int* perm = (int*)(ws + L.perm[l]);
      double* R = (double*)(ws + L.R[l]);
      double* Sc = (double*)(ws + L.S[l]);
      const double mu = squeeze ? batch_mu(B, fmt) : 1.0;
      const unsigned long long tf0 = gtimer();
      if (squeeze) batch_squeeze<A0>(Au, ldu, n, R, Sc);
      batch_make_factor<A0>(fmt, Au, ldu, n, Fl, squeeze ? R : nullptr, Sc, mu);
      nfact += squeeze ? 0 : 1;
      batch_lu_fmt(fmt, Fl, ldu, n, nb, nbo, ipiv, &s_info, &s_nonfinite, smem_raw);
      const int info = s_info, nonfin = s_nonfinite;
      __syncthreads();
      if (info != 0 || nonfin != 0) {
        t_factor += 1e-6 * (double)(gtimer() - tf0);
        lu_info = info;
        if (!squeeze && fmt != MSIR_FP64) {
          squeeze = true;
          continue;
        }
        const int nx = next_uf_d(fmt);
        if (!nx || !B.allow_escalation) {
          status = fmt == MSIR_FP64 ? MSIR_ERR_SINGULAR : MSIR_NOT_CONVERGED;
          break;
        }
        fmt = nx;
        squeeze = false;
        continue;
      }
      lu_info = 0;
      scaled = squeeze ? 1 : 0;
      batch_perm(ipiv, n, perm);
      float* inv32 = (float*)(ws + L.inv32[l]);
      double* inv_hi = (double*)(ws + L.inv_hi[l]);
      double* inv_lo = (double*)(ws + L.inv_lo[l]);
      batch_inv_fmt(fmt, Fl, ldu, n, inv32, inv_hi, inv_lo, smem_raw);
      t_factor += 1e-6 * (double)(gtimer() - tf0);
      if (tid == 0 && fmt != S.uf) {  // precision raised (Algorithm 4's escalation)
        S.uf = fmt;
        if (unit_roundoff(fmt) < unit_roundoff(S.u)) S.u = fmt;
        if (unit_roundoff(S.ur) > unit_roundoff(S.u) * unit_roundoff(S.u)) S.ur = square_of(S.u);
        if (!initial) S.phase = PH_ESCALATED;
      }
      __syncthreads();
      a.LU = Fl;
      a.f_fmt = fmt;
      a.perm = perm;
      a.Rsc = squeeze ? R : nullptr;
      a.Ssc = squeeze ? Sc : nullptr;
      a.mu = mu;
      a.inv32 = inv32;
      a.inv_hi = inv_hi;
      a.inv_lo = inv_lo;
      cx.epoch = S.epoch;
      cx.mready = 0;  // the scaled blocks belong to the previous factors
      const unsigned long long tr0 = gtimer();
      ok = batch_refine<A0>(cx, a, S, gsm, s_act, s_reset, s_alg);
      ok = __syncthreads_and(ok) != 0;  // one decision for the whole block
      if (tid == 0) S.epoch = cx.epoch;
      __syncthreads();
      t_refine += 1e-6 * (double)(gtimer() - tr0);
      if (!ok) {
        status = MSIR_ERR_TIMEOUT;
        break;
      }
      if (S.phase == PH_NEED_ESC) {
        const int nx = next_uf_d(S.uf);
        if (!nx || !B.allow_escalation) {
          // nothing finer: the iterate of smallest nbe
          for (int i = tid; i < n; i += kBatchThreads) a.x[i] = a.xbest[i];
          if (tid == 0) S.nbe = S.best_nbe;
          status = MSIR_NOT_CONVERGED;
          break;
        }
        initial = false;
        fmt = nx;
        squeeze = false;
        continue;
      }
      status = S.cged ? MSIR_OK : MSIR_NOT_CONVERGED;
      break;
    }
    __syncthreads();
    epoch = S.epoch;
    // ---- results
    const bool have_x = status >= 0;
    for (int i = tid; i < n; i += kBatchThreads) T.x[i] = have_x ? a.x[i] : 0.0;
    if (tid == 0) {
      rep->status = status;
      rep->cged = S.cged;
      rep->n_stages = min(S.nstages, MSIR_MAX_STAGES);
      rep->n_factorizations = nfact;
      rep->scaled = scaled;
      rep->lu_info = lu_info;
      rep->nb = nb_used;
      rep->nbo = nbo_used;
      rep->total_steps = S.total_steps;
      rep->total_gmres_iters = S.total_gmres;
      rep->nbe = S.cged ? S.nbe : S.best_nbe;
      rep->phi = S.phi;
      rep->t_factor_ms = t_factor;
      rep->t_refine_ms = t_refine;
      double acc = 0.0;
      for (int i = 0; i < 7; ++i) {
        rep->t_phase_ms[i] = 1e-6 * (double)S.t_ns[i];
        acc += rep->t_phase_ms[i];
      }
      rep->t_phase_ms[7] = fmax(0.0, t_refine - acc);
      rep->n_launches = 0;
      rep->n_refine_launches = 0;
      B.status[t] = status;
    }
    __syncthreads();
  }
}

// Batched factorisation only: block b factors tasks b, b + grid, ...
template <typename F>
__global__ void __launch_bounds__(kBatchThreads, 1)
    batched_factor_kernel(const BatchFactorTask* tasks, int count, char* ws, size_t ws_stride, int nb, int nbo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_info, s_nonfinite;
  F* Af = (F*)(ws + (size_t)blockIdx.x * ws_stride);
  int* ipiv = (int*)(ws + (size_t)blockIdx.x * ws_stride + (size_t)kBatchMaxN * kBatchMaxN * sizeof(F));
  for (int t = blockIdx.x; t < count; t += gridDim.x) {
    const BatchFactorTask T = tasks[t];
    const int n = T.n;
    for (int e = threadIdx.x; e < n * n; e += kBatchThreads) {
      const int j = e / n, i = e % n;
      Af[(size_t)i * n + j] = from_d<F>(T.A[(size_t)j * n + i]);
    }
    __syncthreads();
    cta_lu<F>(Af, n, n, nb, nbo, ipiv, &s_info, &s_nonfinite, smem_raw);
    for (int e = threadIdx.x; e < n * n; e += kBatchThreads) T.F_out[e] = (double)to_f(Af[e]);
    for (int i = threadIdx.x; i < n; i += kBatchThreads) T.ipiv_out[i] = ipiv[i];
    if (threadIdx.x == 0) {
      T.flags_out[0] = s_info;
      T.flags_out[1] = s_nonfinite;
    }
    __syncthreads();
  }
}

}  // namespace msir
