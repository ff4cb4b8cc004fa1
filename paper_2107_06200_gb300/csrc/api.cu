// Host side of libmsir: the C interface declared in include/msir.h.
//
// A *slot* is one CUDA stream with a device workspace; it runs one system
// at a time through the steps of Algorithm 4 that need the host:
//   ingest -> LU in u_f (retried with the squeezing scaling, or u_f raised,
//   when the factors hold Inf/NaN or a zero pivot, Sec. 2.1.2) -> one
//   persistent refinement launch -> [if it asks for a finer u_f: LU at the
//   next precision -> refinement launch again] -> copy x out.
// Each step is enqueued asynchronously and followed by an event; a runner
// polls the events of all slots, so several systems overlap on the device.
// msir_solve uses one slot, msir_solve_batched several, and the server a
// worker thread that admits queued requests into free slots (continuous
// batching).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/msir.h"
#include "batched.h"
#include "ingest.h"
#include "kernels.h"
#include "refine.h"

using namespace msir;

// ------------------------------------------------------------ utilities

static int elem_size(int fmt) {
  switch (fmt) {
    case MSIR_BF16:
    case MSIR_FP16: return 2;
    case MSIR_FP32: return 4;
    default: return 8;
  }
}
static double unit_roundoff_h(int f) {
  switch (f) {
    case MSIR_BF16: return std::ldexp(1.0, -8);
    case MSIR_FP16: return std::ldexp(1.0, -11);
    case MSIR_FP32: return std::ldexp(1.0, -24);
    case MSIR_FP64: return std::ldexp(1.0, -53);
    default: return std::ldexp(1.0, -106);
  }
}
static int next_uf(int f) {
  if (f == MSIR_BF16 || f == MSIR_FP16) return MSIR_FP32;
  if (f == MSIR_FP32) return MSIR_FP64;
  return 0;
}
static int square_of_h(int u) { return u == MSIR_FP32 ? MSIR_FP64 : MSIR_DD; }
static double xmax_of(int f) {
  switch (f) {
    case MSIR_FP16: return 65504.0;
    case MSIR_BF16: return 3.3895313892515355e38;
    case MSIR_FP32: return 3.4028234663852886e38;
    default: return 1.7976931348623157e308;
  }
}
static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static msir_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MSIR_OK;
  if (e == cudaErrorMemoryAllocation) return MSIR_ERR_NOMEM;
  return MSIR_ERR_CUDA;
}
#define CK(x)                                  \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

static bool valid_triple(msir_triple t) {
  if (t.u != MSIR_FP32 && t.u != MSIR_FP64) return false;
  if (t.ur != square_of_h(t.u)) return false;
  if (t.uf < MSIR_BF16 || t.uf > MSIR_FP64) return false;
  if (unit_roundoff_h(t.uf) < unit_roundoff_h(t.u)) return false;
  return true;
}

// Default LU blocking (numeric parameters, reported back): panels of nb
// columns inside outer blocks of nbo columns.  The outer update runs on the
// tensor cores (bf16/fp16) or as a SIMT GEMM; the inner updates run inside
// the panel kernel, so nbo is kept small.
// From n = 4096 the outer blocks are 128 wide: the trailing matrix is stored
// in u_f after every outer block, so fewer, wider blocks round it fewer
// times (measured: fewer GMRES iterations at n = 8192 and 16384, about half
// the solve time at n = 16384, kappa = 1e3).
static void default_blocking(int fmt, int n, int* nb, int* nbo) {
  *nbo = n >= 4096 ? 128 : 64;
  *nb = fmt == MSIR_FP64 ? 16 : 32;
}

// ------------------------------------------------------------ TMA maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2-D map over a row-major 16-bit matrix: box of 64 columns x 128 rows,
// 128-byte swizzle (the canonical K-major operand layout of tcgen05).
static bool make_tmap(CUtensorMap* m, void* base, int fmt, uint64_t cols, uint64_t rows,
                      uint64_t row_bytes) {
  EncodeTiledFn fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, fmt == MSIR_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                  2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------ context

struct Slot;
struct msir_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int max_dyn_smem = 0;
  std::vector<Slot*> pool;  // slots kept across calls (streams, pinned buffers, workspaces)
  // the batched engine's LU blocking by [u_f - 1][size bucket] (0: default),
  // from msir_autotune_batched
  int tune_nb[4][4] = {}, tune_nbo[4][4] = {};
};

struct Level {  // one factorisation of the current matrix
  int fmt = 0;
  bool valid = false, failed = false;
  int scaled = 0;
  int info = 0, nonfinite = 0;
  int nb = 0, nbo = 0;
  void* F = nullptr;
  int* ipiv = nullptr;
  int* perm = nullptr;
  double* R = nullptr;
  double* S = nullptr;
  double mu = 1.0;
  float* inv32 = nullptr;    // inverses of the diagonal blocks (inv.cu)
  double* inv_hi = nullptr;
  double* inv_lo = nullptr;
  int serial = 0;            // identifies this factorisation (scaled blocks follow it)
  float t_ms = 0;            // device time of this factorisation
};

// Device workspace of one slot, sized for systems up to nmax.
struct Workspace {
  int nmax = 0, kcapmax = 0, G = 0;
  char* base = nullptr;
  size_t bytes = 0;
  int ldu = 0;
  void* Au = nullptr;
  double* b_u = nullptr;
  double* rowsum = nullptr;
  double* rowmax = nullptr;
  double* colmax = nullptr;
  double* scal = nullptr;   // scalar outputs
  void* Fbuf[3] = {nullptr, nullptr, nullptr};
  int* ipiv[3] = {};
  int* perm[3] = {};
  double* R[3] = {};
  double* S[3] = {};
  float* inv32[3] = {};
  double* inv_hi[3] = {};
  double* inv_lo[3] = {};
  void* Ut = nullptr;
  int* map = nullptr;       // map_pos | map_val | map_cnt
  int* iflags = nullptr;    // info, nonfinite, err
  double *x, *xn, *x0, *xbest, *r_hi, *r_lo, *c_hi, *c_lo, *y_hi, *y_lo, *z_hi, *z_lo, *d, *w, *vk;
  double* V = nullptr;
  int ldv = 0;
  double *H, *yv, *red, *hred, *hvec;
  unsigned long long* ll = nullptr;  // substitution hand-off words
  // scaled off-diagonal blocks of the current factorisation (built by the
  // refinement kernel): fp32, fp64, dd high and low words; ldu x n each
  float* M32 = nullptr;
  double* M64 = nullptr;
  double* Mdh = nullptr;
  double* Mdl = nullptr;
  unsigned* bar = nullptr;
  RefState* st = nullptr;
  msir_report* rep = nullptr;
  int* ident = nullptr;
  unsigned long long* tsv = nullptr;
};

// bytes of the substitution hand-off buffer for size n (zeroed whenever the
// substitution epoch restarts)
// ints of one outer block's permutation map (map_pos | map_val | map_cnt)
constexpr int kMapInts = 4 * 256 + 8;

static size_t ll_bytes(int n) {
  return (size_t)4 * ((n + kBlk - 1) / kBlk) * kBlk * kLLWords * sizeof(unsigned long long);
}

static size_t ws_layout(Workspace& w, int n, int kcap, int G, bool alloc_f64_level, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = round_up(off, 256);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t ldu = round_up((size_t)n, 64);
  w.ldu = (int)ldu;
  w.Au = take(ldu * n * 8);
  w.b_u = (double*)take(n * 8);
  w.rowsum = (double*)take(n * 8);
  w.rowmax = (double*)take(n * 8);
  w.colmax = (double*)take(n * 8);
  w.scal = (double*)take(16 * 8);
  const size_t lvl_bytes[3] = {ldu * n * 4, ldu * n * 4, alloc_f64_level ? ldu * n * 8 : 0};
  for (int l = 0; l < 3; ++l) {
    w.Fbuf[l] = lvl_bytes[l] ? take(lvl_bytes[l]) : nullptr;
    w.ipiv[l] = (int*)take(n * 4);
    w.perm[l] = (int*)take(n * 4);
    w.R[l] = (double*)take(n * 8);
    w.S[l] = (double*)take(n * 8);
    const size_t ninv = lvl_bytes[l] ? (size_t)2 * ((n + kBlk - 1) / kBlk) * kBlk * kBlk : 0;
    w.inv32[l] = ninv ? (float*)take(ninv * 4) : nullptr;
    w.inv_hi[l] = ninv ? (double*)take(ninv * 8) : nullptr;
    w.inv_lo[l] = ninv ? (double*)take(ninv * 8) : nullptr;
  }
  w.Ut = take((size_t)n * 256 * 2);
  w.map = (int*)take(2 * kMapInts * 4);  // two outer blocks' maps (look-ahead)
  w.iflags = (int*)take(32 * 4);
  double** vecs[] = {&w.x, &w.xn, &w.x0, &w.xbest, &w.r_hi, &w.r_lo, &w.c_hi,
                     &w.c_lo, &w.y_hi, &w.y_lo, &w.z_hi, &w.z_lo, &w.d, &w.w, &w.vk};
  for (double** v : vecs) *v = (double*)take(n * 8);
  w.ldv = (int)round_up((size_t)kcap + 1, 32);
  w.V = (double*)take((size_t)n * w.ldv * 8);
  w.H = (double*)take((size_t)(kcap + 1) * kcap * 8);
  w.yv = (double*)take((size_t)(kcap + 1) * 8);
  w.red = (double*)take((size_t)2 * G * kRedW * 8);
  w.hred = (double*)take((size_t)G * (kcap + 1) * 8);
  w.hvec = (double*)take((size_t)(kcap + 1) * 8);
  w.ll = (unsigned long long*)take(ll_bytes(n));
  w.M32 = (float*)take(ldu * n * 4);
  w.M64 = (double*)take(ldu * n * 8);
  w.Mdh = (double*)take(ldu * n * 8);
  w.Mdl = (double*)take(ldu * n * 8);
  w.bar = (unsigned*)take(64);
  w.st = (RefState*)take(sizeof(RefState));
  w.rep = (msir_report*)take(sizeof(msir_report));
  w.ident = (int*)take(n * 4);
  w.tsv = (unsigned long long*)take(((size_t)(n + kBlk - 1) / kBlk) * 8 * 8);
  return off + 256;
}

static int kcap_of(int n, double kmax_frac) {
  int k = (int)std::ceil(std::fabs(kmax_frac) * n);
  return std::max(1, std::min(k, kMaxKcap));
}

// Grid of the refinement kernel for size n: up to four CTAs per 64-row
// block (fp64 and double-double substitutions split each block over a team
// of CTAs), and enough CTAs that the O(n^2) fp64 work (residual, u^2
// operator) is spread over the SMs; never more than the SMs.
static int refine_grid(msir_ctx* ctx, int n, int share, int kcap) {
  const int nblk = (n + kBlk - 1) / kBlk;
  const long long work = ((long long)n * n + 16383) / 16384;
  int g = (int)std::min<long long>(ctx->num_sms, std::max<long long>(4LL * nblk, work));
  (void)kcap;
  if (share > 1) g = std::max(1, std::min(g, ctx->num_sms / share));  // systems running together split the SMs
  return g;
}

// Cluster size of a solve's refinement launch.  Clusters are opt-in
// (MSIR_CLUSTER = 2, 4 or 8), for a solve that runs alone on the GPU with at
// least 16 blocks of rows (a cooperative launch of clusters needs whole
// free GPCs, which concurrent solves would fragment).  Measured on one
// GB300 (n = 8192, (bf16, single, double), 328 GMRES iterations): with 8-CTA
// clusters the fp32 substitution hand-off falls from 1.27 to 1.0 us per
// block, but the launch then has 144 instead of 152 CTAs and the whole
// refinement takes 328 instead of 288 ms (the other phases ran 25-40 %
// slower); 2- and 4-CTA clusters gave 288 and 294 ms.  Default: no clusters.
static int env_int(const char* name, int dflt, int lo, int hi);
static int refine_cluster_size(int n, int share) {
  static const int env = [] {
    const int v = env_int("MSIR_CLUSTER", 0, 1, kMaxCluster);
    return (v == 2 || v == 4 || v == 8) ? v : 1;
  }();
  if (share > 1 || (n + kBlk - 1) / kBlk < 16) return 1;
  return env;
}

// exact_n: the workspace must be laid out for exactly nmax (its leading
// dimension then equals that of another workspace laid out for nmax).
static msir_status ws_alloc(Workspace& w, int nmax, int kcapmax, int G, cudaStream_t st,
                            bool exact_n = false) {
  Workspace probe;
  size_t bytes = ws_layout(probe, nmax, kcapmax, G, true, nullptr);
  if (w.base && w.bytes >= bytes && (exact_n ? w.nmax == nmax : w.nmax >= nmax) && w.kcapmax >= kcapmax &&
      w.G >= G)
    return MSIR_OK;
  if (w.base) { cudaFreeAsync(w.base, st); w.base = nullptr; }
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, bytes, st);
  if (e != cudaSuccess) return cuda_status(e);
  w = Workspace();
  w.base = base;
  w.bytes = bytes;
  w.nmax = nmax;
  w.kcapmax = kcapmax;
  w.G = G;
  ws_layout(w, nmax, kcapmax, G, true, base);
  return MSIR_OK;
}

static void ws_free(Workspace& w, cudaStream_t st) {
  if (w.base) cudaFreeAsync(w.base, st);
  w = Workspace();
}

static size_t ws_bytes_for(int n, int kcap, int G) {
  Workspace probe;
  return ws_layout(probe, n, kcap, G, true, nullptr);
}

// ------------------------------------------------------------ LU driver

static bool trsv_timers_enabled();

// MSIR_LU_TIMERS=1: the panel kernel accumulates section timers that the
// factor call prints to stderr (diagnostics only).
// MSIR_LU_LOOKAHEAD=0 turns the look-ahead off (the same arithmetic, one
// stream; for timing comparisons).
static bool lu_no_lookahead() {
  const char* e = getenv("MSIR_LU_LOOKAHEAD");
  return e && e[0] == '0';
}

static bool lu_timers_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("MSIR_LU_TIMERS");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

// CTAs of the panel's cluster: enough to hold the panel in shared memory,
// and otherwise one per kPanelRows rows, up to 16 for panels of more than
// 4096 rows and up to 8 below (a smaller cluster finds free SMs sooner
// beside the persistent refinement kernels of concurrent solves).
// MSIR_PANEL_CTAS and MSIR_PANEL_ROWS override the cap and the row count
// (tuning only).
static int env_int(const char* name, int dflt, int lo, int hi) {
  const char* e = getenv(name);
  if (!e) return dflt;
  const int v = atoi(e);
  return v >= lo && v <= hi ? v : dflt;
}
static int panel_ctas(int m, int Rmax) {
  static const int kPanelCtas = env_int("MSIR_PANEL_CTAS", 0, 1, 16);
  static const int kPanelRows = env_int("MSIR_PANEL_ROWS", 192, 32, 4096);
  const int cap = kPanelCtas > 0 ? kPanelCtas : (m > 4096 ? 16 : 8);
  int C = (m + Rmax - 1) / Rmax;
  if (C > 16) return -1;
  C = std::max(C, std::min(cap, (m + kPanelRows - 1) / kPanelRows));
  return std::max(1, std::min(C, 16));
}

// Streams and events of one LU: the panel of the next outer block runs on
// `aux` (higher priority) while the current block's remaining trailing
// update runs on the main stream (look-ahead).
struct LuStreams {
  cudaStream_t aux = nullptr;
  cudaEvent_t ready = nullptr;   // next block's columns updated (main -> aux)
  cudaEvent_t panel = nullptr;   // next block's panel factored (aux -> main)
};

// Enqueue the LU of fl_fmt(A_u) (optionally squeezed) into level slot l.
// The host reads info / nonfinite after the stream reaches the end.
//
// Right-looking blocked GEPP with a look-ahead of one outer block: for block
// k (columns [k, k+W)), after its panel:
//   main: interchanges + U12 + trailing update of the next block's columns
//         [k+W, k+2W) only, then record `ready`;
//   aux:  wait `ready`, factor the panel of block k+W, record `panel`;
//   main: interchanges of the columns left of the block, U12 and trailing
//         update of the columns [k+2W, n) (with SMs left free for the
//         panel), then wait `panel` before block k+W continues.
// The panel of block k+W reads and writes only its own columns, which the
// rest of block k's work does not touch, so the two run concurrently; the
// two blocks' permutation maps live in separate buffers.
static msir_status enqueue_lu(msir_ctx* ctx, Workspace& w, int n, int u0, int l, int fmt, int nb,
                              int nbo, bool squeeze, Level& L, cudaStream_t st, const LuStreams& ls,
                              int* launches) {
  const int ldf = w.ldu;
  L = Level();
  L.fmt = fmt;
  L.nb = nb;
  L.nbo = nbo;
  L.F = w.Fbuf[l];
  L.ipiv = w.ipiv[l];
  L.perm = w.perm[l];
  if (!L.F) return MSIR_ERR_INVALID;
  const double* R = nullptr;
  const double* S = nullptr;
  if (squeeze) {
    CK(squeeze_scalings(w.Au, w.ldu, n, u0, w.rowmax, w.R[l], w.colmax, w.S[l], st));
    *launches += 4;
    R = w.R[l];
    S = w.S[l];
    L.R = w.R[l];
    L.S = w.S[l];
    L.mu = std::ldexp(1.0, (int)std::floor(std::log2(0.1 * xmax_of(fmt))));
    L.scaled = 1;
  }
  CK(make_factor_matrix(w.Au, w.ldu, n, u0, fmt, L.F, ldf, R, S, L.mu, st));
  *launches += 1;
  CK(cudaMemsetAsync(w.iflags, 0, 32 * sizeof(int), st));
  const bool tc = fmt == MSIR_FP16 || fmt == MSIR_BF16;
  CUtensorMap tmA, tmB;
  if (tc && n > nbo) {
    if (!make_tmap(&tmA, L.F, fmt, (uint64_t)n, (uint64_t)n, (uint64_t)ldf * 2) ||
        !make_tmap(&tmB, w.Ut, fmt, (uint64_t)nbo, (uint64_t)n, (uint64_t)nbo * 2))
      return MSIR_ERR_UNSUPPORTED;
  }
  const int ts = fmt == MSIR_FP64 ? 8 : 4;
  const size_t fixed = panel_smem_bytes(fmt, 0, nb, nbo);
  const size_t budget = std::min<size_t>((size_t)ctx->max_dyn_smem, 220 * 1024);
  const int Rmax = (int)((budget - fixed) / ((size_t)(nb + 1) * ts));
  const bool lookahead = ls.aux != nullptr && !lu_no_lookahead();

  auto panel_args = [&](int k, PanelArgs& pa, int& C) -> msir_status {
    const int m = n - k;
    C = panel_ctas(m, Rmax);
    if (C < 0) return MSIR_ERR_UNSUPPORTED;
    int* map = w.map + ((k / nbo) & 1) * kMapInts;
    pa.A = L.F;
    pa.lda = ldf;
    pa.n = n;
    pa.k = k;
    pa.W = std::min(nbo, n - k);
    pa.nb = nb;
    pa.R_cap = (m + C - 1) / C;
    pa.ipiv = L.ipiv;
    pa.info = w.iflags + 0;
    pa.nonfinite = w.iflags + 1;
    pa.map_pos = map;
    pa.map_val = map + 2 * nbo;
    pa.map_cnt = map + 4 * nbo;
    pa.tdbg = lu_timers_enabled() ? (unsigned long long*)(w.iflags + 8) : nullptr;
    return MSIR_OK;
  };
  // interchanges / U12 / update of block k on the columns [c0, c1) right of
  // it (and the interchanges left of it if left); max_ctas limits the
  // tensor-core update's persistent grid
  auto block_columns = [&](int k, const PanelArgs& pa, bool left, int c0, int c1, int max_ctas,
                           cudaStream_t s2) -> msir_status {
    const int W = pa.W;
    const int ncols = std::max(0, c1 - c0);
    const int nleft = left ? k : 0;
    if (nleft == 0 && ncols == 0) return MSIR_OK;
    SwapTrsmArgs sa;
    sa.A = L.F;
    sa.lda = ldf;
    sa.n = n;
    sa.k = k;
    sa.W = W;
    sa.do_left = left ? 1 : 0;
    sa.c_begin = c0;
    sa.c_end = c0 + ncols;
    sa.map_pos = pa.map_pos;
    sa.map_val = pa.map_val;
    sa.map_cnt = pa.map_cnt;
    sa.Ut = (tc && ncols > 0) ? w.Ut : nullptr;
    sa.ldut = nbo;
    sa.nonfinite = w.iflags + 1;
    const int tiles = (nleft + 31) / 32 + (ncols + 31) / 32;
    CK(launch_swap_trsm(fmt, sa, std::max(1, std::min(tiles, ctx->num_sms)), s2));
    *launches += 1;
    if (ncols > 0) {
      if (tc) {
        TcUpdateArgs ta;
        ta.C = (char*)L.F + ((size_t)(k + W) * ldf + c0) * 2;
        ta.ldc = ldf;
        ta.M = n - k - W;
        ta.N = ncols;
        ta.a_row0 = k + W;
        ta.a_col0 = k;
        ta.b_row0 = c0 - (k + W);
        ta.K = W;
        ta.err = w.iflags + 2;
        CK(launch_update_tc(fmt, &tmA, &tmB, ta, max_ctas, s2));
        *launches += 1;
      } else {
        UpdateArgs ua;
        ua.A = L.F;
        ua.lda = ldf;
        ua.n = n;
        ua.k = k;
        ua.W = W;
        ua.c_begin = c0;
        ua.c_end = c0 + ncols;
        CK(launch_update_simt(fmt, ua, s2));
        *launches += 1;
      }
    }
    return MSIR_OK;
  };

  PanelArgs pa;
  int C = 0;
  msir_status r = panel_args(0, pa, C);
  if (r != MSIR_OK) return r;
  CK(launch_panel(fmt, pa, C, st));
  *launches += 1;
  for (int k = 0; k < n; k += nbo) {
    const int W = pa.W;
    const int knext = k + W;
    if (!lookahead || knext >= n) {
      r = block_columns(k, pa, true, knext, n, ctx->num_sms, st);
      if (r != MSIR_OK) return r;
      if (knext >= n) break;
      r = panel_args(knext, pa, C);
      if (r != MSIR_OK) return r;
      CK(launch_panel(fmt, pa, C, st));
      *launches += 1;
      continue;
    }
    const int la_end = std::min(n, knext + nbo);
    r = block_columns(k, pa, false, knext, la_end, ctx->num_sms, st);
    if (r != MSIR_OK) return r;
    CK(cudaEventRecord(ls.ready, st));
    PanelArgs pn;
    int Cn = 0;
    r = panel_args(knext, pn, Cn);
    if (r != MSIR_OK) return r;
    CK(cudaStreamWaitEvent(ls.aux, ls.ready, 0));
    CK(launch_panel(fmt, pn, Cn, ls.aux));
    *launches += 1;
    CK(cudaEventRecord(ls.panel, ls.aux));
    r = block_columns(k, pa, true, la_end, n, std::max(1, ctx->num_sms - Cn), st);
    if (r != MSIR_OK) return r;
    CK(cudaStreamWaitEvent(st, ls.panel, 0));
    pa = pn;
    C = Cn;
  }
  CK(ipiv_to_perm(L.ipiv, n, L.perm, st));
  *launches += 1;
  L.inv32 = w.inv32[l];
  L.inv_hi = w.inv_hi[l];
  L.inv_lo = w.inv_lo[l];
  static std::atomic<int> serials{0};
  L.serial = ++serials;
  CK(launch_inv_diag(fmt, L.F, ldf, n, L.inv32, L.inv_hi, L.inv_lo, st));
  *launches += 1;
  return MSIR_OK;
}

// ------------------------------------------------------------ jobs/slots

struct MatrixShare;

struct Job {
  int n = 0;
  const double* A = nullptr;  // device, column-major
  int lda = 0;
  const double* b = nullptr;  // device
  double* x = nullptr;        // device output
  msir_triple t{};
  msir_params p{};
  uint64_t matrix_id = 0;     // jobs with equal ids share the ingest and factors
  const double* xref = nullptr;  // MSIR_CONV_TRUE: exact solution (device)
  MatrixShare* share = nullptr;  // columns of one solve running on several slots
  msir_report rep{};
  int status = MSIR_OK;
  bool done = false;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

enum SlotStep { S_IDLE, S_FACTOR, S_REFINE, S_FINISH, S_WAIT };

struct Slot {
  cudaStream_t st = nullptr;
  LuStreams lu;               // look-ahead stream and events of the LU
  Workspace w;
  int m_serial = -1;          // factorisation whose scaled blocks the workspace holds
  Job* job = nullptr;
  SlotStep step = S_IDLE;
  cudaEvent_t ev = nullptr, e0 = nullptr, e1 = nullptr;
  int* h_flags = nullptr;     // pinned: info, nonfinite, err
  RefState* h_state = nullptr;  // pinned
  msir_report* h_rep = nullptr; // pinned
  uint64_t loaded_id = 0;
  int u0 = 0;
  Level lv[3];
  int cur = 0;                // level in use
  int try_fmt = 0;            // format being factored
  bool try_squeeze = false;
  int try_level = 0;
  int G = 1;
  int C = 1;                  // CTAs per thread-block cluster of the refinement launch
  double normA = 0, normb = 0;
  float t_factor = 0, t_refine = 0;
  bool factoring_initial = true;
  int nfact = 0;
  int launches = 0, refine_launches = 0;
  double iter_ms = 0;         // measured device time per GMRES iteration (cost-aware k_max)
  int wait_fmt = 0;           // S_WAIT: the shared level this slot waits for
  RefState state{};
};

// The columns of one multi-right-hand-side solve run on several slots at
// once and share the matrix: A_u and the factor levels live in the
// workspace of the slot that started first (the owner); the other slots
// point their workspaces at those buffers and keep their own vectors,
// Krylov basis, scaled blocks and controller.  Each level is factored once,
// by the first slot that needs it; a slot that needs a level being factored
// waits (S_WAIT).  Levels are factored one after another (a level is only
// needed after the previous one), so the factorisation scratch (Ut, maps,
// flags) stays with the factoring slot.
struct MatrixShare {
  Slot* owner = nullptr;
  bool ready_to_attach = false;  // owner's ingest done (normA known)
  double normA = 0;
  Level lv[3];
  int state[3] = {0, 0, 0};      // 0 none, 1 being factored, 2 ready, 3 failed
};

static int level_index(int fmt) {
  if (fmt == MSIR_FP16 || fmt == MSIR_BF16) return 0;
  if (fmt == MSIR_FP32) return 1;
  return 2;
}

static msir_status slot_init(Slot& s, int device) {
  CK(cudaSetDevice(device));
  CK(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
  int lo_prio = 0, hi_prio = 0;
  CK(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
  CK(cudaStreamCreateWithPriority(&s.lu.aux, cudaStreamNonBlocking, hi_prio));
  CK(cudaEventCreateWithFlags(&s.lu.ready, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s.lu.panel, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
  CK(cudaEventCreate(&s.e0));
  CK(cudaEventCreate(&s.e1));
  CK(cudaMallocHost((void**)&s.h_flags, 16 * sizeof(int)));
  CK(cudaMallocHost((void**)&s.h_state, sizeof(RefState)));
  CK(cudaMallocHost((void**)&s.h_rep, sizeof(msir_report)));
  return MSIR_OK;
}

static void slot_destroy(Slot& s) {
  if (s.st) {
    cudaStreamSynchronize(s.st);
    ws_free(s.w, s.st);
    cudaStreamSynchronize(s.st);
    cudaStreamDestroy(s.st);
  }
  if (s.lu.aux) {
    cudaStreamSynchronize(s.lu.aux);
    cudaStreamDestroy(s.lu.aux);
  }
  if (s.lu.ready) cudaEventDestroy(s.lu.ready);
  if (s.lu.panel) cudaEventDestroy(s.lu.panel);
  if (s.ev) cudaEventDestroy(s.ev);
  if (s.e0) cudaEventDestroy(s.e0);
  if (s.e1) cudaEventDestroy(s.e1);
  if (s.h_flags) cudaFreeHost(s.h_flags);
  if (s.h_state) cudaFreeHost(s.h_state);
  if (s.h_rep) cudaFreeHost(s.h_rep);
  s = Slot();
}

static msir_status pooled_slots(msir_ctx* ctx, int k, std::vector<Slot*>& out) {
  while ((int)ctx->pool.size() < k) {
    Slot* s = new Slot();
    msir_status r = slot_init(*s, ctx->device);
    if (r != MSIR_OK) {
      slot_destroy(*s);
      delete s;
      return r;
    }
    ctx->pool.push_back(s);
  }
  out.assign(ctx->pool.begin(), ctx->pool.begin() + k);
  return MSIR_OK;
}

// Cost-aware k_max (kmax_frac < 0; the paper leaves the thresholds to the
// costs of the machine, Sec. 2.1.1): a GMRES stage stops once its iterations
// have cost about as much as factoring at the next precision, where the
// stages would go after GMRES-IR.  Next factorisation: the current level's
// measured time times 1.15 (16-bit -> fp32; both LUs are bound by the same
// panel kernel on GB300) or 10 (fp32 -> fp64, the fp64 pipe); none after fp64.
// Per-iteration time: the previous refinement launch's measured time per
// GMRES iteration, else a model of one iteration (two substitution chains
// of ceil(n/64) blocks at 1.5 us, plus A_u and the factors at 6.8 TB/s).
// The cap is never above the paper's k_max and never below 8.
static double cost_aware_kmax(const Slot& s, int n, double kmax_paper) {
  const Level& L = s.lv[s.cur];
  double t_next;
  if (L.fmt == MSIR_FP64) return kmax_paper;
  t_next = L.t_ms * (L.fmt == MSIR_FP32 ? 10.0 : 1.15);
  double t_it = s.iter_ms;
  if (t_it <= 0) {
    const double nb = std::ceil(n / 64.0);
    t_it = 2.0 * nb * 1.5e-3 + (double)n * n * 8.0 / 6.8e9;
  }
  const double k = std::ceil(t_next / t_it);
  return std::max(8.0, std::min(kmax_paper, k));
}

static void fill_args(msir_ctx* ctx, Slot& s, RefineArgs& a, int mode) {
  Job& j = *s.job;
  Workspace& w = s.w;
  Level& L = s.lv[s.cur];
  memset(&a, 0, sizeof(a));
  a.mode = mode;
  a.n = j.n;
  a.a_fmt = s.u0;
  a.A = w.Au;
  a.lda = w.ldu;
  a.b = w.b_u;
  a.LU = L.F;
  a.ldf = w.ldu;
  a.f_fmt = L.fmt;
  a.perm = L.perm;
  a.Rsc = L.scaled ? L.R : nullptr;
  a.Ssc = L.scaled ? L.S : nullptr;
  a.mu = L.scaled ? L.mu : 1.0;
  a.normA = s.normA;
  a.normb = s.normb;
  a.x = w.x; a.xn = w.xn; a.x0 = w.x0; a.xbest = w.xbest;
  a.r_hi = w.r_hi; a.r_lo = w.r_lo; a.c_hi = w.c_hi; a.c_lo = w.c_lo;
  a.y_hi = w.y_hi; a.y_lo = w.y_lo; a.z_hi = w.z_hi; a.z_lo = w.z_lo;
  a.d = w.d; a.w = w.w; a.V = w.V; a.ldv = w.ldv; a.vk = w.vk;
  a.H = w.H; a.yv = w.yv; a.red = w.red; a.hred = w.hred; a.hvec = w.hvec;
  a.ll = w.ll; a.bar = w.bar;
  a.inv32 = L.inv32; a.inv_hi = L.inv_hi; a.inv_lo = L.inv_lo;
  a.M32 = w.M32; a.M64 = w.M64; a.Mdh = w.Mdh; a.Mdl = w.Mdl; a.err = w.iflags + 2; a.st = w.st; a.rep = w.rep;
  a.tsv = trsv_timers_enabled() ? w.tsv : nullptr;
  a.i_max = j.p.i_max;
  a.rho_thresh = j.p.rho_thresh;
  a.kmax = std::fabs(j.p.kmax_frac) * j.n;
  a.kcap = kcap_of(j.n, std::fabs(j.p.kmax_frac));
  if (j.p.kmax_frac < 0) {
    const double k = cost_aware_kmax(s, j.n, a.kmax);
    a.kmax = k;
    a.kcap = std::min(a.kcap, std::max(1, (int)std::ceil(k)));
  }
  // MSIR_TEAM_K (1, 2, 4 or 8) fixes the fp64/dd substitution team size
  // (tuning only; the default rule is in team_size)
  static const int team_k = [] {
    const int v = env_int("MSIR_TEAM_K", 0, 1, 8);
    return (v == 1 || v == 2 || v == 4 || v == 8) ? v : 0;
  }();
  a.team_k = team_k;
  a.cluster = (mode == MODE_SOLVE && s.C > 1 && s.G % s.C == 0) ? s.C : 1;
  a.tau = j.p.tau;
  a.gamma = j.p.gamma;
  a.conv = j.p.conv;
  a.xref = j.p.conv == MSIR_CONV_TRUE ? j.xref : nullptr;
  a.allow_escalation = j.p.allow_escalation;
  a.u0 = j.t.u;
  (void)ctx;
}

// Enqueue one factorisation attempt of the slot's current job.
// MSIR_TRSV_TIMERS=1: per-block timestamps of the last substitution pair of
// each refinement launch, summarised on stderr (diagnostics only).
static bool trsv_timers_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("MSIR_TRSV_TIMERS");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

// MSIR_DEBUG_WAITS=1: after a device wait ran out, print where (the site
// record the kernels leave next to the error flag; diagnostics only).
static void print_wait_site(Slot& s) {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("MSIR_DEBUG_WAITS");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  if (v != 1) return;
  int d[5] = {0, 0, 0, 0, 0};
  cudaMemcpy(d, s.w.iflags + 24, sizeof(d), cudaMemcpyDeviceToHost);  // err (iflags + 2) + 22
  static const char* names[] = {"?", "grid barrier", "substitution hand-off", "?", "tensor-core mbarrier"};
  fprintf(stderr, "[msir wait] n=%d G=%d site=%s block=%d values=%d %d %d (0x%x; 0x%x)\n", s.job ? s.job->n : 0, s.G,
          names[(d[0] >= 0 && d[0] <= 4) ? d[0] : 0], d[1], d[2], d[3], d[4], (unsigned)d[2], (unsigned)d[4]);
}

static void print_trsv_timers(Slot& s) {
  if (!trsv_timers_enabled() || !s.job) return;
  const int nblk = (s.job->n + kBlk - 1) / kBlk;
  std::vector<unsigned long long> t((size_t)nblk * 8);
  cudaStreamSynchronize(s.st);
  cudaMemcpy(t.data(), s.w.tsv, t.size() * 8, cudaMemcpyDeviceToHost);
  for (int dir = 0; dir < 2; ++dir) {
    unsigned long long t0 = ~0ull, t1 = 0;
    double off = 0, diag = 0, offmax = 0, diagmax = 0, gap = 0, seen = 0, last = 0;
    int ngap = 0;
    for (int b = 0; b < nblk; ++b) {
      const unsigned long long* q = &t[((size_t)dir * nblk + b) * 4];
      t0 = std::min(t0, q[0]);
      t1 = std::max(t1, q[2]);
      off += (double)(q[1] - q[0]);
      diag += (double)(q[2] - q[1]);
      offmax = std::max(offmax, (double)(q[1] - q[0]));
      diagmax = std::max(diagmax, (double)(q[2] - q[1]));
      const int pb = dir ? b + 1 : b - 1;  // the block this one waits for last
      if (pb >= 0 && pb < nblk) {
        const unsigned long long* pq = &t[((size_t)dir * nblk + pb) * 4];
        if (q[1] > pq[2] && q[3] >= pq[2] && q[1] >= q[3]) {
          gap += (double)(q[1] - pq[2]);
          seen += (double)(q[3] - pq[2]);
          last += (double)(q[1] - q[3]);
          ++ngap;
        }
      }
    }
    const double g = ngap ? 1e-3 / ngap : 0.0;
    fprintf(stderr, "[msir trsv %s] blocks %d span %.1f us, per block: offdiag avg %.2f max %.2f us, diag avg %.2f max %.2f us, "
            "publish->next offdiag done %.2f us (publish->seen %.2f, last tile %.2f)\n",
            dir ? "upper" : "lower", nblk, (t1 - t0) * 1e-3, off / nblk * 1e-3, offmax * 1e-3,
            diag / nblk * 1e-3, diagmax * 1e-3, gap * g, seen * g, last * g);
  }
}

static void print_lu_timers(Slot& s) {
  if (!lu_timers_enabled()) return;
  unsigned long long t[8];
  cudaStreamSynchronize(s.st);
  cudaMemcpy(t, s.w.iflags + 8, sizeof(t), cudaMemcpyDeviceToHost);
  fprintf(stderr, "[msir lu timers ms] colloop %.3f clsync %.3f pivot+push %.3f update %.3f store+maps %.3f inner_swap_trsm %.3f inner_update %.3f load %.3f\n",
          t[0] * 1e-6, t[1] * 1e-6, t[2] * 1e-6, t[3] * 1e-6, t[4] * 1e-6, t[5] * 1e-6, t[6] * 1e-6, t[7] * 1e-6);
}

static msir_status slot_enqueue_factor(msir_ctx* ctx, Slot& s, int fmt, bool squeeze) {
  Job& j = *s.job;
  int nb = j.p.nb, nbo = j.p.nbo;
  int dnb, dnbo;
  default_blocking(fmt, j.n, &dnb, &dnbo);
  if (nb <= 0) nb = dnb;
  if (nbo <= 0) nbo = dnbo;
  const int nbmax = fmt == MSIR_FP64 ? 16 : 32;
  if (nb > nbmax || nbo % nb != 0 || nbo > 256) return MSIR_ERR_INVALID;
  if ((fmt == MSIR_FP16 || fmt == MSIR_BF16) && nbo % 64 != 0 && j.n > nbo) return MSIR_ERR_INVALID;
  s.try_fmt = fmt;
  s.try_squeeze = squeeze;
  s.try_level = level_index(fmt);
  s.nfact += squeeze ? 0 : 1;
  CK(cudaEventRecord(s.e0, s.st));
  msir_status r = enqueue_lu(ctx, s.w, j.n, s.u0, s.try_level, fmt, nb, nbo, squeeze, s.lv[s.try_level], s.st,
                             s.lu, &s.launches);
  if (r != MSIR_OK) return r;
  CK(cudaMemcpyAsync(s.h_flags, s.w.iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, s.st));
  CK(cudaEventRecord(s.e1, s.st));
  CK(cudaEventRecord(s.ev, s.st));
  s.step = S_FACTOR;
  return MSIR_OK;
}

static msir_status slot_enqueue_refine(msir_ctx* ctx, Slot& s) {
  RefineArgs a;
  fill_args(ctx, s, a, MODE_SOLVE);
  // the scaled blocks in the workspace belong to one factorisation
  if (s.m_serial != s.lv[s.cur].serial) {
    s.state.mready = 0;
    s.m_serial = s.lv[s.cur].serial;
  }
  CK(cudaMemcpyAsync(s.w.st, &s.state, sizeof(RefState), cudaMemcpyHostToDevice, s.st));
  CK(cudaMemsetAsync(s.w.bar, 0, 64, s.st));
  CK(cudaEventRecord(s.e0, s.st));
  CK(launch_refine(s.u0, s.lv[s.cur].fmt, a, s.G, s.st));
  s.launches += 1;
  s.refine_launches += 1;
  CK(cudaEventRecord(s.e1, s.st));
  CK(cudaMemcpyAsync(s.h_state, s.w.st, sizeof(RefState), cudaMemcpyDeviceToHost, s.st));
  CK(cudaMemcpyAsync(s.h_rep, s.w.rep, sizeof(msir_report), cudaMemcpyDeviceToHost, s.st));
  CK(cudaMemcpyAsync(s.h_flags, s.w.iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, s.st));
  CK(cudaEventRecord(s.ev, s.st));
  s.step = S_REFINE;
  return MSIR_OK;
}

static void slot_finish(Slot& s, int status) {
  Job& j = *s.job;
  j.status = status;
  s.step = S_FINISH;
  cudaMemcpyAsync(j.x, s.w.x, (size_t)j.n * sizeof(double), cudaMemcpyDeviceToDevice, s.st);
  cudaEventRecord(s.ev, s.st);
}

// ---------------------------------------------- shared matrix (columns)

// Point slot workspace w at the owner's A_u and factor levels.
static void ws_alias(Workspace& w, const Workspace& o) {
  w.Au = o.Au;
  w.ident = o.ident;
  for (int l = 0; l < 3; ++l) {
    w.Fbuf[l] = o.Fbuf[l];
    w.ipiv[l] = o.ipiv[l];
    w.perm[l] = o.perm[l];
    w.R[l] = o.R[l];
    w.S[l] = o.S[l];
    w.inv32[l] = o.inv32[l];
    w.inv_hi[l] = o.inv_hi[l];
    w.inv_lo[l] = o.inv_lo[l];
  }
}

// Give a workspace its own buffers back (after it pointed at an owner's).
static void ws_restore(Workspace& w) {
  if (w.base) ws_layout(w, w.nmax, w.kcapmax, w.G, true, w.base);
}

// Start refining with the shared level of format fmt (ready).
static msir_status slot_use_shared_level(msir_ctx* ctx, Slot& s, int fmt) {
  MatrixShare& sh = *s.job->share;
  const int li = level_index(fmt);
  // this slot's status flags (the factoring slot's LU cleared its own)
  CK(cudaMemsetAsync(s.w.iflags, 0, 32 * sizeof(int), s.st));
  s.lv[li] = sh.lv[li];
  s.cur = li;
  s.nfact += 1;
  if (fmt != s.state.uf) {  // precision was raised
    s.state.uf = fmt;
    if (unit_roundoff_h(s.state.uf) < unit_roundoff_h(s.state.u)) s.state.u = s.state.uf;
    if (unit_roundoff_h(s.state.ur) > unit_roundoff_h(s.state.u) * unit_roundoff_h(s.state.u))
      s.state.ur = square_of_h(s.state.u);
    if (!s.factoring_initial) s.state.phase = PH_ESCALATED;
  }
  return slot_enqueue_refine(ctx, s);
}

// Move a shared-matrix slot to the level of format fmt: use it if it is
// ready, wait if another slot is factoring it, factor it if nobody has, or
// go on to the next format if it failed.  With nothing left the job ends
// (singular when even fp64 failed, else the best iterate).
static msir_status slot_goto_shared_level(msir_ctx* ctx, Slot& s, int fmt) {
  MatrixShare& sh = *s.job->share;
  while (fmt) {
    const int li = level_index(fmt);
    if (sh.state[li] == 2 && sh.lv[li].fmt == fmt) return slot_use_shared_level(ctx, s, fmt);
    if (sh.state[li] == 1) {
      s.step = S_WAIT;
      s.wait_fmt = fmt;
      return MSIR_OK;
    }
    if (sh.state[li] == 0) {
      sh.state[li] = 1;
      return slot_enqueue_factor(ctx, s, fmt, false);
    }
    fmt = s.job->p.allow_escalation ? next_uf(fmt) : 0;
  }
  if (s.factoring_initial) {
    slot_finish(s, MSIR_ERR_SINGULAR);
  } else {
    cudaMemcpyAsync(s.w.x, s.w.xbest, (size_t)s.job->n * 8, cudaMemcpyDeviceToDevice, s.st);
    s.state.nbe = s.state.best_nbe;
    *s.h_state = s.state;
    slot_finish(s, MSIR_NOT_CONVERGED);
  }
  return MSIR_OK;
}


// Start a job in a slot: ingest (unless the matrix is already loaded) and
// the first factorisation.
static msir_status slot_start(msir_ctx* ctx, Slot& s, Job* job, int share) {
  s.job = job;
  Job& j = *job;
  s.u0 = j.t.u;
  s.G = refine_grid(ctx, j.n, share, kcap_of(j.n, j.p.kmax_frac));
  const int kcap = kcap_of(j.n, j.p.kmax_frac);
  // a solve that has the GPU to itself runs its refinement in clusters, so
  // that most substitution hand-offs go through distributed shared memory
  s.C = 1;
  const int C = refine_cluster_size(j.n, share);
  if (C > 1) {
    const int gc = refine_max_cluster_grid(s.u0, kcap, C);
    const int g = std::min(s.G, gc) / C * C;
    if (g >= C) {
      s.G = g;
      s.C = C;
    }
  }
  MatrixShare* sh0 = j.share;
  const bool attaching = sh0 && sh0->owner && sh0->owner != &s;
  // a slot that uses the owner's matrix is laid out for the owner's size,
  // so that both index A_u and the factors with the same leading dimension
  msir_status r = attaching
                      ? ws_alloc(s.w, sh0->owner->w.nmax, std::max(kcap, s.w.kcapmax), std::max(s.G, s.w.G),
                                 s.st, true)
                      : ws_alloc(s.w, std::max(j.n, s.w.nmax), std::max(kcap, s.w.kcapmax),
                                 std::max(s.G, s.w.G), s.st);
  if (r != MSIR_OK) return r;
  s.t_factor = s.t_refine = 0;
  s.iter_ms = 0;
  s.nfact = 0;
  s.launches = 0;
  s.refine_launches = 0;
  memset(&j.rep, 0, sizeof(j.rep));
  MatrixShare* sh = j.share;
  const bool attach = sh && sh->owner && sh->owner != &s;
  if (attach) {
    ws_alias(s.w, sh->owner->w);
    s.loaded_id = 0;
  }
  const bool same = !attach && j.matrix_id != 0 && j.matrix_id == s.loaded_id;
  if (!same && !attach) {
    for (auto& L : s.lv) L = Level();
    CK(ingest_matrix(j.A, j.lda, j.n, s.u0, s.w.Au, s.w.ldu, s.st));
    CK(row_stats(s.w.Au, s.w.ldu, j.n, s.u0, s.w.rowsum, nullptr, s.st));
    CK(max_abs(s.w.rowsum, j.n, 0, s.w.scal + 0, s.st));
    CK(iota(s.w.ident, j.n, s.st));
    s.loaded_id = j.matrix_id;
    s.launches += 4;
  }
  CK(round_vec(j.b, j.n, s.u0, s.w.b_u, s.st));
  CK(max_abs(s.w.b_u, j.n, 1, s.w.scal + 1, s.st));
  s.launches += 2;
  double hs[2];
  CK(cudaMemcpyAsync(hs, s.w.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s.st));
  CK(cudaStreamSynchronize(s.st));
  s.normA = attach ? sh->normA : hs[0];
  s.normb = hs[1];
  if (sh && !sh->owner) {
    sh->owner = &s;
    sh->normA = s.normA;
    sh->ready_to_attach = true;
  }
  memset(&s.state, 0, sizeof(s.state));
  s.state.phase = PH_START;
  s.state.uf = j.t.uf;
  s.state.u = j.t.u;
  s.state.ur = j.t.ur;
  s.state.delta_prev = INFINITY;
  CK(cudaMemsetAsync(s.w.rep, 0, sizeof(msir_report), s.st));
  CK(cudaMemsetAsync(s.w.ll, 0, ll_bytes(j.n), s.st));
  s.factoring_initial = true;
  const int li = level_index(j.t.uf);
  if (sh) return slot_goto_shared_level(ctx, s, j.t.uf);
  if (same && s.lv[li].valid && s.lv[li].fmt == j.t.uf) {
    s.cur = li;
    return slot_enqueue_refine(ctx, s);
  }
  return slot_enqueue_factor(ctx, s, j.t.uf, false);
}

static void fill_report(Slot& s) {
  Job& j = *s.job;
  msir_report& R = j.rep;
  memcpy(&R, s.h_rep, sizeof(msir_report));
  R.status = j.status;
  R.cged = s.h_state->cged;
  R.n_stages = std::min(s.h_state->nstages, MSIR_MAX_STAGES);
  R.n_factorizations = s.nfact;
  R.scaled = s.lv[s.cur].scaled;
  R.lu_info = s.lv[s.cur].info;
  R.nb = s.lv[s.cur].nb;
  R.nbo = s.lv[s.cur].nbo;
  R.total_steps = s.h_state->total_steps;
  R.total_gmres_iters = s.h_state->total_gmres;
  R.nbe = s.h_state->cged ? s.h_state->nbe : s.h_state->best_nbe;
  R.phi = s.h_state->phi;
  R.t_factor_ms = s.t_factor;
  R.t_refine_ms = s.t_refine;
  R.n_launches = s.launches;
  R.n_refine_launches = s.refine_launches;
  for (int i = 0; i < 7; ++i) R.t_phase_ms[i] = 1e-6 * (double)s.h_state->t_ns[i];
  double acc = 0;
  for (int i = 0; i < 7; ++i) acc += R.t_phase_ms[i];
  R.t_phase_ms[7] = std::max(0.0, R.t_refine_ms - acc);
}

// Advance a slot whose event has completed.  Returns true when its job is done.
static bool slot_advance(msir_ctx* ctx, Slot& s) {
  Job& j = *s.job;
  float ms = 0;
  if (s.step == S_WAIT) {  // a shared level another slot is factoring
    if (j.share->state[level_index(s.wait_fmt)] == 1) return false;
    msir_status r = slot_goto_shared_level(ctx, s, s.wait_fmt);
    if (r != MSIR_OK) slot_finish(s, r);
    return false;
  }
  if (s.step == S_FACTOR) {
    cudaEventElapsedTime(&ms, s.e0, s.e1);
    s.t_factor += ms;
    print_lu_timers(s);
    Level& L = s.lv[s.try_level];
    L.t_ms = ms;
    L.info = s.h_flags[0];
    L.nonfinite = s.h_flags[1];
    const int err = s.h_flags[2];
    if (err) { print_wait_site(s); slot_finish(s, err); return false; }
    const bool good = L.info == 0 && L.nonfinite == 0;
    if (good) {
      L.valid = true;
      if (j.share) {
        j.share->lv[s.try_level] = L;
        j.share->state[s.try_level] = 2;
      }
      s.cur = s.try_level;
      if (s.try_fmt != s.state.uf) {  // precision was raised
        s.state.uf = s.try_fmt;
        if (unit_roundoff_h(s.state.uf) < unit_roundoff_h(s.state.u)) s.state.u = s.state.uf;
        if (unit_roundoff_h(s.state.ur) > unit_roundoff_h(s.state.u) * unit_roundoff_h(s.state.u))
          s.state.ur = square_of_h(s.state.u);
        if (!s.factoring_initial) s.state.phase = PH_ESCALATED;
      }
      msir_status r = slot_enqueue_refine(ctx, s);
      if (r != MSIR_OK) slot_finish(s, r);
      return false;
    }
    L.valid = false;
    L.failed = true;
    if (getenv("MSIR_DEBUG_WAITS"))
      fprintf(stderr, "[msir factor] n=%d format=%d squeeze=%d info=%d nonfinite=%d\n", j.n, s.try_fmt,
              (int)s.try_squeeze, L.info, L.nonfinite);
    msir_status r;
    if (!s.try_squeeze && s.try_fmt != MSIR_FP64) {
      r = slot_enqueue_factor(ctx, s, s.try_fmt, true);
    } else {
      const int nx = next_uf(s.try_fmt);
      if (j.share) j.share->state[s.try_level] = 3;  // slots waiting for it move on
      if (!nx || !j.p.allow_escalation) {
        slot_finish(s, s.try_fmt == MSIR_FP64 ? MSIR_ERR_SINGULAR : MSIR_NOT_CONVERGED);
        return false;
      }
      r = j.share ? slot_goto_shared_level(ctx, s, nx) : slot_enqueue_factor(ctx, s, nx, false);
    }
    if (r != MSIR_OK) slot_finish(s, r);
    return false;
  }
  if (s.step == S_REFINE) {
    cudaEventElapsedTime(&ms, s.e0, s.e1);
    s.t_refine += ms;
    print_trsv_timers(s);
    {
      const int iters = s.h_state->total_gmres - s.state.total_gmres;
      if (iters >= 8) s.iter_ms = ms / iters;  // the launch's time per GMRES iteration (an upper bound)
    }
    s.state = *s.h_state;
    const int err = s.h_flags[2];
    if (err || s.state.phase == PH_ERROR) {
      print_wait_site(s);
      slot_finish(s, err ? err : MSIR_ERR_TIMEOUT);
      return false;
    }
    if (s.state.phase == PH_NEED_ESC) {
      const int nx = next_uf(s.state.uf);
      if (!nx || !j.p.allow_escalation) {
        // nothing left: return the best iterate
        cudaMemcpyAsync(s.w.x, s.w.xbest, (size_t)j.n * 8, cudaMemcpyDeviceToDevice, s.st);
        s.state.nbe = s.state.best_nbe;
        *s.h_state = s.state;
        slot_finish(s, MSIR_NOT_CONVERGED);
        return false;
      }
      s.factoring_initial = false;
      if (j.share) {
        msir_status r = slot_goto_shared_level(ctx, s, nx);
        if (r != MSIR_OK) slot_finish(s, r);
        return false;
      }
      const int li = level_index(nx);
      if (s.lv[li].valid && s.lv[li].fmt == nx && j.matrix_id != 0) {
        s.cur = li;
        s.state.uf = nx;
        if (unit_roundoff_h(nx) < unit_roundoff_h(s.state.u)) s.state.u = nx;
        if (unit_roundoff_h(s.state.ur) > unit_roundoff_h(s.state.u) * unit_roundoff_h(s.state.u))
          s.state.ur = square_of_h(s.state.u);
        s.state.phase = PH_ESCALATED;
        msir_status r = slot_enqueue_refine(ctx, s);
        if (r != MSIR_OK) slot_finish(s, r);
        return false;
      }
      msir_status r = slot_enqueue_factor(ctx, s, nx, false);
      if (r != MSIR_OK) slot_finish(s, r);
      return false;
    }
    slot_finish(s, s.state.cged ? MSIR_OK : MSIR_NOT_CONVERGED);
    return false;
  }
  if (s.step == S_FINISH) {
    fill_report(s);
    j.t_done = std::chrono::steady_clock::now();
    j.done = true;
    s.step = S_IDLE;
    s.job = nullptr;
    return true;
  }
  return false;
}

// Run jobs over nslots slots until all are done (used by solve and batched).
// A job of a shared matrix starts on a slot other than the owner's only once
// the owner has loaded the matrix.
static msir_status run_jobs(msir_ctx* ctx, std::vector<Job*>& jobs, std::vector<Slot*>& slots) {
  size_t next = 0, done = 0;
  const int share = (int)slots.size();
  for (Slot* s : slots) s->loaded_id = 0;
  auto can_start = [&](Slot* s, Job* j) {
    return !j->share || !j->share->owner || j->share->owner == s || j->share->ready_to_attach;
  };
  while (done < jobs.size()) {
    bool progressed = false;
    for (Slot* s : slots) {
      if (!s->job) {
        if (next < jobs.size() && can_start(s, jobs[next])) {
          msir_status r = slot_start(ctx, *s, jobs[next++], share);
          if (r != MSIR_OK) return r;
          progressed = true;
        }
        continue;
      }
      cudaError_t q = cudaEventQuery(s->ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_status(q);
      if (s->step != S_WAIT) progressed = true;
      if (slot_advance(ctx, *s)) ++done;
    }
    if (!progressed) std::this_thread::yield();
  }
  return MSIR_OK;
}

// ------------------------------------------------------------ C ABI

extern "C" {

const char* msir_status_string(int s) {
  switch (s) {
    case MSIR_OK: return "ok";
    case MSIR_NOT_CONVERGED: return "not converged";
    case MSIR_ERR_INVALID: return "invalid argument";
    case MSIR_ERR_NOMEM: return "out of device memory";
    case MSIR_ERR_SINGULAR: return "singular (zero pivot in fp64)";
    case MSIR_ERR_TIMEOUT: return "device wait timed out";
    case MSIR_ERR_CUDA: return "CUDA error";
    case MSIR_ERR_UNSUPPORTED: return "unsupported device or size";
    case MSIR_ERR_BUSY: return "server queue full";
  }
  return "unknown";
}

msir_status msir_params_default(msir_params* p) {
  if (!p) return MSIR_ERR_INVALID;
  p->i_max = 10;
  p->rho_thresh = 0.5;
  p->kmax_frac = 0.1;
  p->tau = 0.0;
  p->gamma = 0.0;
  p->conv = MSIR_CONV_COMBINED;
  p->nb = 0;
  p->nbo = 0;
  p->allow_escalation = 1;
  return MSIR_OK;
}

static msir_params resolve_params(const msir_params* p) {
  msir_params q;
  msir_params_default(&q);
  return p ? *p : q;
}

static bool valid_params(const msir_params& p) {
  return p.i_max >= 1 && p.rho_thresh > 0 && p.kmax_frac != 0 && std::fabs(p.kmax_frac) <= 1.0 &&
         (p.conv == MSIR_CONV_COMBINED || p.conv == MSIR_CONV_EST ||
          (p.conv == MSIR_CONV_TRUE && p.x_ref_dev != nullptr)) &&
         p.nb >= 0 && p.nbo >= 0;
}

msir_status msir_create(msir_ctx** out, int device, void* stream) {
  if (!out) return MSIR_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MSIR_ERR_CUDA;
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) return MSIR_ERR_UNSUPPORTED;
  CK(cudaSetDevice(device));
  {
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  msir_ctx* c = new msir_ctx();
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  c->max_dyn_smem = (int)prop.sharedMemPerBlockOptin;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MSIR_ERR_CUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return MSIR_OK;
}

msir_status msir_destroy(msir_ctx* ctx) {
  if (!ctx) return MSIR_ERR_INVALID;
  cudaSetDevice(ctx->device);
  for (Slot* s : ctx->pool) {
    slot_destroy(*s);
    delete s;
  }
  ctx->pool.clear();
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MSIR_OK;
}

struct msir_factors {
  msir_ctx* ctx = nullptr;
  Slot slot;
  Job job;
};

msir_status msir_factor(msir_ctx* ctx, int n, const double* A_dev, int lda, int u, int uf,
                        const msir_params* params, msir_factors** out, int* info, int* nonfinite) {
  if (!ctx || !out || n <= 0 || lda < n || !A_dev) return MSIR_ERR_INVALID;
  if ((u != MSIR_FP32 && u != MSIR_FP64) || uf < MSIR_BF16 || uf > MSIR_FP64) return MSIR_ERR_INVALID;
  msir_triple t{uf, u, u == MSIR_FP32 ? MSIR_FP64 : MSIR_DD};
  msir_params p = resolve_params(params);
  if (!valid_params(p)) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  auto* f = new msir_factors();
  f->ctx = ctx;
  msir_status r = slot_init(f->slot, ctx->device);
  if (r != MSIR_OK) { slot_destroy(f->slot); delete f; return r; }
  f->job.n = n;
  f->job.A = A_dev;
  f->job.lda = lda;
  f->job.t = t;
  f->job.p = p;
  Slot& s = f->slot;
  s.job = &f->job;
  s.u0 = u;
  s.G = refine_grid(ctx, n, 1, 1);
  r = ws_alloc(s.w, n, kcap_of(n, p.kmax_frac), s.G, s.st);
  if (r == MSIR_OK) r = cuda_status(ingest_matrix(A_dev, lda, n, u, s.w.Au, s.w.ldu, s.st));
  if (r == MSIR_OK) r = slot_enqueue_factor(ctx, s, uf, false);
  if (r == MSIR_OK) r = cuda_status(cudaStreamSynchronize(s.st));
  if (r == MSIR_OK) print_lu_timers(s);
  if (r != MSIR_OK) { slot_destroy(s); delete f; return r; }
  Level& L = s.lv[s.try_level];
  L.info = s.h_flags[0];
  L.nonfinite = s.h_flags[1];
  L.valid = true;
  s.cur = s.try_level;
  if (s.h_flags[2]) { int e = s.h_flags[2]; slot_destroy(s); delete f; return (msir_status)e; }
  if (info) *info = L.info;
  if (nonfinite) *nonfinite = L.nonfinite;
  *out = f;
  return MSIR_OK;
}

msir_status msir_factors_destroy(msir_factors* f) {
  if (!f) return MSIR_ERR_INVALID;
  cudaSetDevice(f->ctx->device);
  slot_destroy(f->slot);
  delete f;
  return MSIR_OK;
}

msir_status msir_factors_export(msir_ctx* ctx, const msir_factors* fc, double* F_host, int* ipiv_host) {
  if (!ctx || !fc) return MSIR_ERR_INVALID;
  const Slot& s = fc->slot;
  const Level& L = s.lv[s.cur];
  const int n = fc->job.n;
  CK(cudaSetDevice(ctx->device));
  if (ipiv_host) CK(cudaMemcpy(ipiv_host, L.ipiv, (size_t)n * 4, cudaMemcpyDeviceToHost));
  if (F_host) {
    const int es = elem_size(L.fmt);
    std::vector<unsigned char> raw((size_t)n * s.w.ldu * es);
    CK(cudaMemcpy(raw.data(), L.F, raw.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const unsigned char* p = raw.data() + ((size_t)i * s.w.ldu + j) * es;
        double v;
        if (L.fmt == MSIR_FP64) {
          memcpy(&v, p, 8);
        } else if (L.fmt == MSIR_FP32) {
          float f;
          memcpy(&f, p, 4);
          v = f;
        } else {
          uint16_t h;
          memcpy(&h, p, 2);
          uint32_t bits;
          if (L.fmt == MSIR_BF16) {
            bits = (uint32_t)h << 16;
          } else {  // IEEE half -> single, exact
            const uint32_t sgn = (uint32_t)(h & 0x8000) << 16;
            int e = (h >> 10) & 0x1f;
            uint32_t m = h & 0x3ff;
            if (e == 0x1f) {
              bits = sgn | 0x7f800000u | (m << 13);
            } else if (e == 0) {
              if (m == 0) {
                bits = sgn;
              } else {
                e = 1;
                while (!(m & 0x400)) { m <<= 1; --e; }
                m &= 0x3ff;
                bits = sgn | ((uint32_t)(e + 112) << 23) | (m << 13);
              }
            } else {
              bits = sgn | ((uint32_t)(e + 112) << 23) | (m << 13);
            }
          }
          float f;
          memcpy(&f, &bits, 4);
          v = f;
        }
        F_host[(size_t)i * n + j] = v;
      }
  }
  return MSIR_OK;
}

msir_status msir_factors_apply(msir_ctx* ctx, const msir_factors* fc, int nrhs, const double* B_dev,
                               int ldb, double* X_dev, int ldx, int arith, int store) {
  if (!ctx || !fc || nrhs < 1 || !B_dev || !X_dev) return MSIR_ERR_INVALID;
  const int n = fc->job.n;
  if (ldb < n || ldx < n) return MSIR_ERR_INVALID;
  if (arith != MSIR_FP32 && arith != MSIR_FP64 && arith != MSIR_DD) return MSIR_ERR_INVALID;
  if (arith != MSIR_DD && (store < MSIR_BF16 || store > MSIR_FP64)) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  Slot& s = const_cast<Slot&>(fc->slot);
  CK(cudaMemsetAsync(s.w.ll, 0, ll_bytes(n), s.st));
  RefState st0;
  memset(&st0, 0, sizeof(st0));
  for (int c = 0; c < nrhs; ++c) {
    RefineArgs a;
    fill_args(ctx, s, a, MODE_APPLY);
    a.ap_arith = arith;
    a.ap_store = store;
    a.ap_in = B_dev + (size_t)c * ldb;
    a.ap_out = X_dev + (size_t)c * ldx;
    st0.epoch = (unsigned)(2 * c);
    if (s.m_serial != s.lv[s.cur].serial) {
      st0.mready = 0;
      s.m_serial = s.lv[s.cur].serial;
    }
    CK(cudaMemcpyAsync(s.w.st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s.st));
    CK(cudaMemsetAsync(s.w.bar, 0, 64, s.st));
    CK(launch_refine(s.u0, s.lv[s.cur].fmt, a, s.G, s.st));
    CK(cudaStreamSynchronize(s.st));
    RefState back;
    CK(cudaMemcpy(&back, s.w.st, sizeof(back), cudaMemcpyDeviceToHost));
    st0.mready = back.mready;  // scaled blocks built by this launch stay valid
  }
  int flags[16];
  CK(cudaMemcpy(flags, s.w.iflags, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags[2]) return (msir_status)flags[2];
  return MSIR_OK;
}

msir_status msir_residual(msir_ctx* ctx, int n, const double* A_dev, int lda, int u0,
                          const double* x_dev, const double* b_dev, int ur, double* r_dev,
                          double* s_host) {
  if (!ctx || n <= 0 || lda < n || !A_dev || !x_dev || !b_dev || !r_dev) return MSIR_ERR_INVALID;
  if ((u0 != MSIR_FP32 && u0 != MSIR_FP64) || (ur != MSIR_FP64 && ur != MSIR_DD)) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  Slot s;
  msir_status r = slot_init(s, ctx->device);
  Job j;
  j.n = n;
  j.p = resolve_params(nullptr);
  j.t = msir_triple{MSIR_FP64, u0, ur};
  s.job = &j;
  s.u0 = u0;
  s.G = refine_grid(ctx, n, 1, 1);
  if (r == MSIR_OK) r = ws_alloc(s.w, n, 1, s.G, s.st);
  if (r == MSIR_OK) {
    ingest_matrix(A_dev, lda, n, u0, s.w.Au, s.w.ldu, s.st);
    round_vec(b_dev, n, u0, s.w.b_u, s.st);
    iota(s.w.ident, n, s.st);
    copy_vec(x_dev, n, s.w.x, s.st);
    cudaMemsetAsync(s.w.iflags, 0, 64, s.st);
    s.lv[0].perm = s.w.ident;
    s.cur = 0;
    RefineArgs a;
    fill_args(ctx, s, a, MODE_RESIDUAL);
    a.ap_arith = ur;
    a.res_s = s.w.scal + 2;
    RefState st0;
    memset(&st0, 0, sizeof(st0));
    cudaMemcpyAsync(s.w.st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s.st);
    cudaMemsetAsync(s.w.bar, 0, 64, s.st);
    r = cuda_status(launch_refine(u0, MSIR_FP64, a, s.G, s.st));
    if (r == MSIR_OK) {
      cudaMemcpyAsync(r_dev, s.w.r_hi, (size_t)n * 8, cudaMemcpyDeviceToDevice, s.st);
      if (ur == MSIR_DD) cudaMemcpyAsync(r_dev + n, s.w.r_lo, (size_t)n * 8, cudaMemcpyDeviceToDevice, s.st);
      double sv = 0;
      cudaMemcpyAsync(&sv, s.w.scal + 2, 8, cudaMemcpyDeviceToHost, s.st);
      r = cuda_status(cudaStreamSynchronize(s.st));
      if (s_host) *s_host = sv;
    }
  }
  slot_destroy(s);
  return r;
}

msir_status msir_solve(msir_ctx* ctx, int n, int nrhs, const double* A_dev, int lda, const double* B_dev,
                       int ldb, double* X_dev, int ldx, msir_triple t, const msir_params* params,
                       msir_report* rep) {
  if (!ctx || n <= 0 || nrhs < 1 || nrhs > 16 || lda < n || ldb < n || ldx < n || !A_dev || !B_dev ||
      !X_dev)
    return MSIR_ERR_INVALID;
  if (!valid_triple(t)) return MSIR_ERR_INVALID;
  msir_params p = resolve_params(params);
  if (!valid_params(p)) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  static std::atomic<uint64_t> ids{1};
  const uint64_t id = ids++;
  std::vector<Job> jobs(nrhs);
  std::vector<Job*> jp;
  MatrixShare share;
  for (int c = 0; c < nrhs; ++c) {
    jobs[c].n = n;
    jobs[c].A = A_dev;
    jobs[c].lda = lda;
    jobs[c].b = B_dev + (size_t)c * ldb;
    jobs[c].x = X_dev + (size_t)c * ldx;
    jobs[c].t = t;
    jobs[c].p = p;
    jobs[c].matrix_id = id;
    jobs[c].xref = p.x_ref_dev ? p.x_ref_dev + (size_t)c * n : nullptr;
    jobs[c].share = nrhs > 1 ? &share : nullptr;
    jp.push_back(&jobs[c]);
  }
  // several right-hand sides: columns run on up to K slots at once, sharing
  // the matrix and its factors.  K = 4 by default (at n = 8192 with 16
  // columns, 1 / 4 / 9 / 16 slots measured 466 / 340 / 535 / 638 ms: each
  // column's refinement needs a large share of the SMs for its substitution
  // chains); MSIR_RHS_SLOTS overrides it for tuning
  const int K = nrhs > 1 ? std::min(nrhs, env_int("MSIR_RHS_SLOTS", 4, 1, 64)) : 1;
  std::vector<Slot*> slots;
  msir_status r = pooled_slots(ctx, K, slots);
  // order the slots' work after the caller's stream
  if (r == MSIR_OK) {
    cudaEventRecord(slots[0]->e0, ctx->stream);
    for (Slot* sl : slots) cudaStreamWaitEvent(sl->st, slots[0]->e0, 0);
  }
  if (r == MSIR_OK) r = run_jobs(ctx, jp, slots);
  for (Slot* sl : slots) cudaStreamSynchronize(sl->st);
  // slots that pointed at the owner's matrix get their own buffers back
  for (Slot* sl : slots)
    if (sl != share.owner) {
      ws_restore(sl->w);
      sl->loaded_id = 0;
    }
  if (r != MSIR_OK) return r;
  msir_status agg = MSIR_OK;
  for (int c = 0; c < nrhs; ++c) {
    if (rep) rep[c] = jobs[c].rep;
    if (jobs[c].status < 0) agg = (msir_status)jobs[c].status;
    else if (jobs[c].status == MSIR_NOT_CONVERGED && agg == MSIR_OK) agg = MSIR_NOT_CONVERGED;
  }
  return agg;
}

msir_status msir_solve_host(msir_ctx* ctx, int n, const double* A_host, int lda, const double* b_host,
                            double* x_host, msir_triple t, const msir_params* params, msir_report* rep) {
  if (!ctx || n <= 0 || lda < n || !A_host || !b_host || !x_host) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  double *A = nullptr, *b = nullptr, *x = nullptr;
  CK(cudaMallocAsync((void**)&A, (size_t)lda * n * 8, ctx->stream));
  CK(cudaMallocAsync((void**)&b, (size_t)n * 8, ctx->stream));
  CK(cudaMallocAsync((void**)&x, (size_t)n * 8, ctx->stream));
  cudaMemcpyAsync(A, A_host, (size_t)lda * n * 8, cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(b, b_host, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream);
  msir_status r = msir_solve(ctx, n, 1, A, lda, b, n, x, n, t, params, rep);
  if (r >= 0) cudaMemcpyAsync(x_host, x, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(A, ctx->stream);
  cudaFreeAsync(b, ctx->stream);
  cudaFreeAsync(x, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  return r;
}

// ------------------------------------------------- batched engine (host)

// Byte offsets of one block workspace of the batched engine: the
// single-system layout for (nmax, kcap) and a grid of one block.
static BatchLayout batch_layout(int nmax, int kcap) {
  Workspace w;
  char* const base = reinterpret_cast<char*>((uintptr_t)1 << 20);  // any aligned non-null base
  const size_t bytes = ws_layout(w, nmax, kcap, 1, true, base);
  auto off = [&](const void* p) { return (size_t)((const char*)p - base); };
  BatchLayout L;
  memset(&L, 0, sizeof(L));
  L.Au = off(w.Au); L.b_u = off(w.b_u); L.rowsum = off(w.rowsum); L.rowmax = off(w.rowmax);
  L.colmax = off(w.colmax);
  for (int l = 0; l < 3; ++l) {
    L.F[l] = off(w.Fbuf[l]); L.ipiv[l] = off(w.ipiv[l]); L.perm[l] = off(w.perm[l]);
    L.R[l] = off(w.R[l]); L.S[l] = off(w.S[l]); L.inv32[l] = off(w.inv32[l]);
    L.inv_hi[l] = off(w.inv_hi[l]); L.inv_lo[l] = off(w.inv_lo[l]);
  }
  L.x = off(w.x); L.xn = off(w.xn); L.x0 = off(w.x0); L.xbest = off(w.xbest);
  L.r_hi = off(w.r_hi); L.r_lo = off(w.r_lo); L.c_hi = off(w.c_hi); L.c_lo = off(w.c_lo);
  L.y_hi = off(w.y_hi); L.y_lo = off(w.y_lo); L.z_hi = off(w.z_hi); L.z_lo = off(w.z_lo);
  L.d = off(w.d); L.w = off(w.w); L.vk = off(w.vk);
  L.V = off(w.V); L.H = off(w.H); L.yv = off(w.yv); L.red = off(w.red); L.hred = off(w.hred);
  L.hvec = off(w.hvec); L.ll = off(w.ll); L.M32 = off(w.M32); L.M64 = off(w.M64); L.Mdh = off(w.Mdh);
  L.Mdl = off(w.Mdl); L.bar = off(w.bar); L.iflags = off(w.iflags);
  L.ldu = w.ldu;
  L.ldv = w.ldv;
  L.kcap = kcap;
  L.nmax = nmax;
  L.bytes = round_up(bytes, 256);
  return L;
}

// Systems of the batch that the engine takes: n <= kBatchMaxN.  One launch
// per working precision u0, captured in a CUDA graph (the work counter's
// reset and the persistent kernel) and replayed once.
static msir_status run_batch_engine(msir_ctx* ctx, const std::vector<int>& idx, int u0, const int* n,
                                    const double* const* A_dev, const double* const* b_dev,
                                    double* const* x_dev, const msir_triple* t, const msir_params& p,
                                    msir_report* reps, std::vector<int>& status) {
  const int count = (int)idx.size();
  if (count == 0) return MSIR_OK;
  int nmax = 0;
  for (int i : idx) nmax = std::max(nmax, n[i]);
  const int kcap = kcap_of(nmax, std::fabs(p.kmax_frac));
  const BatchLayout L = batch_layout(nmax, kcap);
  const int gmax = batched_max_grid(u0, kcap);
  if (gmax <= 0) return MSIR_ERR_UNSUPPORTED;
  const int grid = std::max(1, std::min(gmax, count));
  // largest systems first, so the last systems to start are small ones
  std::vector<int> order(idx);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<BatchTask> tasks(count);
  for (int q = 0; q < count; ++q) {
    const int i = order[q];
    tasks[q].A = A_dev[i];
    tasks[q].b = b_dev[i];
    tasks[q].x = x_dev[i];
    tasks[q].n = n[i];
    tasks[q].uf = t[i].uf;
    tasks[q].u = t[i].u;
    tasks[q].ur = t[i].ur;
  }
  cudaStream_t st = ctx->stream;
  char* ws = nullptr;
  BatchTask* d_tasks = nullptr;
  msir_report* d_reps = nullptr;
  int* d_status = nullptr;
  unsigned* d_next = nullptr;
  msir_status r = MSIR_OK;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (r == MSIR_OK) r = cuda_status(cudaMallocAsync(ptr, bytes, st));
  };
  alloc((void**)&ws, L.bytes * (size_t)grid);
  alloc((void**)&d_tasks, sizeof(BatchTask) * count);
  alloc((void**)&d_reps, sizeof(msir_report) * count);
  alloc((void**)&d_status, sizeof(int) * count);
  alloc((void**)&d_next, 256);
  std::vector<msir_report> h_reps(count);
  std::vector<int> h_status(count, 0);
  if (r == MSIR_OK)
    r = cuda_status(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(BatchTask) * count, cudaMemcpyHostToDevice, st));
  if (r == MSIR_OK) {
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.tasks = d_tasks;
    B.count = count;
    B.next = d_next;
    B.ws = ws;
    B.layout = L;
    B.reps = d_reps;
    B.status = d_status;
    B.i_max = p.i_max;
    B.rho_thresh = p.rho_thresh;
    B.kmax_frac = std::fabs(p.kmax_frac);
    B.tau = p.tau;
    B.gamma = p.gamma;
    B.conv = p.conv;
    B.allow_escalation = p.allow_escalation;
    B.nb = p.nb;
    B.nbo = p.nbo;
    memcpy(B.tune_nb, ctx->tune_nb, sizeof(B.tune_nb));
    memcpy(B.tune_nbo, ctx->tune_nbo, sizeof(B.tune_nbo));
    B.mu_half = std::ldexp(1.0, (int)std::floor(std::log2(0.1 * xmax_of(MSIR_FP16))));
    B.mu_bf16 = std::ldexp(1.0, (int)std::floor(std::log2(0.1 * xmax_of(MSIR_BF16))));
    B.mu_single = std::ldexp(1.0, (int)std::floor(std::log2(0.1 * xmax_of(MSIR_FP32))));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemsetAsync(d_next, 0, sizeof(unsigned), st);
      cudaError_t e2 = e1 == cudaSuccess ? launch_batched(u0, B, grid, st) : e1;
      e = cudaStreamEndCapture(st, &graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_reps.data(), d_reps, sizeof(msir_report) * count,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_status.data(), d_status, sizeof(int) * count,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    r = cuda_status(e);
  }
  if (ws) cudaFreeAsync(ws, st);
  if (d_tasks) cudaFreeAsync(d_tasks, st);
  if (d_reps) cudaFreeAsync(d_reps, st);
  if (d_status) cudaFreeAsync(d_status, st);
  if (d_next) cudaFreeAsync(d_next, st);
  cudaStreamSynchronize(st);
  if (r != MSIR_OK) return r;
  for (int q = 0; q < count; ++q) {
    const int i = order[q];
    status[i] = h_status[q];
    if (reps) {
      reps[i] = h_reps[q];
      reps[i].n_launches = q == 0 ? 1 : 0;  // the batch's one launch, counted on its first system
    }
  }
  return MSIR_OK;
}

msir_status msir_solve_batched_host(msir_ctx* ctx, int count, const int* n, const double* const* A_host,
                                    const double* const* b_host, double* const* x_host, const msir_triple* t,
                                    const msir_params* params, msir_report* reps) {
  if (!ctx || count < 0 || (count > 0 && (!n || !A_host || !b_host || !x_host || !t))) return MSIR_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (n[i] <= 0 || !A_host[i] || !b_host[i] || !x_host[i]) return MSIR_ERR_INVALID;
  if (count == 0) return MSIR_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  std::vector<size_t> offA(count), offb(count), offx(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    offA[i] = total;
    total += round_up((size_t)n[i] * n[i] * 8, 256);
    offb[i] = total;
    total += round_up((size_t)n[i] * 8, 256);
    offx[i] = total;
    total += round_up((size_t)n[i] * 8, 256);
  }
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, total, st) != cudaSuccess) {
    cudaGetLastError();
    return MSIR_ERR_NOMEM;
  }
  std::vector<const double*> dA(count), db(count);
  std::vector<double*> dx(count);
  msir_status r = MSIR_OK;
  for (int i = 0; i < count && r == MSIR_OK; ++i) {
    dA[i] = (const double*)(buf + offA[i]);
    db[i] = (const double*)(buf + offb[i]);
    dx[i] = (double*)(buf + offx[i]);
    r = cuda_status(cudaMemcpyAsync((void*)dA[i], A_host[i], (size_t)n[i] * n[i] * 8, cudaMemcpyHostToDevice, st));
    if (r == MSIR_OK)
      r = cuda_status(cudaMemcpyAsync((void*)db[i], b_host[i], (size_t)n[i] * 8, cudaMemcpyHostToDevice, st));
  }
  msir_status rs = r;
  if (r == MSIR_OK) rs = msir_solve_batched(ctx, count, n, dA.data(), db.data(), dx.data(), t, params, reps);
  if (rs >= 0) {
    for (int i = 0; i < count && r == MSIR_OK; ++i)
      r = cuda_status(cudaMemcpyAsync(x_host[i], dx[i], (size_t)n[i] * 8, cudaMemcpyDeviceToHost, st));
    if (r == MSIR_OK) r = cuda_status(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  if (r != MSIR_OK) return r;
  return rs;
}

msir_status msir_factor_batched(msir_ctx* ctx, int count, const int* n, const double* const* A_dev, int fmt,
                                int nb, int nbo, double* const* F_dev, int* const* ipiv_dev,
                                int* const* flags_dev) {
  if (!ctx || count < 0 || (count > 0 && (!n || !A_dev || !F_dev || !ipiv_dev || !flags_dev)))
    return MSIR_ERR_INVALID;
  if (fmt != MSIR_FP16 && fmt != MSIR_BF16 && fmt != MSIR_FP32 && fmt != MSIR_FP64) return MSIR_ERR_INVALID;
  if (nb <= 0) nb = fmt == MSIR_FP64 ? 16 : 32;
  if (nbo <= 0) nbo = 64;
  if (nb > (fmt == MSIR_FP64 ? 16 : 32) || nbo % nb != 0 || nbo > 64) return MSIR_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > kBatchMaxN || !A_dev[i] || !F_dev[i] || !ipiv_dev[i] || !flags_dev[i])
      return MSIR_ERR_INVALID;
  if (count == 0) return MSIR_OK;
  CK(cudaSetDevice(ctx->device));
  std::vector<BatchFactorTask> tasks(count);
  for (int i = 0; i < count; ++i) tasks[i] = BatchFactorTask{A_dev[i], n[i], F_dev[i], ipiv_dev[i], flags_dev[i]};
  const int grid = std::max(1, std::min(count, ctx->num_sms));
  const size_t stride = batched_factor_ws_bytes(fmt);
  cudaStream_t st = ctx->stream;
  BatchFactorTask* d_tasks = nullptr;
  char* ws = nullptr;
  msir_status r = cuda_status(cudaMallocAsync((void**)&d_tasks, sizeof(BatchFactorTask) * count, st));
  if (r == MSIR_OK) r = cuda_status(cudaMallocAsync((void**)&ws, stride * grid, st));
  if (r == MSIR_OK)
    r = cuda_status(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(BatchFactorTask) * count, cudaMemcpyHostToDevice, st));
  if (r == MSIR_OK) r = cuda_status(launch_batched_factor(fmt, d_tasks, count, ws, stride, nb, nbo, grid, st));
  if (r == MSIR_OK) r = cuda_status(cudaStreamSynchronize(st));
  if (ws) cudaFreeAsync(ws, st);
  if (d_tasks) cudaFreeAsync(d_tasks, st);
  cudaStreamSynchronize(st);
  return r;
}

// ------------------------------------------------ the engine's autotuner

static const char* kTuneHeader = "msir batched LU blocking v1";

static bool tune_load(msir_ctx* ctx, const char* path, const char* dev) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool any = false;
  if (!fgets(line, sizeof line, f) || strncmp(line, kTuneHeader, strlen(kTuneHeader)) != 0) {
    fclose(f);
    return false;
  }
  while (fgets(line, sizeof line, f)) {
    char name[256];
    int fmt = 0, bucket = -1, nb = 0, nbo = 0;
    double ms = 0;
    if (sscanf(line, "%255[^|]|%d|%d|%d|%d|%lf", name, &fmt, &bucket, &nb, &nbo, &ms) != 6) continue;
    if (strcmp(name, dev) != 0 || fmt < MSIR_BF16 || fmt > MSIR_FP64 || bucket < 0 || bucket > 3) continue;
    if (nb < 1 || nb > (fmt == MSIR_FP64 ? 16 : 32) || nbo < nb || nbo > 64 || nbo % nb) continue;
    ctx->tune_nb[fmt - 1][bucket] = nb;
    ctx->tune_nbo[fmt - 1][bucket] = nbo;
    any = true;
  }
  fclose(f);
  return any;
}

msir_status msir_autotune_batched(msir_ctx* ctx, int samples, const char* cache_path, int* nb_out, int* nbo_out,
                                  double* ms_out) {
  if (!ctx || samples < 0 || samples > 4096 || (samples == 0 && !cache_path)) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, ctx->device));
  std::string dev(prop.name);
  for (char& c : dev)
    if (c == '|' || c == '\n') c = ' ';
  double best_ms[4][4] = {};
  if (samples == 0) {
    if (!tune_load(ctx, cache_path, dev.c_str())) return MSIR_ERR_INVALID;
  } else {
    cudaStream_t st = ctx->stream;
    const int nmax = kBatchMaxN;
    double *A = nullptr, *F = nullptr;
    int *ipiv = nullptr, *flags = nullptr;
    BatchFactorTask* d_tasks = nullptr;
    char* ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int grid = std::max(1, std::min(samples, ctx->num_sms));
    const size_t stride = batched_factor_ws_bytes(MSIR_FP64);
    msir_status r = MSIR_OK;
    auto alloc = [&](void** p, size_t b) {
      if (r == MSIR_OK) r = cuda_status(cudaMallocAsync(p, b, st));
    };
    alloc((void**)&A, sizeof(double) * samples * nmax * nmax);
    alloc((void**)&F, sizeof(double) * samples * nmax * nmax);
    alloc((void**)&ipiv, sizeof(int) * samples * nmax);
    alloc((void**)&flags, sizeof(int) * samples * 2);
    alloc((void**)&d_tasks, sizeof(BatchFactorTask) * samples);
    alloc((void**)&ws, stride * grid);
    if (r == MSIR_OK) r = cuda_status(cudaEventCreate(&e0));
    if (r == MSIR_OK) r = cuda_status(cudaEventCreate(&e1));
    std::vector<BatchFactorTask> tasks(samples);
    for (int fmt = MSIR_BF16; fmt <= MSIR_FP64 && r == MSIR_OK; ++fmt) {
      const int cand[4][2] = {{fmt == MSIR_FP64 ? 8 : 16, 32}, {fmt == MSIR_FP64 ? 8 : 16, 64},
                              {fmt == MSIR_FP64 ? 16 : 32, 32}, {fmt == MSIR_FP64 ? 16 : 32, 64}};
      for (int b = 0; b < 4 && r == MSIR_OK; ++b) {
        const int n = 64 << b;
        r = cuda_status(launch_fill_random(A, (size_t)samples * n * n, 7u * fmt + b, st));
        for (int i = 0; i < samples; ++i)
          tasks[i] = BatchFactorTask{A + (size_t)i * n * n, n, F + (size_t)i * n * n, ipiv + (size_t)i * nmax,
                                     flags + 2 * i};
        if (r == MSIR_OK)
          r = cuda_status(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(BatchFactorTask) * samples,
                                          cudaMemcpyHostToDevice, st));
        double best = 1e30;
        int bnb = 0, bnbo = 0;
        for (int c = 0; c < 4 && r == MSIR_OK; ++c) {
          float tmin = 1e30f;
          for (int rep = 0; rep < 3 && r == MSIR_OK; ++rep) {  // the first is a warm-up
            cudaEventRecord(e0, st);
            r = cuda_status(launch_batched_factor(fmt, d_tasks, samples, ws, stride, cand[c][0], cand[c][1], grid, st));
            cudaEventRecord(e1, st);
            if (r == MSIR_OK) r = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tmin = std::min(tmin, ms);
          }
          if (tmin < best) {
            best = tmin;
            bnb = cand[c][0];
            bnbo = cand[c][1];
          }
        }
        ctx->tune_nb[fmt - 1][b] = bnb;
        ctx->tune_nbo[fmt - 1][b] = bnbo;
        best_ms[fmt - 1][b] = best;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (void* p : {(void*)A, (void*)F, (void*)ipiv, (void*)flags, (void*)d_tasks, (void*)ws})
      if (p) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    if (r != MSIR_OK) return r;
    if (cache_path) {
      FILE* f = fopen(cache_path, "w");
      if (!f) return MSIR_ERR_INVALID;
      fprintf(f, "%s\n", kTuneHeader);
      for (int fmt = MSIR_BF16; fmt <= MSIR_FP64; ++fmt)
        for (int b = 0; b < 4; ++b)
          fprintf(f, "%s|%d|%d|%d|%d|%.6f\n", dev.c_str(), fmt, b, ctx->tune_nb[fmt - 1][b],
                  ctx->tune_nbo[fmt - 1][b], best_ms[fmt - 1][b]);
      fclose(f);
    }
  }
  for (int i = 0; i < 16; ++i) {
    if (nb_out) nb_out[i] = ctx->tune_nb[i / 4][i % 4];
    if (nbo_out) nbo_out[i] = ctx->tune_nbo[i / 4][i % 4];
    if (ms_out) ms_out[i] = best_ms[i / 4][i % 4];
  }
  return MSIR_OK;
}

// MSIR_BATCH_ENGINE=0 sends every system of msir_solve_batched through the
// concurrent slots (as systems larger than kBatchMaxN always go).
static bool batch_engine_enabled() {
  static const int v = env_int("MSIR_BATCH_ENGINE", 1, 0, 1);
  return v == 1;
}

msir_status msir_solve_batched(msir_ctx* ctx, int count, const int* n, const double* const* A_dev,
                               const double* const* b_dev, double* const* x_dev, const msir_triple* t,
                               const msir_params* params, msir_report* reps) {
  if (!ctx || count < 0 || (count > 0 && (!n || !A_dev || !b_dev || !x_dev || !t))) return MSIR_ERR_INVALID;
  msir_params p = resolve_params(params);
  if (!valid_params(p)) return MSIR_ERR_INVALID;
  if (p.conv == MSIR_CONV_TRUE) return MSIR_ERR_INVALID;  // one exact solution per call only
  for (int i = 0; i < count; ++i)
    if (n[i] <= 0 || !valid_triple(t[i]) || !A_dev[i] || !b_dev[i] || !x_dev[i]) return MSIR_ERR_INVALID;
  if (count == 0) return MSIR_OK;
  CK(cudaSetDevice(ctx->device));
  // small systems: the batched engine (one persistent launch per u0)
  std::vector<int> eng32, eng64, rest;
  for (int i = 0; i < count; ++i) {
    if (batch_engine_enabled() && n[i] <= kBatchMaxN)
      (t[i].u == MSIR_FP32 ? eng32 : eng64).push_back(i);
    else
      rest.push_back(i);
  }
  std::vector<int> eng_status(count, 0);
  msir_status re = run_batch_engine(ctx, eng32, MSIR_FP32, n, A_dev, b_dev, x_dev, t, p, reps, eng_status);
  if (re == MSIR_OK) re = run_batch_engine(ctx, eng64, MSIR_FP64, n, A_dev, b_dev, x_dev, t, p, reps, eng_status);
  if (re != MSIR_OK) return re;
  msir_status agg = MSIR_OK;
  for (int i = 0; i < count; ++i) {
    if (eng_status[i] < 0) agg = (msir_status)eng_status[i];
    else if (eng_status[i] == MSIR_NOT_CONVERGED && agg == MSIR_OK) agg = MSIR_NOT_CONVERGED;
  }
  if (rest.empty()) return agg;
  // the others: concurrent slots, largest systems first (longest-processing-time order)
  const int nrest = (int)rest.size();
  std::vector<Job> jobs(count);
  std::vector<Job*> jp(nrest);
  std::vector<int> order(rest);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  for (int q = 0; q < nrest; ++q) {
    const int i = order[q];
    jobs[i].n = n[i];
    jobs[i].A = A_dev[i];
    jobs[i].lda = n[i];
    jobs[i].b = b_dev[i];
    jobs[i].x = x_dev[i];
    jobs[i].t = t[i];
    jobs[i].p = p;
    jp[q] = &jobs[i];
  }
  int nmax = 0;
  for (int i : rest) nmax = std::max(nmax, n[i]);
  // Concurrency: each system gets about 7/6 CTAs per 64-row block (at least
  // 16): its substitution chains need a CTA per block, and the rest of the
  // SMs are better spent on other systems than on wider grids (the
  // measured optimum for the n = 2000 sweep is 4 systems of 38 CTAs).
  const int nblk_max = (nmax + kBlk - 1) / kBlk;
  const int per_sys = std::max(16, (7 * nblk_max + 5) / 6);
  int nslots = std::max(1, std::min(nrest, std::min(32, ctx->num_sms / per_sys)));
  if (const char* e = getenv("MSIR_BATCH_SLOTS")) {  // tuning override of the concurrency
    const int v = atoi(e);
    if (v > 0) nslots = std::max(1, std::min(nrest, std::min(32, v)));
  }
  std::vector<Slot*> slots;
  msir_status r = pooled_slots(ctx, nslots, slots);
  if (r == MSIR_OK) {
    for (Slot* s : slots) {
      cudaEventRecord(s->e0, ctx->stream);
      cudaStreamWaitEvent(s->st, s->e0, 0);
    }
    r = run_jobs(ctx, jp, slots);
  }
  for (Slot* s : slots) cudaStreamSynchronize(s->st);
  if (r != MSIR_OK) return r;
  for (int i : rest) {
    if (reps) reps[i] = jobs[i].rep;
    if (jobs[i].status < 0) agg = (msir_status)jobs[i].status;
    else if (jobs[i].status == MSIR_NOT_CONVERGED && agg == MSIR_OK) agg = MSIR_NOT_CONVERGED;
  }
  return agg;
}

// ------------------------------------------------------------ server

struct Request {
  uint64_t ticket;
  Job job;
  std::vector<double> A_host;  // column-major n x n copy, held while queued
  std::vector<double> b_host;
  std::vector<double> x_host;
  int state = 0;               // 0 queued, 1 running, 2 done
  size_t footprint = 0;        // device bytes while running (workspace + A, b, x)
  int bypassed = 0;            // admissions of later requests while this one waited first in line
};

// A server slot: a solve slot plus device buffers for the admitted
// request's A, b and x.  Slots keep their workspace and buffers between
// requests (grown when a larger request arrives), so admission allocates
// only when a request needs more than the slot holds.
struct ServerSlot {
  Slot s;
  double* dA = nullptr;
  double* db = nullptr;
  double* dx = nullptr;
  int ncap = 0;             // dA / db / dx sized for n <= ncap
  size_t held = 0;          // device bytes held: workspace + buffers
  Request* req = nullptr;
};

// Host bytes of request copies the server holds at most (queued and running
// requests); a submission beyond it is refused with MSIR_ERR_NOMEM, so an
// overloaded open-loop client gets back-pressure instead of exhausting the
// host's memory.
constexpr size_t kServerHostQueueBytes = (size_t)64 << 30;

struct msir_server {
  msir_ctx* ctx = nullptr;
  size_t budget = 0, in_use = 0;  // in_use: bytes held by all slots
  size_t host_held = 0;           // host bytes of the requests' copies
  int max_slots = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::vector<ServerSlot> slots;
  // admission by expected waiting time (msir_server_set_backlog_limit)
  double max_backlog_ms = 0.0;
  double queued_work = 0.0;   // sum of n^3 over queued requests
  double running_work = 0.0;  // sum of n^3 over admitted, unfinished requests
  std::deque<std::pair<double, double>> done_log;  // (completion time in ms, n^3), last kRateWindow
};

// Completions over which the server's work rate is measured.
constexpr size_t kRateWindow = 32;

static double request_work(int n) { return (double)n * (double)n * (double)n; }

static double steady_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Expected waiting time of a new request in ms: the queued and running
// requests' work over the measured rate (running work counted whole: an
// upper bound), or -1 while fewer than 4 requests have completed.  Caller
// holds S->mu.
static double server_backlog_ms(const msir_server* S) {
  if (S->done_log.size() < 4) return -1.0;
  double w = 0.0;
  for (size_t i = 1; i < S->done_log.size(); ++i) w += S->done_log[i].second;
  const double span = S->done_log.back().first - S->done_log.front().first;
  if (!(span > 0.0) || !(w > 0.0)) return -1.0;
  return (S->queued_work + S->running_work) / (w / span);
}

static size_t request_footprint(int n, const msir_params& p, int u) {
  const size_t nn = (size_t)n * n;
  const size_t ws = ws_bytes_for(n, kcap_of(n, p.kmax_frac), std::min(256, (n + kBlk - 1) / kBlk));
  (void)u;
  return ws + nn * 8 + (size_t)n * 16;
}

// A request that arrives first in line is passed by smaller ones that fit
// while it does not; after this many such admissions no later request is
// admitted before it (it waits for memory to free up instead).
constexpr int kMaxBypass = 8;

// Device bytes that admitting a request of footprint fp into slot ss adds
// to what the slot already holds (slots keep what they allocated).
static size_t admit_delta(const ServerSlot& ss, size_t fp) { return fp > ss.held ? fp - ss.held : 0; }

// Frees what an idle slot holds (workspace and buffers).  Worker only.
static void server_release(msir_server* S, ServerSlot& ss) {
  Slot& s = ss.s;
  ws_free(s.w, s.st);
  if (ss.dA) cudaFreeAsync(ss.dA, s.st);
  if (ss.db) cudaFreeAsync(ss.db, s.st);
  if (ss.dx) cudaFreeAsync(ss.dx, s.st);
  cudaStreamSynchronize(s.st);
  ss.dA = ss.db = ss.dx = nullptr;
  ss.ncap = 0;
  s.loaded_id = 0;
  S->in_use -= ss.held;
  ss.held = 0;
}

// Bring slot ss's buffers and workspace up to request q and copy q's A and
// b to the device (on the slot's stream).  Called by the worker only.
static msir_status server_load(msir_server* S, ServerSlot& ss, Request* q) {
  Slot& s = ss.s;
  const int n = q->job.n;
  const msir_params& p = q->job.p;
  if (n > ss.ncap) {
    if (ss.dA) cudaFreeAsync(ss.dA, s.st);
    if (ss.db) cudaFreeAsync(ss.db, s.st);
    if (ss.dx) cudaFreeAsync(ss.dx, s.st);
    ss.dA = ss.db = ss.dx = nullptr;
    ss.ncap = 0;
    CK(cudaMallocAsync((void**)&ss.dA, (size_t)n * n * 8, s.st));
    CK(cudaMallocAsync((void**)&ss.db, (size_t)n * 8, s.st));
    CK(cudaMallocAsync((void**)&ss.dx, (size_t)n * 8, s.st));
    ss.ncap = n;
  }
  CK(cudaMemcpyAsync(ss.dA, q->A_host.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(ss.db, q->b_host.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s.st));
  q->job.A = ss.dA;
  q->job.lda = n;
  q->job.b = ss.db;
  q->job.x = ss.dx;
  (void)p;
  (void)S;
  return MSIR_OK;
}

static void server_loop(msir_server* S) {
  cudaSetDevice(S->ctx->device);
  const int share = S->max_slots;
  while (true) {
    // admit: requests in arrival order into free slots while the memory
    // they add fits the budget; a request that does not fit is passed by
    // later ones that do, at most kMaxBypass times
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (size_t si = 0; si < S->slots.size(); ++si) {
        ServerSlot& ss = S->slots[si];
        if (ss.req || S->queue.empty()) continue;
        Request* pick = nullptr;
        size_t delta = 0;
        for (int attempt = 0; attempt < 2 && !pick; ++attempt) {
          // the smallest waiting request that fits (fewest rows: least work),
          // unless the head of the queue has been passed kMaxBypass times
          const bool head_turn = S->queue.front()->bypassed >= kMaxBypass;
          auto pick_it = S->queue.end();
          for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
            Request* q = *it;
            const size_t d = admit_delta(ss, q->footprint);
            const bool fits = S->in_use + d <= S->budget || S->in_use == 0;
            if (fits && (!pick || q->job.n < pick->job.n)) {
              pick = q;
              pick_it = it;
              delta = d;
            }
            if (head_turn) break;  // only the head may go (or nothing, until memory frees up)
          }
          if (pick) {
            S->queue.erase(pick_it);
            S->queued_work -= request_work(pick->job.n);
            S->running_work += request_work(pick->job.n);
          }
          if (pick || attempt > 0) break;
          // nothing fits: idle slots give back what they keep, then retry
          bool freed = false;
          for (auto& o : S->slots)
            if (!o.req && o.held > 0) {
              server_release(S, o);
              freed = true;
            }
          if (!freed) break;
        }
        if (!pick) continue;
        if (!S->queue.empty() && S->queue.front()->job.t_submit < pick->job.t_submit)
          S->queue.front()->bypassed++;
        S->in_use += delta;
        ss.held += delta;
        pick->state = 1;
        ss.req = pick;
        lk.unlock();
        Slot& s = ss.s;
        s.loaded_id = 0;
        msir_status r = server_load(S, ss, pick);
        if (r == MSIR_OK) r = slot_start(S->ctx, s, &pick->job, share);
        lk.lock();
        if (r != MSIR_OK) {
          pick->job.status = r;
          pick->state = 2;
          pick->job.t_done = std::chrono::steady_clock::now();
          ss.req = nullptr;
          s.job = nullptr;
          s.step = S_IDLE;
        }
      }
      if (S->stop && S->queue.empty()) {
        bool any = false;
        for (auto& ss : S->slots) any = any || ss.req;
        if (!any) break;
      }
    }
    bool progressed = false;
    for (size_t si = 0; si < S->slots.size(); ++si) {
      ServerSlot& ss = S->slots[si];
      Slot& s = ss.s;
      Request* q = ss.req;
      if (!q || !s.job) continue;
      cudaError_t e = cudaEventQuery(s.ev);
      if (e == cudaErrorNotReady) continue;
      progressed = true;
      bool done = false;
      if (e != cudaSuccess) {
        q->job.status = MSIR_ERR_CUDA;
        done = true;
        s.job = nullptr;
        s.step = S_IDLE;
      } else {
        done = slot_advance(S->ctx, s);
      }
      if (done) {
        cudaMemcpyAsync(q->x_host.data(), ss.dx, (size_t)q->job.n * 8, cudaMemcpyDeviceToHost, s.st);
        cudaStreamSynchronize(s.st);
        std::lock_guard<std::mutex> lk(S->mu);
        S->host_held -= (size_t)q->job.n * q->job.n * 8;
        q->A_host.clear();
        q->A_host.shrink_to_fit();
        q->job.t_done = std::chrono::steady_clock::now();
        q->state = 2;
        ss.req = nullptr;
        S->running_work -= request_work(q->job.n);
        S->done_log.emplace_back(steady_ms(), request_work(q->job.n));
        if (S->done_log.size() > kRateWindow) S->done_log.pop_front();
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(S->mu);
      bool idle = S->queue.empty();
      for (auto& ss : S->slots) idle = idle && !ss.req;
      if (idle && !S->stop)
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
      else
        S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

msir_status msir_server_create(msir_ctx* ctx, size_t hbm_budget_bytes, int max_slots, msir_server** out) {
  if (!ctx || !out || max_slots < 1 || max_slots > 64) return MSIR_ERR_INVALID;
  CK(cudaSetDevice(ctx->device));
  auto* S = new msir_server();
  S->ctx = ctx;
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    hbm_budget_bytes = (size_t)(0.9 * (double)fr);
  }
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->slots.resize(max_slots);
  for (auto& ss : S->slots) {
    msir_status r = slot_init(ss.s, ctx->device);
    if (r != MSIR_OK) {
      for (auto& s2 : S->slots) slot_destroy(s2.s);
      delete S;
      return r;
    }
  }
  S->worker = std::thread(server_loop, S);
  *out = S;
  return MSIR_OK;
}

msir_status msir_server_submit(msir_server* S, int n, const double* A_host, int lda, const double* b_host,
                               msir_triple t, const msir_params* params, uint64_t* ticket) {
  if (!S || n <= 0 || lda < n || !A_host || !b_host || !ticket) return MSIR_ERR_INVALID;
  if (!valid_triple(t)) return MSIR_ERR_INVALID;
  msir_params p = resolve_params(params);
  if (!valid_params(p)) return MSIR_ERR_INVALID;
  if (p.conv == MSIR_CONV_TRUE) return MSIR_ERR_INVALID;  // the server does not keep device x_ref
  auto* q = new (std::nothrow) Request();
  if (!q) return MSIR_ERR_NOMEM;
  q->job.n = n;
  q->job.lda = n;
  q->job.t = t;
  q->job.p = p;
  q->footprint = request_footprint(n, p, t.u);
  // copy in now (host memory; the caller may free its buffers on return);
  // the device copy is made when the request is admitted
  const size_t hb = ((size_t)n * n + 2 * (size_t)n) * 8;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const double bl = S->max_backlog_ms > 0.0 ? server_backlog_ms(S) : -1.0;
    if (S->host_held + hb > kServerHostQueueBytes || (bl >= 0.0 && bl > S->max_backlog_ms)) {
      delete q;
      return MSIR_ERR_BUSY;
    }
    S->host_held += hb;
  }
  try {
    q->A_host.resize((size_t)n * n);
    q->b_host.assign(b_host, b_host + n);
    q->x_host.assign(n, 0.0);
  } catch (...) {
    delete q;
    std::lock_guard<std::mutex> lk(S->mu);
    S->host_held -= hb;
    return MSIR_ERR_NOMEM;
  }
  for (int j = 0; j < n; ++j) memcpy(q->A_host.data() + (size_t)j * n, A_host + (size_t)j * lda, (size_t)n * 8);
  q->job.t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->ticket = S->next_ticket++;
    S->all[q->ticket] = q;
    S->queue.push_back(q);
    S->queued_work += request_work(n);
  }
  S->cv.notify_all();
  *ticket = q->ticket;
  return MSIR_OK;
}

msir_status msir_server_set_backlog_limit(msir_server* S, double max_backlog_ms) {
  if (!S || !(max_backlog_ms >= 0.0) || !std::isfinite(max_backlog_ms)) return MSIR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_backlog_ms = max_backlog_ms;
  return MSIR_OK;
}

msir_status msir_server_poll(msir_server* S, uint64_t ticket, int* state, double* x_host, msir_report* rep,
                             double* latency_ms) {
  if (!S || !state) return MSIR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return MSIR_ERR_INVALID;
  Request* q = it->second;
  *state = q->state;
  if (q->state != 2) return MSIR_OK;
  if (x_host) memcpy(x_host, q->x_host.data(), (size_t)q->job.n * 8);
  if (rep) *rep = q->job.rep;
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(q->job.t_done - q->job.t_submit).count();
  const int st = q->job.status;
  S->host_held -= 2 * (size_t)q->job.n * 8;
  S->all.erase(it);
  delete q;
  return st < 0 ? (msir_status)st : MSIR_OK;
}

msir_status msir_server_destroy(msir_server* S) {
  if (!S) return MSIR_ERR_INVALID;
  S->stop = true;
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& ss : S->slots) {
    if (ss.s.st) {
      if (ss.dA) cudaFreeAsync(ss.dA, ss.s.st);
      if (ss.db) cudaFreeAsync(ss.db, ss.s.st);
      if (ss.dx) cudaFreeAsync(ss.dx, ss.s.st);
    }
    slot_destroy(ss.s);
  }
  for (auto& kv : S->all) delete kv.second;
  delete S;
  return MSIR_OK;
}

}  // extern "C"
