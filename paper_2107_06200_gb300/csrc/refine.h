// Arguments and state of the persistent refinement kernel (refine.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msir.h"

namespace msir {

constexpr int kRefThreads = 256;  // 8 warps
constexpr int kBlk = 64;          // rows per block of the row distribution / TRSV
constexpr int kMaxKcap = 2048;    // GMRES iteration cap supported
// 64-bit payload words per value of the substitution hand-off buffer (4:
// enough for a double-double value).  The buffer holds, per direction
// (forward, backward), the solved values and the team-exchanged z of every
// block: 2 * 2 * ceil(n/kBlk) * kBlk * kLLWords words.
constexpr int kLLWords = 4;
// Shared scratch of the substitutions: 8 warps x 64 staged values plus the
// 64 values of z, for the widest value type (double-double, 16 bytes).
constexpr int kTrsvSmem = (kRefThreads / 32 + 1) * kBlk * 16;
// Shared staging of the scaled-block construction: half the inner
// dimension of one tile at a time (inverse high and low words, 64 x 33
// doubles each; factor rows, 32 x 65 doubles).
constexpr int kScLd = kBlk + 1;
constexpr int kScaledSmem = (2 * kBlk * (kBlk / 2 + 1) + (kBlk / 2) * kScLd) * 8;
// Thread-block clusters of the refinement launch: at most kMaxCluster CTAs.
// Each CTA keeps an inbox in shared memory where the CTAs of its cluster
// that solve the blocks just before it (forward) or after it (backward)
// write their solved values: one slot of kBlk values of kLLWords words per
// team position in the cluster.
constexpr int kMaxCluster = 8;
constexpr int kInboxSmem = kMaxCluster * kBlk * kLLWords * 8;

enum RefMode { MODE_SOLVE = 0, MODE_APPLY = 1, MODE_RESIDUAL = 2 };
enum RefPhase {
  PH_START = 0,      // compute x0, then refine
  PH_ESCALATED = 1,  // factors replaced by a finer u_f: recompute r, start SIR
  PH_DONE = 2,
  PH_NEED_ESC = 3,   // GMRES-IR stage ended without convergence: host refactors
  PH_ERROR = 4
};

// Controller state of Algorithm 4 kept on the device between launches.
struct RefState {
  int phase;
  int alg, it;
  int uf, u, ur;
  int cged, status;
  int have_phi0;
  unsigned epoch;     // substitution epoch (one per triangular solve)
  unsigned mready;    // scaled blocks built for the current factors: bit 0 fp32+fp64, bit 1 dd
  int nstages;
  int total_steps, total_gmres;
  double rho_max, delta_prev, phi0, phi;
  double s, nbe, best_nbe;
  // device time (ns) spent by CTA 0 per phase: 0 residual, 1 forward
  // substitution, 2 backward substitution, 3 Gram-Schmidt, 4 operator
  // matrix-vector product, 5 update/norm reductions, 6 Givens/least squares
  unsigned long long t_ns[8];
};

struct RefineArgs {
  int mode;
  int n;
  int a_fmt;               // storage of A_u: MSIR_FP32 or MSIR_FP64
  const void* A;           // A_u, row-major
  int lda;
  const double* b;         // b_u (values in u0)
  const void* LU;          // packed factors in u_f storage, row-major
  int ldf;
  int f_fmt;               // storage format of LU (MSIR_BF16 .. MSIR_FP64)
  const int* perm;         // (P A)[i] = A[perm[i]]
  const double* Rsc;       // squeezing row scalings (nullptr: none)
  const double* Ssc;       // column scalings
  double mu;
  double normA, normb;
  double* x;               // current iterate (values in u)
  double* xn;              // next iterate
  double* x0;
  double* xbest;
  double* r_hi;            // residual, permuted order: r_p[i] = r[perm[i]]
  double* r_lo;
  double* c_hi;            // TRSV right-hand side / work (permuted order)
  double* c_lo;
  double* y_hi;            // forward-substitution result
  double* y_lo;
  double* z_hi;            // backward-substitution result (natural order)
  double* z_lo;
  double* d;               // correction
  double* w;               // GMRES work vector
  double* V;               // Krylov basis in u, row-major: entry j of row i at
  int ldv;                 //   V + i*ldv (ldv >= kcap + 1)
  double* vk;              // the newest basis vector, contiguous (operator input)
  double* H;               // rotated Hessenberg, column-major (kcap+1) x kcap
  double* yv;              // GMRES least-squares solution (kcap)
  double* red;             // reduction scratch: 2 * gridDim.x * kRedW
  double* hred;            // CGS partial sums: gridDim.x * (kcap+1)
  double* hvec;            // reduced CGS coefficients (kcap+1)
  unsigned long long* ll;  // substitution hand-off words (see kLLWords)
  const float* inv32;      // inverses of the diagonal blocks of L and U:
  const double* inv_hi;    // [2][ceil(n/kBlk)][kBlk][kBlk], fp32 and dd
  const double* inv_lo;
  // scaled off-diagonal blocks D_b^{-1} F_bj (j != b) of L (j < b) and U
  // (j > b), row-major with leading dimension ldf, built in the kernel when a
  // solve in that precision first needs them (RefState::mready)
  float* M32;
  double* M64;
  double* Mdh;
  double* Mdl;
  unsigned* bar;           // grid barrier counter (zeroed before launch)
  int* err;
  RefState* st;
  msir_report* rep;        // device copy of the report
  // parameters of Algorithm 4
  int i_max;
  double rho_thresh;
  double kmax;
  int kcap;
  int team_k;              // substitution team size for fp64/dd (0: the rule in team_size)
  double tau;              // <= 0: by u
  double gamma;
  int conv;
  const double* xref;      // MSIR_CONV_TRUE: exact solution (natural order), else nullptr
  int allow_escalation;
  int u0;
  // MODE_APPLY: arith / store formats and input/output (natural order)
  int ap_arith, ap_store;
  const double* ap_in;
  double* ap_out;
  // MODE_RESIDUAL: output s
  double* res_s;
  // optional wavefront timestamps of the last substitution pair (ns):
  // [direction][block][start, off-diagonal done, published, last dependency seen]
  unsigned long long* tsv;
  // CTAs per thread-block cluster of this launch (1: no clusters); the
  // substitutions hand solved blocks to the CTAs of their cluster through
  // distributed shared memory
  int cluster;
};

constexpr int kRedW = 4;

cudaError_t launch_refine(int a_fmt, int f_fmt, const RefineArgs& a, int grid, cudaStream_t st);
int refine_max_grid(int a_fmt, int f_fmt, int kcap);
// Largest cooperative grid of `cluster`-CTA clusters that fits on the
// device for every u_f instantiation with A_u in a_fmt (0 if none).
int refine_max_cluster_grid(int a_fmt, int kcap, int cluster);
size_t refine_smem_bytes(int kcap);

}  // namespace msir
