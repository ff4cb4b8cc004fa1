// The batched engine: many small systems solved by one persistent launch,
// one thread block per system at a time (batched.cu, batched_impl.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/msir.h"
#include "refine.h"

namespace msir {

// Byte offsets of the buffers of one block's workspace, laid out for
// systems of up to nmax rows (every block has its own workspace, reused for
// each system it solves).
struct BatchLayout {
  size_t Au, b_u, rowsum, rowmax, colmax;
  size_t F[3], ipiv[3], perm[3], R[3], S[3], inv32[3], inv_hi[3], inv_lo[3];
  size_t x, xn, x0, xbest, r_hi, r_lo, c_hi, c_lo, y_hi, y_lo, z_hi, z_lo, d, w, vk;
  size_t V, H, yv, red, hred, hvec, ll, M32, M64, Mdh, Mdl, bar, iflags;
  int ldu, ldv, kcap, nmax;
  size_t bytes;  // size of one workspace (256-byte multiple)
};

// One system of the batch: A column-major (lda = n), b, x on the device.
struct BatchTask {
  const double* A;
  const double* b;
  double* x;
  int n;
  int uf, u, ur;
};

struct BatchArgs {
  const BatchTask* tasks;
  int count;
  unsigned* next;       // work counter (zeroed before the launch)
  char* ws;             // gridDim.x workspaces of layout.bytes
  BatchLayout layout;
  msir_report* reps;    // per task (device)
  int* status;          // per task (device)
  // Algorithm 4's parameters, one set for the batch
  int i_max;
  double rho_thresh, kmax_frac, tau, gamma;
  int conv, allow_escalation, nb, nbo;  // nb, nbo > 0: this blocking for every LU
  double mu_half, mu_bf16, mu_single;   // squeezing mu = 2^floor(log2(0.1 x_max)) per u_f
  // nb, nbo <= 0: the blocking of an LU in u_f = fmt of a system of n rows
  // is tune_nb/nbo[fmt - 1][bucket], bucket = 0, 1, 2, 3 for n <= 64, 128,
  // 256, 512 (0 there: the defaults 32 (fp64 16) and 64)
  int tune_nb[4][4], tune_nbo[4][4];
};

// size bucket of the tuning table
__host__ __device__ inline int batch_bucket(int n) { return n <= 64 ? 0 : (n <= 128 ? 1 : (n <= 256 ? 2 : 3)); }

// Smallest and largest n the engine takes (one block factors and refines
// the whole system); systems of other sizes go through the slots.
constexpr int kBatchMaxN = 512;

// dynamic shared memory of the engine for a GMRES cap of kcap iterations
size_t batch_smem_bytes(int kcap);
cudaError_t launch_batched(int u0, const BatchArgs& args, int grid, cudaStream_t st);
int batched_max_grid(int u0, int kcap);

// Batched factorisation only (no refinement): system i's n_i x n_i fp64
// column-major A_i is rounded to u_f and factored by one block; the stored
// factors are written as fp64 row-major (L strictly below, U on and above
// the diagonal) with their ipiv and factor-check flags.
struct BatchFactorTask {
  const double* A;
  int n;
  double* F_out;  // n x n row-major
  int* ipiv_out;  // n
  int* flags_out; // [info, nonfinite]
};
cudaError_t launch_batched_factor(int fmt, const BatchFactorTask* tasks, int count, char* ws,
                                  size_t ws_stride, int nb, int nbo, int grid, cudaStream_t st);
// seeded uniform values in [-1, 1) (the autotuner's matrices)
cudaError_t launch_fill_random(double* A, size_t count, unsigned seed, cudaStream_t st);
size_t batched_factor_ws_bytes(int fmt);

}  // namespace msir
