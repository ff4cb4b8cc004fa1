// Argument blocks and launchers of the MSIR kernels (host + device view).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace msir {

constexpr int kPanelThreads = 512;

// lu_outer_panel: factor the (n-k) x W outer block at column k in panels of nb.
struct PanelArgs {
  void* A;        // matrix in its storage format, row-major
  int lda, n, k, W, nb;
  int R_cap;      // rows of a panel held per CTA (>= ceil((n-k)/cluster))
  int* ipiv;      // n global row interchanges (0-based)
  int* info;      // first zero pivot (1-based) or 0
  int* nonfinite; // set to 1 if a stored factor value is Inf/NaN
  int* map_pos;   // outer composite permutation (positions relative to k), 2W
  int* map_val;
  int* map_cnt;
  unsigned long long* tdbg;  // optional section timers of rank 0 / thread 0 (ns), 8
};

// lu_outer_swap_trsm: interchanges of the outer block on the other columns,
// U12 = L11^{-1} A12, and (if Ut) U12^T into Ut (ldut per output column).
// Columns handled: [0, k) if do_left, and [c_begin, c_end) of the columns
// right of the block (k + W <= c_begin).
struct SwapTrsmArgs {
  void* A;
  int lda, n, k, W;
  int do_left, c_begin, c_end;
  const int* map_pos;
  const int* map_val;
  const int* map_cnt;
  void* Ut;
  int ldut;
  int* nonfinite;
};

// A22 <- fl(A22 - L21 U12) with K = W, for the trailing columns
// [c_begin, c_end) (k + W <= c_begin) and every row below the block.
struct UpdateArgs {
  void* A;
  int lda, n, k, W;
  int c_begin, c_end;
};

size_t panel_smem_bytes(int fmt, int R_cap, int nb, int W);
size_t swap_trsm_smem_bytes(int fmt, int W);
cudaError_t launch_panel(int fmt, const PanelArgs& a, int cluster, cudaStream_t st);
cudaError_t launch_swap_trsm(int fmt, const SwapTrsmArgs& a, int grid, cudaStream_t st);
cudaError_t launch_update_simt(int fmt, const UpdateArgs& a, cudaStream_t st);

// tcgen05 trailing update for bf16/fp16 factors (lu_tc.cu).  tmA / tmB are
// CUtensorMap objects (128-byte blobs) for the matrix and for U12^T.
struct TcUpdateArgs {
  void* C;        // &A[k+W][c_begin]
  int ldc;
  int M, N;       // rows, columns updated
  int a_row0, a_col0;  // TMA coordinates of L21 in the matrix map
  int b_row0;     // row of U12^T (in its map) of the first updated column
  int K;          // W (multiple of 64)
  int* err;
};
// max_ctas: persistent grid limit (SMs left free for a concurrent panel).
cudaError_t launch_update_tc(int fmt, const void* tmA, const void* tmB, const TcUpdateArgs& a,
                             int max_ctas, cudaStream_t st);

// Inverses of the 64x64 diagonal blocks of L and U (inv.cu): outputs are
// [2][ceil(n/64)][64][64] (triangle 0 = L, 1 = U).
cudaError_t launch_inv_diag(int fmt, const void* LU, int ldf, int n, float* inv32, double* inv_hi,
                            double* inv_lo, cudaStream_t st);

}  // namespace msir
