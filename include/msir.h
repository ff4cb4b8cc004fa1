/*
 * msir.h -- C interface of libmsir, a GB300 (sm_103a) implementation of
 * multistage mixed-precision iterative refinement (MSIR) for dense A x = b
 * (Oktay & Carson, "Multistage Mixed Precision Iterative Refinement").
 *
 * The method (Algorithm 4 of the paper): factor A = LU by Gaussian
 * elimination with partial pivoting in the factorisation precision u_f;
 * solve A x_0 = b with the factors in u_f; then refine.  Each step computes
 * r = b - A x in the residual precision u_r, scales it by ||r||_inf
 * (Sec. 2.1.2) and solves the correction equation either with the factors
 * (SIR, Algorithm 1), by GMRES preconditioned with the factors whose
 * operator is applied in the working precision u (SGMRES-IR, Algorithm 3),
 * or by the same GMRES with the operator applied in u^2 (GMRES-IR,
 * Algorithm 2).  The stopping criteria of Sec. 2.1.1 switch SIR ->
 * SGMRES-IR -> GMRES-IR; after GMRES-IR the factorisation precision is
 * raised (half/bfloat16 -> single -> double), the matrix refactored and SIR
 * restarts.  The paper's quad residual precision is stood in for by
 * double-double (MSIR_DD).
 *
 * Conventions for every entry point
 *   - Matrices passed in are fp64, column-major with a leading dimension
 *     (LAPACK style).  Vectors are fp64.  "_dev" pointers are CUDA device
 *     pointers on the context's device; "_host" pointers are host memory.
 *   - The caller owns every buffer it passes; the library never frees them
 *     and keeps no pointer to them after the call returns.  The library owns
 *     contexts, factor objects and servers; each has a destroy call.
 *   - Work is ordered after the context's CUDA stream: device inputs must be
 *     complete on that stream (or on the host) when a call starts; work a
 *     caller enqueued on other streams is not waited for.  Every call except
 *     msir_residual_noalloc returns with its outputs complete (it
 *     synchronises the streams it used).
 *   - No call throws across this interface.  Every call returns an
 *     msir_status; on error nothing is written to the caller's outputs
 *     except where a call says otherwise.
 *   - One context may be used by one host thread at a time.  A server is
 *     internally synchronised and may be called from several threads.
 */
#ifndef MSIR_H
#define MSIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number formats.  Unit roundoffs (Table 3 of the paper, bf16 and dd added):
 * bf16 2^-8, fp16 2^-11, fp32 2^-24, fp64 2^-53, dd 2^-106. */
typedef enum {
  MSIR_BF16 = 1,
  MSIR_FP16 = 2,
  MSIR_FP32 = 3,
  MSIR_FP64 = 4,
  MSIR_DD = 5
} msir_prec;

/* Initial precisions (u_f, u, u_r) of Algorithm 4, as msir_prec values.
 * Requirements (Sec. 1 assumes u_f >= u >= u_r; Sec. 2 enforces u_r <= u^2):
 * u in {FP32, FP64}; u_r = FP64 when u = FP32 and DD when u = FP64;
 * u_f in {BF16, FP16, FP32, FP64} and not more precise than u. */
typedef struct {
  int uf;
  int u;
  int ur;
} msir_triple;

/* Convergence test applied after every refinement step (Sec. 2.1.1). */
typedef enum {
  /* 0 <= phi <= gamma*u0 and nbe(x_{i+1}) <= 2*u0 (default) */
  MSIR_CONV_COMBINED = 0,
  /* 0 <= phi <= gamma*u0 only (Eq. (1) estimate, Algorithm 4 literally) */
  MSIR_CONV_EST = 1,
  /* ferr(x_{i+1}) <= u0 and nbe(x_{i+1}) <= u0 against a given exact
   * solution (the stopping rule of the paper's experiments, Sec. 3); needs
   * msir_params.x_ref_dev; msir_solve only */
  MSIR_CONV_TRUE = 2
} msir_conv;

typedef enum {
  MSIR_OK = 0,
  MSIR_NOT_CONVERGED = 1,   /* x holds the iterate of smallest nbe */
  MSIR_ERR_INVALID = -1,    /* bad argument (sizes, triple, params) */
  MSIR_ERR_NOMEM = -2,      /* device allocation failed */
  MSIR_ERR_SINGULAR = -3,   /* exact zero pivot with u_f = fp64 */
  MSIR_ERR_TIMEOUT = -4,    /* a device-side wait hit its deadline */
  MSIR_ERR_CUDA = -5,       /* a CUDA runtime call failed */
  MSIR_ERR_UNSUPPORTED = -6, /* device is not sm_103 or lacks a feature */
  MSIR_ERR_BUSY = -7         /* msir_server_submit: the server's queue is at its
                                host-memory or backlog limit; nothing was queued */
} msir_status;

/* Parameters of Algorithm 4.  msir_params_default() fills the paper's
 * values: i_max = 10, rho_thresh = 0.5 (the "cautious" setting of
 * Sec. 2.1.1), k_max = 0.1 n (Sec. 3), tau by u (1e-6 single, 1e-10
 * double, Sec. 3), gamma = sqrt(n) (Algorithm 4). */
typedef struct {
  int i_max;            /* maximum steps of each variant (Sec. 2.1)          */
  double rho_thresh;    /* ratio threshold of successive corrections; 0.5 is
                           Sec. 2.1.1's cautious setting, 0.9 its aggressive
                           one (more steps per stage on hard problems)       */
  double kmax_frac;     /* k_max = kmax_frac * n GMRES iterations per step;
                           < 0: cost-aware k_max, at most |kmax_frac| * n: a
                           GMRES stage stops once its iterations have cost
                           about as much as the next factorisation (from the
                           measured LU and iteration times)                   */
  double tau;           /* GMRES tolerance; <= 0 picks 1e-6 / 1e-10 by u      */
  double gamma;         /* convergence factor; <= 0 picks sqrt(n)             */
  int conv;             /* msir_conv                                          */
  int nb;               /* panel width of the LU (numeric parameter); 0: default */
  int nbo;              /* outer block width of the LU (multiple of nb); 0: default */
  int allow_escalation; /* 0: stop after GMRES-IR instead of raising u_f      */
  const double* x_ref_dev; /* MSIR_CONV_TRUE: device pointer to the exact
                              solution of (fl_u0(A), fl_u0(B)), n x nrhs
                              column-major with leading dimension n; ferr is
                              ||x - x_ref||_inf / ||x_ref||_inf; otherwise
                              ignored (NULL) */
} msir_params;

#define MSIR_MAX_STAGES 24
#define MSIR_MAX_STEPS 48

typedef enum { MSIR_ALG_SIR = 0, MSIR_ALG_SGMRES = 1, MSIR_ALG_GMRES = 2 } msir_alg;

/* One stage: a run of one variant at one precision triple. */
typedef struct {
  int uf, u, ur;       /* precisions in effect                              */
  int alg;             /* msir_alg                                          */
  int steps;           /* counted refinement steps of this stage            */
  int nonfinite;       /* 1 if the stage ended on an Inf/NaN correction     */
  int gmres_iters[MSIR_MAX_STEPS]; /* GMRES iterations per step (GMRES stages) */
} msir_stage;

/* Written by the library, owned by the caller. */
typedef struct {
  int status;            /* msir_status of this system                       */
  int cged;              /* Algorithm 4's cged                               */
  int n_stages;
  int n_factorizations;
  int scaled;            /* 1 if a squeezed (two-sided scaled) LU was used    */
  int lu_info;           /* first zero pivot of the last LU (1-based), 0 none */
  int nb, nbo;           /* LU blocking actually used                        */
  int total_steps;       /* refinement steps of all stages                   */
  int total_gmres_iters;
  double nbe;            /* normwise backward error of x (infinity norms)    */
  double phi;            /* last convergence estimate phi_i                  */
  double t_factor_ms;    /* device time in LU factorisations                 */
  double t_refine_ms;    /* device time in refinement                        */
  double t_phase_ms[8];  /* refinement time by phase: residual, forward and
                            backward substitution, Gram-Schmidt, operator
                            product, reductions, Givens; other               */
  int n_launches;        /* kernels this library launched for the system     */
  int n_refine_launches; /* of which persistent refinement launches          */
  msir_stage stage[MSIR_MAX_STAGES];
} msir_report;

typedef struct msir_ctx msir_ctx;
typedef struct msir_factors msir_factors;
typedef struct msir_server msir_server;

/* Fills *p with the defaults listed above.  Returns MSIR_ERR_INVALID on NULL. */
msir_status msir_params_default(msir_params* p);

/* Creates a context on CUDA device `device` whose work is ordered on
 * `cuda_stream` (a cudaStream_t; NULL = a stream the library creates).
 * Fails with MSIR_ERR_UNSUPPORTED if the device is not compute capability
 * 10.3.  The context owns a device workspace that grows on demand. */
msir_status msir_create(msir_ctx** out, int device, void* cuda_stream);
msir_status msir_destroy(msir_ctx* ctx);

/* Factor the n x n matrix A (fp64, column-major, leading dimension lda,
 * device memory) in precision uf: the working copy is A_u = fl_u(A) and the
 * factors are those of fl_uf(A_u) by blocked right-looking GEPP (Algorithm 4,
 * first step).  The factor object is owned by the library.  On success
 * *info receives the first exactly-zero pivot (1-based) or 0, and
 * *nonfinite 1 if L or U contain Inf or NaN (neither is an error here).
 * u must be FP32 or FP64, uf one of BF16/FP16/FP32/FP64 (a u_f finer than u
 * is what Algorithm 4 uses after raising u_f while u0 stays, e.g. fp64
 * factors of fl_fp32(A)).  nb / nbo of params select the blocking (0: the
 * library defaults for uf). */
msir_status msir_factor(msir_ctx* ctx, int n, const double* A_dev, int lda, int u, int uf,
                        const msir_params* params, msir_factors** out, int* info,
                        int* nonfinite);
msir_status msir_factors_destroy(msir_factors* f);

/* Copies the packed factors of f to host memory: F_host (n*n doubles,
 * row-major: strictly lower part = L without its unit diagonal, upper part
 * = U, each value exactly the stored u_f value) and ipiv_host (n ints,
 * 0-based LAPACK-style row interchanges: row j was swapped with ipiv[j] at
 * step j).  Either pointer may be NULL. */
msir_status msir_factors_export(msir_ctx* ctx, const msir_factors* f, double* F_host,
                                int* ipiv_host);

/* Applies M^{-1} = U^{-1} L^{-1} P of f to nrhs vectors: X = M^{-1} B, with
 * the substitutions carried out in `arith` (FP32, FP64 or DD) and every
 * computed component rounded to `store` (BF16/FP16/FP32/FP64; ignored for
 * DD).  B_dev, X_dev: device, column-major n x nrhs with leading dimension
 * ldb / ldx.  This is the correction solve of SIR (arith FP32, store u_f)
 * and the preconditioner of SGMRES-IR / GMRES-IR (arith u or u^2). */
msir_status msir_factors_apply(msir_ctx* ctx, const msir_factors* f, int nrhs,
                               const double* B_dev, int ldb, double* X_dev, int ldx,
                               int arith, int store);

/* Residual of Algorithm 4 for one vector: r = b - A_u x in precision ur
 * (FP64 or DD) with A_u = fl_u0(A), and s = ||r||_inf.  A_dev as in
 * msir_factor; x_dev, b_dev: n doubles (b is rounded to u0 first, x is used
 * as given).  r_dev: n doubles (FP64) or 2n doubles (DD: high words then low
 * words).  *s_host receives ||r||_inf (fp64). */
msir_status msir_residual(msir_ctx* ctx, int n, const double* A_dev, int lda, int u0,
                          const double* x_dev, const double* b_dev, int ur, double* r_dev,
                          double* s_host);

/* The paper has no counterpart of this entry point: msir_residual for
 * callers that may not allocate device memory.  Some callers cannot call
 * cudaMalloc themselves -- code running inside a host framework whose
 * memory manager owns every device allocation, or code that must not
 * allocate while a stream is being captured.  This call computes the same
 * residual r = b_u - A_u x (A_u = fl_u0(A), b_u = fl_u0(b), in ur = FP64 or
 * DD) and s = ||r||_inf into caller-provided device buffers: A_dev
 * (column-major, lda), x_dev, b_dev (n doubles), r_dev (n doubles, or 2n
 * for DD: high words then low words), s_dev (one double, device).  Work is
 * enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream)
 * and the call does not wait for it.  Its only scratch is a file-scope
 * device array (about 8 KB per GPU, held until the process exits); the
 * first call on a device looks up that array's device address, so make the
 * first call on each device before any stream capture.  The address is kept
 * for the life of the process: after cudaDeviceReset on a device, do not
 * call this entry point on that device again.  If a CUDA error from earlier
 * work is pending on the calling thread, the call returns MSIR_ERR_CUDA
 * without launching.  Calls share the
 * scratch: calls that overlap on the GPU (different streams, or different
 * host threads on one device) race.  n must be at most 131072
 * (MSIR_ERR_INVALID otherwise).  Never allocates or frees device memory. */
msir_status msir_residual_noalloc(int n, const double* A_dev, int lda, int u0,
                                  const double* x_dev, const double* b_dev, int ur,
                                  double* r_dev, double* s_dev, void* cuda_stream);

/* Solves A X = B for nrhs right-hand sides with MSIR (Algorithm 4) from the
 * initial precisions t.  A_dev: fp64 column-major n x n (lda >= n); B_dev,
 * X_dev: fp64 column-major n x nrhs (ldb, ldx >= n); 1 <= nrhs <= 16.
 * Each column runs its own stage controller (factors are shared per u_f).
 * rep: nrhs reports (may be NULL).  Returns MSIR_OK if every column
 * converged, MSIR_NOT_CONVERGED if some did not (their X columns hold the
 * iterate of smallest nbe), or an error. */
msir_status msir_solve(msir_ctx* ctx, int n, int nrhs, const double* A_dev, int lda,
                       const double* B_dev, int ldb, double* X_dev, int ldx, msir_triple t,
                       const msir_params* params, msir_report* rep);

/* Same as msir_solve for one right-hand side with host buffers: A_host
 * (column-major), b_host, x_host.  Copies in and out on the context stream. */
msir_status msir_solve_host(msir_ctx* ctx, int n, const double* A_host, int lda,
                            const double* b_host, double* x_host, msir_triple t,
                            const msir_params* params, msir_report* rep);

/* Solves `count` independent systems of possibly different sizes.  n[i],
 * A_dev[i] (n[i] x n[i], column-major, lda = n[i]), b_dev[i], x_dev[i]
 * (n[i] doubles) and t[i] are host arrays of device pointers / values;
 * reps: count reports (may be NULL).
 * Systems with n <= 512 go to the batched engine: one persistent launch per
 * working precision u (captured in a CUDA graph), in which each thread
 * block takes the next system and runs all of Algorithm 4 on it (ingest,
 * the LU of msir_factor_batched, the factor check and squeezed retry, SIR /
 * SGMRES-IR / GMRES-IR with the stopping logic, escalation of u_f with
 * refactoring on the device).  A cost-aware k_max (kmax_frac < 0) is taken
 * there as the fixed k_max = |kmax_frac| n.  Larger systems share the GPU
 * as concurrent solves whose refinement runs as persistent launches over
 * groups of SMs.  Returns MSIR_OK if all converged, MSIR_NOT_CONVERGED if
 * some did not.  MSIR_CONV_TRUE is not accepted here (MSIR_ERR_INVALID). */
msir_status msir_solve_batched(msir_ctx* ctx, int count, const int* n,
                               const double* const* A_dev, const double* const* b_dev,
                               double* const* x_dev, const msir_triple* t,
                               const msir_params* params, msir_report* reps);

/* msir_solve_batched with host buffers: A_host[i] (n[i] x n[i], column-
 * major, lda = n[i]), b_host[i] and x_host[i] (n[i] doubles) are host
 * memory (pinned memory copies fastest).  The call copies A and b into one
 * device allocation on the context stream, solves as msir_solve_batched
 * and copies every x back before it returns.  Errors as msir_solve_batched,
 * and MSIR_ERR_NOMEM if the device copy cannot be allocated. */
msir_status msir_solve_batched_host(msir_ctx* ctx, int count, const int* n, const double* const* A_host,
                                    const double* const* b_host, double* const* x_host, const msir_triple* t,
                                    const msir_params* params, msir_report* reps);

/* Batched LU, the factorisation of the batched engine (Algorithm 4's first
 * step for many small systems in one launch; Sec. 1).  System i:
 * A_dev[i] is n[i] x n[i] fp64 column-major (lda = n[i]), 1 <= n[i] <= 512;
 * it is rounded to u_f = fmt (bf16 / fp16 through fp32) and factored by one
 * thread block with blocking nb, nbo (<= 0: 32, or 16 for fp64, and 64;
 * nb <= 32 (16), nbo a multiple of nb, nbo <= 64).  The bf16 / fp16 outer
 * trailing update is the fp32 fused multiply-add chain in ascending order
 * (no tensor cores).  Outputs, device memory the caller owns: F_dev[i] n x n
 * fp64 row-major, the stored u_f values of L (strictly lower, unit diagonal
 * implied) and U; ipiv_dev[i] n ints, LAPACK-style (row j was swapped with
 * row ipiv[j], 0-based); flags_dev[i] 2 ints: the first zero pivot
 * (1-based, 0: none) and 1 if a stored value is Inf or NaN.  Blocks until
 * done.  MSIR_ERR_INVALID for bad arguments. */
msir_status msir_factor_batched(msir_ctx* ctx, int count, const int* n, const double* const* A_dev, int fmt,
                                int nb, int nbo, double* const* F_dev, int* const* ipiv_dev,
                                int* const* flags_dev);

/* Autotuner of the batched engine's tile shapes: the LU blocking (nb, nbo)
 * that msir_factor_batched and the engine's factorisations use when
 * msir_params.nb / nbo are <= 0.  For u_f in {bf16, fp16, fp32, fp64} and
 * n in {64, 128, 256, 512} it times msir_factor_batched (CUDA events, best
 * of two after a warm-up) on `samples` seeded random matrices for each
 * candidate blocking, nb in {16, 32} (fp64: {8, 16}) x nbo in {32, 64},
 * and keeps the fastest for systems of that size bucket (n <= 64, 128, 256,
 * 512).  With cache_path non-NULL the table is written there, one line per
 * entry keyed by the device name, u_f and the bucket; samples = 0 instead
 * only reads this device's entries from cache_path (MSIR_ERR_INVALID if
 * there are none).  nb_out, nbo_out (16 ints each) and ms_out (16 doubles;
 * 0 when read from a file), may be NULL: the table by [u_f - 1][bucket].
 * The blocking changes the LU's rounding points (the reports state the
 * blocking used).  Blocks until done; device memory about
 * 2 samples * 512^2 * 8 bytes. */
msir_status msir_autotune_batched(msir_ctx* ctx, int samples, const char* cache_path, int* nb_out, int* nbo_out,
                                  double* ms_out);

/* Continuous-batching solve server on the context's device.
 * hbm_budget_bytes: device memory the server may hold (0 = 90% of the free
 * memory).  max_slots: requests in flight on the device at once.  A worker
 * thread admits queued requests into free slots, each on its own stream:
 * a request is admitted when the device memory it needs (its workspace and
 * its A, b, x in the slot) fits the budget.  Among the waiting requests
 * that fit, the one with the fewest rows (the least work) goes first; once
 * the request at the head of the queue (the oldest) has been passed 8
 * times it goes next, waiting for memory to free up if it must.  Slots keep
 * their workspaces between requests and give them back only when a request
 * would not fit otherwise. */
msir_status msir_server_create(msir_ctx* ctx, size_t hbm_budget_bytes, int max_slots,
                               msir_server** out);

/* Queues one request.  A_host (column-major, lda) and b_host are host
 * memory; they are copied into host memory that the server owns before the
 * call returns, and to the device when the request is admitted (inside
 * hbm_budget_bytes).  *ticket receives an id.  Errors: MSIR_ERR_INVALID for
 * bad arguments; MSIR_ERR_BUSY when the requests the server holds already
 * take 64 GiB of host memory, or when a backlog limit is set
 * (msir_server_set_backlog_limit) and the queued work would exceed it;
 * MSIR_ERR_NOMEM when the host copy cannot be allocated.  Nothing is queued
 * on an error. */
msir_status msir_server_submit(msir_server* s, int n, const double* A_host, int lda,
                               const double* b_host, msir_triple t, const msir_params* params,
                               uint64_t* ticket);

/* Admission by expected waiting time (the paper has no counterpart; a
 * serving policy).  With max_backlog_ms > 0, a submission is refused with
 * MSIR_ERR_BUSY when the queued and running requests' work, sum of n^3,
 * divided by the server's recent completion rate (n^3 per ms over its last
 * 32 completed requests) exceeds max_backlog_ms.  Until 4 requests have completed there
 * is no rate and only the host-memory limit applies.  0 (the default)
 * removes the limit.  MSIR_ERR_INVALID for a negative or non-finite value. */
msir_status msir_server_set_backlog_limit(msir_server* s, double max_backlog_ms);

/* Non-blocking poll.  *state: 0 queued, 1 running, 2 done.  When done, x_host
 * (n doubles, may be NULL) and *rep (may be NULL) are filled and the ticket
 * is released; *latency_ms (may be NULL) receives submit-to-done wall time.
 * MSIR_ERR_INVALID for an unknown ticket. */
msir_status msir_server_poll(msir_server* s, uint64_t ticket, int* state, double* x_host,
                             msir_report* rep, double* latency_ms);

/* Stops the worker after the requests in flight finish; frees everything. */
msir_status msir_server_destroy(msir_server* s);

/* Measurement helper; the paper has no counterpart.  Measures the fused
 * multiply-add throughput of device `device` in fmt (FP64 or FP32): one
 * launch of independent fma chains over every SM (iters dependent steps
 * per chain), timed with CUDA events.  *tflops = 2 * fmas / time / 1e12,
 * *seconds = the launch's time.  It is the measured peak that the refinement
 * kernel's fp64 work is compared with.  Blocks until the launch is done;
 * allocates nothing on the device. */
msir_status msir_probe_fma_rate(int device, int fmt, int iters, double* tflops, double* seconds);

/* Arithmetic check; the paper has no counterpart.  The fp64 operator on
 * fp32 data widens operands with integer instructions (the IEEE binary32 ->
 * binary64 field mapping) instead of the hardware conversion.  This runs
 * that widening on all 2^32 fp32 bit patterns on device `device`:
 * *mismatches counts patterns where it differs from the hardware conversion
 * or where its test for subnormal / infinite / NaN input is wrong (0
 * expected); *checked counts the patterns it converted itself.  Blocks; a
 * few milliseconds. */
msir_status msir_probe_widen_check(int device, unsigned long long* mismatches, unsigned long long* checked);

/* Failure-handling check; the paper has no counterpart.  Runs one block
 * into the library's bounded grid-barrier wait for a grid of two blocks, so
 * that the wait can only run out: after limit_s seconds (0 < limit_s <= 10)
 * it records MSIR_ERR_TIMEOUT and the kernel returns, leaving the context
 * usable.  *status receives the recorded code (MSIR_ERR_TIMEOUT expected).
 * Blocks until done; allocates and frees a few bytes of device memory. */
msir_status msir_probe_wait_timeout(int device, double limit_s, int* status);

/* Short text for a status code (static storage). */
const char* msir_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MSIR_H */
