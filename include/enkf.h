/*
 * enkf.h -- C ABI of the GB300 CGD-EnKF analysis-step library (libenkf.so).
 *
 * The library computes one EnKF analysis step (Lee, Liu, Valyou, Zikatanov, "A Conjugate
 * Gradient Formulation of the EnKF Algorithm"):
 *
 *   Z_obs = H X_f,  zbar = Z_obs 1/N,  HA = Z_obs - zbar 1^T            (Sec. 2.3, Eq. Zhat_def)
 *   D     = y 1^T + E - Z_obs                                          (Sec. 2.3; E = 0 is the
 *                                                                       paper's unperturbed form)
 *   S Z   = D,  S = HA HA^T/(N-1) + R  by conjugate gradients, never
 *           forming S: S V = HA (HA^T V)/(N-1) + R V                   (Sec. 3.1-3.3,
 *                                                                       Eq. matvec_decomp)
 *   X_a   = X_f + A (HA^T Z)/(N-1),  A = X_f - xbar 1^T                (Fig. 2, Algorithm 1)
 *
 * and, as the variant ENKF_CGD_REDUCED, Algorithm 2 with the N x N inverse applied by CG
 * (Sec. 5.2): X_a = X_f (I + P^T P)^{-1} [I + P^T L^{-1}((y - zbar) 1^T + E)],
 * P = L^{-1} HA, L L^T = (N-1) R.
 *
 * The variant ENKF_SENKF is the paper's serial-EnKF comparator (Algorithm 3, Appendix A):
 * S^{-1} replaced by the inverse of its diagonal, with no solve,
 *   X_a = X_f + A HA^T diag(HA HA^T + R_N)^{-1} D,  R_N = (N-1) R.
 * It is an approximation of the EnKF analysis, not the same result.
 *
 * Letters: n = state dimension, m = observation count, N = ensemble size (the paper writes
 * m, p, N).
 *
 * Layouts. Every ensemble-shaped array is row-major with the member index fastest:
 * X_f, X_a are [n][N]; E is [m][N]. H is a CSR index-and-weight operator: observation i is
 * sum_{k = rowptr[i]}^{rowptr[i+1]-1} w[k] * x[col[k]]. R is diagonal, given as r[m] > 0.
 * y, r and E are FP64 in every precision mode; X_f / X_a are FP64 in ENKF_FP64 mode and
 * FP32 in every other mode.
 *
 * Ownership and execution. The caller owns X_f, y, E and X_a (device pointers unless the
 * function says "host"). The handle owns H, R and all workspace, allocated once in
 * enkf_create; enkf_analyze* never allocate. Calls are asynchronous and ordered on the
 * stream given at creation; results of an analysis (status, iteration counts, residuals)
 * are read with enkf_get_stats, which synchronises that stream.
 *
 * Errors. No exception crosses this boundary. Argument errors are returned synchronously
 * and nothing is enqueued. Numerical outcomes (not converged, non-finite values, CG
 * breakdown, a device wait that timed out) are recorded on the device and returned by
 * enkf_get_stats; X_a is written in every case. enkf_last_error gives a message for the
 * last failing call on a handle.
 */
#ifndef ENKF_H
#define ENKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct enkf_handle_s* enkf_handle;

typedef enum {
  ENKF_OK = 0,
  ENKF_ERR_INVALID_ARG = 1,   /* bad argument; nothing was enqueued                     */
  ENKF_ERR_CUDA = 2,          /* a CUDA runtime call failed                             */
  ENKF_ERR_OOM = 3,           /* device memory allocation failed in enkf_create         */
  ENKF_ERR_NOT_CONVERGED = 4, /* some column missed the tolerance within max_iter       */
  ENKF_ERR_NONFINITE = 5,     /* a NaN/Inf appeared in the inputs or the recurrences    */
  ENKF_ERR_BREAKDOWN = 6,     /* p^T S p <= 0 in a CG step (S not positive definite)    */
  ENKF_ERR_TIMEOUT = 7,       /* a bounded device-side grid barrier gave up             */
  ENKF_ERR_UNSUPPORTED = 8    /* configuration outside what this build implements       */
} enkf_status;

typedef enum {
  ENKF_FP64 = 0,        /* FP64 storage and arithmetic throughout (the plain FP64 CG)    */
  ENKF_FP32 = 1,        /* FP32 CG inner solves + double-float (FP32-pair, about 44-bit)
                           residual refresh (iterative refinement) with FP64 scalar
                           recurrences                                                   */
  ENKF_BF16_REFINE = 2, /* BF16 HA contractions on tensor cores (tcgen05), FP32
                           accumulation, FP32 vectors, FP64 scalars; inner solves refined
                           by the same double-float residual refresh (see refresh_every) */
  ENKF_FP16_REFINE = 3  /* as ENKF_BF16_REFINE with FP16 HA; the tensor-core images of HA
                           are scaled by the power of two that brings the largest |HA| of
                           the analysis into [2^13, 2^14) and the products are scaled back
                           exactly; the Gram's z operand is normalised by ||r|| and, with
                           precondition = 1, by the power of two nearest the geometric mean
                           of r_diag: the mode works in any units of the state and of R
                           without FP16 overflow or subnormal loss                        */
} enkf_precision;

typedef enum {
  ENKF_CGD = 0,         /* CGD-EnKF: CG on S Z = D (m x m operator, N columns)           */
  ENKF_CGD_REDUCED = 1, /* CGD-EnKF-Reduced: CG on I + P^T P (N x N, N columns)          */
  ENKF_SENKF = 2        /* sEnKF comparator (Algorithm 3): diagonal inverse, no solve;
                           ENKF_FP64 or ENKF_FP32, no warm start                         */
} enkf_variant;

typedef struct enkf_config {
  int64_t n;              /* state dimension, >= 1                                       */
  int64_t m;              /* observation count, >= 1                                     */
  int32_t N;              /* ensemble size, 2 <= N <= 128                                */
  int32_t precision;      /* enkf_precision                                              */
  int32_t variant;        /* enkf_variant                                                */
  int32_t max_iter;       /* cap on CG iterations per column (inner iterations summed)   */
  double tol;             /* stop column j when ||r_j||_2 <= tol * ||d_j||_2             */
  int32_t fixed_iters;    /* > 0: run exactly this many CG steps (the paper's Tables 4-5
                             mode); tol is then ignored                                  */
  int32_t max_refine;     /* ENKF_FP32: maximum double-float residual refreshes (default
                             4). The tensor-core modes refresh until every column has
                             converged, stalled (no halving over a cycle) or turned
                             non-finite; each refresh follows at least one CG step, so
                             max_iter bounds them                                         */
  double inner_tol;       /* FP32, BF16 and FP16 modes: relative tolerance of each inner
                             solve (default 1e-5); the tensor-core modes raise it to the
                             floor their operator allows (see refresh_every)              */
  int32_t refresh_every;  /* BF16/FP16 modes: cap on CG steps between double-float residual
                             refreshes; 0 (default): each inner solve runs until its
                             residual fell by inner_tol, but not below what the operator
                             allows: 3e-5 for split FP16 with N <= 64, 1e-3 for the other
                             split forms, 2e-2 / 4e-3 for single BF16 / FP16 operands   */
  int32_t perturb_obs;    /* 1: E ~ N(0, R) drawn from (seed, counter); 0: E = 0         */
  int32_t warm_start;     /* 0: start CG from Z = 0; 1: learned warm start from the model
                             attached by enkf_set_warm_model (ENKF_CGD, ENKF_FP32 only) */
  int32_t true_residual;  /* 1: FP64 true residual check (and W = HA^T Z/(N-1) from the
                             final Z) after an FP64 solve; always on in ENKF_FP32        */
  int32_t grid_blocks;    /* 0: automatic persistent-grid size; > 0: use this many CTAs  */
  int32_t precondition;   /* ENKF_CGD: 0 plain CG (the paper's method); 1 CG preconditioned
                             by R (Jacobi), which ends within about N steps because
                             R^-1/2 S R^-1/2 is the identity plus a rank < N term        */
  int32_t lowprec_terms;  /* BF16/FP16 modes: 3 (or 0, the default) splits every operand
                             into hi + lo parts and forms hi*hi + hi*lo + lo*hi (about 16
                             significant bits); 1 uses single BF16/FP16 operands, whose
                             refinement diverges once 2 eps cond(S) > 1                  */
  int32_t warm_accept;    /* learned warm start, how its start is judged by the start's
                             true residual B_j = d_j - S z0_j: 0 (default) a column whose
                             ||B_j|| exceeds ||d_j|| (the zero start's) starts from zero;
                             1 every finite start is kept. Either way a non-finite start
                             starts from zero and the result is certified by the same
                             double-float true residual <= tol                          */
  int32_t reduce_order;   /* 0 (default): every step's column sums and Gram are summed over
                             the CTAs in a fixed order (bitwise repeatable results, two
                             grid barriers per step); 1: ENKF_CGD in the FP32, BF16 and
                             FP16 modes with N <= 64 adds them into the total by
                             atomic adds (one barrier per step, the
                             last bits of the sums depend on the order in which the CTAs
                             arrive, so results can differ from run to run in the last
                             bits; the result is still certified by the double-float true
                             residual <= tol); ignored by the other modes               */
  int32_t reserved[3];    /* must be zero                                                */
} enkf_config;

typedef struct enkf_stats {
  int32_t status;            /* enkf_status of the last analysis                         */
  int32_t iters_max;         /* max over columns of CG iterations                        */
  int32_t iters_min;         /* min over columns of CG iterations                        */
  int32_t refinements;       /* residual refreshes performed (FP64 in ENKF_FP64 mode,
                                double-float in the other modes)                         */
  double relres_max;         /* max over columns of the recursive ||r_j|| / ||d_j||      */
  double true_relres_max;    /* max over columns of the FP64 true residual
                                ||d_j - S z_j|| / ||d_j||; -1 when not computed          */
  int32_t columns_converged; /* columns that met tol                                     */
  int32_t grid_blocks;       /* persistent-grid size used                                */
  double warm_relres_max;    /* learned warm start: max over columns of the start's
                                relative residual ||d_j - S z0_j|| / ||d_j|| (evaluated in
                                FP32 through the N x N identity below); -1 if off         */
  double warm_fallbacks;     /* columns whose start was rejected (non-finite, or a true
                                residual larger than the zero start's) and began at 0    */
  double reserved[2];
} enkf_stats;

/* Fill *cfg with defaults for an (n, m, N) problem: ENKF_FP64, ENKF_CGD, tol 1e-8,
   max_iter 1000, max_refine 4, inner_tol 1e-5, refresh_every 0, perturb_obs 1,
   true_residual 1. Returns ENKF_ERR_INVALID_ARG when cfg is NULL. */
enkf_status enkf_config_default(enkf_config* cfg, int64_t n, int64_t m, int32_t N);

/* Create a handle for one problem shape. h_rowptr[m+1], h_col[nnz], h_w[nnz] (the CSR
   observation operator, nnz = h_rowptr[m]) and r_diag[m] (> 0, finite) are HOST arrays
   and are copied to the device. cuda_stream is a cudaStream_t (NULL: the legacy default
   stream); every later call on the handle is ordered on it. Allocates all workspace
   (about 56 m N + 4 n N bytes in ENKF_FP32 mode, 4 m N more in the tensor-core modes,
   48 m N + 8 n N in ENKF_FP64 mode, plus O(grid N^2); ENKF_CGD_REDUCED and ENKF_SENKF keep
   no m x N arrays: 4 or 8 n N bytes plus O(grid N^2)). Errors: ENKF_ERR_INVALID_ARG (bad
   shape, column index outside [0, n), decreasing rowptr, r <= 0), ENKF_ERR_UNSUPPORTED
   (N > 128, unknown precision or variant, a variant other than ENKF_CGD in the BF16/FP16
   modes), ENKF_ERR_OOM, ENKF_ERR_CUDA. *out is NULL on error. */
enkf_status enkf_create(const enkf_config* cfg, const int32_t* h_rowptr, const int32_t* h_col,
                        const double* h_w, const double* r_diag, void* cuda_stream,
                        enkf_handle* out);

/* As enkf_create with a symmetric tridiagonal R (the observation-noise model of the paper's
   Example 2, Sec. 6.2, whose factorisation costs are discussed in Sec. 5.3): R_ii = r_diag[i]
   and R_{i,i+1} = R_{i+1,i} = r_off[i] (HOST, m - 1 entries, finite; NULL only when m = 1).
   R must be positive definite (ENKF_ERR_INVALID_ARG otherwise, checked through its banded
   Cholesky factor R = L L^T, L lower bidiagonal). ENKF_CGD_REDUCED and ENKF_CGD with
   precondition = 1 (CG preconditioned by R) analyse the whitened problem X' = L^{-1} HA,
   y' = L^{-1}(y - zbar), E' = L^{-1} E with H' = I and R' = I, which is exactly Algorithm 2
   (P = L_N^{-1} HA) and CG on L^{-1} S L^{-T}; the update uses the caller's X_f, and the
   perturbations drawn in an analysis are E = L xi (xi the same standard normals as with a
   diagonal R). The stopping rule, the reported residuals and enkf_copy_intermediates
   (HA, D, Z) are those of the whitened system (Z' = L^T Z; W is unchanged). ENKF_SENKF uses
   only the diagonal of R (Algorithm 3). ENKF_CGD with precondition = 0 is
   ENKF_ERR_UNSUPPORTED with a tridiagonal R. Allocates about 24 m N bytes more than
   enkf_create (the whitened rows and their scan buffers). */
enkf_status enkf_create_tridiag(const enkf_config* cfg, const int32_t* h_rowptr, const int32_t* h_col,
                                const double* h_w, const double* r_diag, const double* r_off,
                                void* cuda_stream, enkf_handle* out);

/* One analysis on the handle's stream. d_Xf: device [n][N] (FP64 in ENKF_FP64 mode, FP32
   otherwise); d_y: device [m] FP64; (seed, counter) select the Philox4x32-10 stream of the
   perturbations E when cfg.perturb_obs = 1 (element (i, j) uses counter
   (i, j >> 1, counter_lo, counter_hi) and key (seed_lo, seed_hi); two 53-bit uniforms and
   Box-Muller give the normal, E_ij = sqrt(r_i) * normal; ENKF_FP64 evaluates Box-Muller in
   FP64, the FP32 and tensor-core modes (every variant) in FP32 from the same uniforms,
   within about 1e-7 of the FP64 normal). d_Xa: device [n][N], same dtype
   as d_Xf; d_Xa == d_Xf (in-place) is allowed, partial overlap is not. Never allocates. */
enkf_status enkf_analyze(enkf_handle h, const void* d_Xf, const double* d_y, uint64_t seed,
                         uint64_t counter, void* d_Xa);

/* As enkf_analyze with the perturbations given explicitly: d_E device [m][N] FP64
   (NULL means E = 0, the paper's unperturbed EnKF). */
enkf_status enkf_analyze_with_E(enkf_handle h, const void* d_Xf, const double* d_y,
                                const double* d_E, void* d_Xa);

/* End-to-end form with HOST buffers: h_Xf [n][N], h_y [m], h_Xa [n][N] (h_Xa == h_Xf is
   allowed); the result is in h_Xa when the call returns (it synchronises the stream).
   Pageable buffers: X_f and y are copied to device staging buffers owned by the handle, the
   analysis runs there and X_a is copied back. Pinned (page-locked, device-mapped) buffers
   with ENKF_CGD: the innovations read the observed rows of X_f directly from host memory
   while the whole X_f is uploaded on a second stream that the handle creates on first use
   (the upload overlaps the innovations and the solve; only the final update waits for it),
   and the update writes a pinned h_Xa directly (else X_a comes back by one copy). Either way
   every X_f byte crosses to the device and every X_a byte back within the call. The
   buffers must hold n N elements of the handle's dtype; the result is the same as
   enkf_analyze's on device copies of the inputs. */
enkf_status enkf_analyze_host(enkf_handle h, const void* h_Xf, const double* h_y,
                              uint64_t seed, uint64_t counter, void* h_Xa);

/* Synchronise the handle's stream and return the last analysis's outcome in *out. The
   return value is out->status. */
enkf_status enkf_get_stats(enkf_handle h, enkf_stats* out);

/* Synchronise and copy per-column results to HOST arrays of length N (any may be NULL):
   CG iterations, recursive relative residual, FP64 true relative residual (-1 if not
   computed). */
enkf_status enkf_get_column_stats(enkf_handle h, int32_t* iters, double* relres,
                                  double* true_relres);

/* Copy the last analysis's intermediate results to DEVICE buffers (any may be NULL):
   d_HA [m][N] and d_D [m][N] (FP64), d_Z [m][N] (FP64 solution of S Z = D), d_W [N][N]
   (FP64, W = HA^T Z/(N-1)). In the FP32 and tensor-core modes HA and Z are the solve's
   double-float arrays (FP32 pairs, about 48 significant bits) widened to FP64. For
   ENKF_CGD_REDUCED, d_HA and d_D must be NULL (that variant never stores them), d_Z receives
   the N x N CG solution V and d_W the N x N matrix G = I + P^T P. For ENKF_SENKF only d_W
   may be non-NULL: it receives W = HA^T diag(HA HA^T + R_N)^{-1} D (X_a = X_f + A W).
   Enqueued on the handle's stream. */
enkf_status enkf_copy_intermediates(enkf_handle h, double* d_HA, double* d_D, double* d_Z,
                                    double* d_W);

/* Draw the observation perturbations exactly as enkf_analyze does in ENKF_FP64 mode (the
   FP32 and tensor-core modes draw the same normals in single precision): d_r device [m]
   FP64, d_E device [m][N] FP64 output, on cuda_stream. */
enkf_status enkf_draw_perturbations(uint64_t seed, uint64_t counter, const double* d_r,
                                    int64_t m, int32_t N, double* d_E, void* cuda_stream);

/* Per-kernel timing of later analyses (enable != 0) with CUDA events recorded on the
   handle's stream around the three kernels of an analysis; off by default. Creating the
   events happens here, not in the analysis calls. enable >= 2 also turns on in-kernel phase
   timers of the persistent solve (read with enkf_get_solve_phases). */
enkf_status enkf_set_phase_timing(enkf_handle h, int32_t enable);

/* Synchronise and return the last timed analysis's kernel durations in milliseconds:
   ms[0] innovations (gather, anomalies, perturbations), ms[1] the persistent CG solve,
   ms[2] the ensemble update. For ENKF_CGD_REDUCED and ENKF_SENKF, ms[0] is the Gram pass
   over the observation rows (gather, anomalies and perturbations included) and ms[1] the
   N x N stage (Reduced: the sums and the N x N CG; sEnKF: the sum of the partials).
   ENKF_ERR_INVALID_ARG if timing is off or nothing was timed. */
enkf_status enkf_get_phase_times(enkf_handle h, float* ms);

/* Synchronise and return the in-kernel phase timers of the last timed solve, measured by
   CTA 0 with the global nanosecond timer, in microseconds: us[0] set-up reductions,
   us[1] fused CG passes, us[2] first grid barrier, us[3] cross-CTA reduction, us[4] second
   grid barrier, us[5] scalar recurrences and staging, us[6] FP64 refreshes, us[7] unused.
   ENKF_ERR_INVALID_ARG unless enkf_set_phase_timing(h, 2) preceded a timed analysis. */
enkf_status enkf_get_solve_phases(enkf_handle h, double* us);

/* One analysis step that allocates no device memory, for callers that cannot call
   cudaMalloc when they need it: code running while a stream is captured into a CUDA graph,
   applications whose own pool allocator owns all device memory, real-time assimilation
   loops that forbid allocation after start-up. The paper has no counterpart; this is a
   deployment form of enkf_create + enkf_analyze + enkf_get_stats without a handle.
   Inputs and outputs are as for enkf_create / enkf_analyze, except that the observation
   operator and R are DEVICE arrays here (d_rowptr[m+1], d_col[nnz], d_w[nnz], d_r[m] > 0;
   they are not validated, so the caller guarantees 0 <= col < n and r > 0), and cfg must
   use ENKF_CGD with ENKF_FP64 or ENKF_FP32. All working memory lives in one fixed 16 MiB
   array in the library's device memory (held by every GPU that loads the library until the
   process exits); problems whose working memory (about 48 m N bytes in FP64 mode, 56 m N in
   FP32 mode, plus the CG partials) exceeds it are rejected with ENKF_ERR_UNSUPPORTED before
   anything is enqueued. X_a == X_f is allowed; a partial overlap is ENKF_ERR_INVALID_ARG.
   The first call on each device looks up the array's device
   address; make that first call before any stream capture. Every call shares the array, so
   calls that may overlap on the GPU (different streams, or different host threads without
   ordering) race and must be serialised by the caller. If out_stats (HOST) is non-NULL the
   call synchronises the stream, fills it, and returns out_stats->status. */
enkf_status enkf_analyze_noalloc(const enkf_config* cfg, const int32_t* d_rowptr,
                                 const int32_t* d_col, const double* d_w, const double* d_r,
                                 const void* d_Xf, const double* d_y, uint64_t seed,
                                 uint64_t counter, void* d_Xa, void* cuda_stream,
                                 enkf_stats* out_stats);

/* ---------------------------------------------------------------- batched analyses
   Many independent analyses of uneven shape (n, m, N differ per problem) in ONE persistent
   cooperative kernel launch, replayed from a CUDA graph. The paper analyses one problem at
   a time; this is the same per-problem computation (innovations, the CG solve of S Z = D with
   the matrix-free product, X_a = X_f + A HA^T Z / (N - 1)) scheduled for throughput. Every
   problem uses ENKF_CGD in ENKF_FP32 with precondition = 1 (Jacobi by R), fixed_iters = 0,
   and the same perturb_obs. A batched handle accepts only the enkf_batch_* calls,
   enkf_last_error and enkf_destroy; the single-analysis calls reject it with
   ENKF_ERR_INVALID_ARG. */

/* Create a batched handle for `count` problems. cfgs[count] are HOST configs, each checked
   as by enkf_create; h_rowptr, h_col, h_w and r_diag are HOST arrays of `count` HOST
   pointers to each problem's CSR operator and R diagonal (copied to the device). cfgs[0]
   .grid_blocks > 0 caps the persistent grid. Allocates one device arena (about 56 m N bytes
   per problem, plus O(grid N_max^2)) and plans the launch as enkf_batch_plan does with
   alpha = 1 (large problems get teams of CTAs, the rest are queued for single CTAs). If the
   environment variable ENKF_TUNE_CACHE names a file holding a tuning result for this batch
   (written by enkf_batch_tune), that plan is used. Errors as enkf_create, with the index of
   the failing problem in enkf_last_error(NULL). */
enkf_status enkf_batch_create(int32_t count, const enkf_config* cfgs,
                              const int32_t* const* h_rowptr, const int32_t* const* h_col,
                              const double* const* h_w, const double* const* r_diag,
                              void* cuda_stream, enkf_handle* out);

/* One batched analysis on the handle's stream. d_Xf, d_y, d_Xa are HOST arrays of `count`
   DEVICE pointers: X_f [n_i][N_i] FP32, y [m_i] FP64, X_a [n_i][N_i] FP32 (X_a == X_f is
   allowed, partial overlap is not). seeds / counters (HOST arrays of `count`, NULL means
   0) select each problem's perturbation stream exactly as enkf_analyze does. The pointer
   table is copied to the device only when it differs from the previous call's. The first
   call after create (or after a plan change) captures the launch into a CUDA graph; make
   it before any capture of the caller's own. Never allocates device memory after that. */
enkf_status enkf_batch_analyze(enkf_handle h, const void* const* d_Xf, const double* const* d_y,
                               const uint64_t* seeds, const uint64_t* counters, void* const* d_Xa);

/* Autotune the plan on real inputs (arguments as enkf_batch_analyze). First it times the
   plans of enkf_batch_plan for the team-scaling exponents alpha in {1, 0.9, 0.8}; then,
   starting from the alpha = 1 plan and, if another alpha was faster, from that plan too, it
   four times re-plans from measured costs (each problem's duration in the last plan, as
   reported by enkf_batch_get_times and averaged over that plan's three timed analyses, times
   k^alpha for a team of k CTAs, averaged with the previous round's estimate) and times that
   plan. Last it searches the row-block floor of each ensemble-size class (N <= 16, <= 32,
   <= 64, <= 128; the fewest rows a team's CTA may get, 64 by default, which caps a problem's
   team at ceil(m / floor) CTAs): classes with at least 5 % of the cost, the largest first,
   each floor in {128, 256, 512} planned from the best plan's costs and, where the plan
   changes, timed, keeping a floor that is at least 1 % faster. It keeps the fastest plan
   and appends it (alpha, the floors, and the measured costs when a measured plan won) to the
   ENKF_TUNE_CACHE file if that variable is set. Runs 28 to 92 analyses (X_a holds the last
   one's result); synchronises the stream. *best_ms (HOST, may be NULL) receives the best
   mean time. */
enkf_status enkf_batch_tune(enkf_handle h, const void* const* d_Xf, const double* const* d_y,
                            const uint64_t* seeds, const uint64_t* counters, void* const* d_Xa,
                            double* best_ms);

/* Synchronise and report the last batched analysis per problem into HOST arrays of length
   count (any may be NULL): enkf_status, max CG iterations over columns, max recursive
   relative residual, refreshes performed. Returns the first problem's non-OK status, or
   ENKF_OK. */
enkf_status enkf_batch_get_stats(enkf_handle h, int32_t* status, int32_t* iters_max,
                                 double* relres_max, int32_t* refinements);

/* The handle's current plan: persistent grid size, number of teams, team sizing alpha, and
   whether analyses replay a CUDA graph (1) or launch directly because capture was refused
   (0; checked at the first analysis) (HOST outputs, any may be NULL). */
enkf_status enkf_batch_get_plan(enkf_handle h, int32_t* grid, int32_t* teams, double* alpha,
                                int32_t* graphed);

/* The row-block floors of the handle's current plan, per ensemble-size class N <= 16, <= 32,
   <= 64, <= 128 (HOST array of 4; see enkf_batch_tune). */
enkf_status enkf_batch_get_row_floors(enkf_handle h, int32_t* row_floors);

/* Per-problem phase timers in later batched analyses (enable != 0) or not (0, the default):
   the first CTA of each team reads the global nanosecond timer around the phases of the CG
   solve, as enkf_get_solve_phases does for one analysis. Re-uploads the problem table and
   re-captures the graph at the next analysis; synchronises the stream. */
enkf_status enkf_batch_set_phase_timing(enkf_handle h, int32_t enable);

/* Synchronise and report when each problem of the last batched analysis ran, into HOST
   arrays of `count` entries (any may be NULL): start_us / end_us, microseconds from the
   earliest start to the moment the first CTA of the problem's team began it (before the
   innovations) and finished it (after its share of the update; -1 if it never finished);
   phase_us [count][8] the solve phase timers in the order of enkf_get_solve_phases (only
   while enkf_batch_set_phase_timing is on, else ENKF_ERR_INVALID_ARG); team_size the number
   of CTAs in the team that ran each problem. The start and end stamps are always taken
   (two timer reads per problem). ENKF_ERR_INVALID_ARG before the first analysis. */
enkf_status enkf_batch_get_times(enkf_handle h, double* start_us, double* end_us, double* phase_us,
                                 int32_t* team_size);

/* Self-test of the failure detection (the paper has no counterpart): run one of the bounded
   device waits on a condition that nothing ever satisfies, with a time limit of timeout_ms
   (0 < timeout_ms <= 10,000) instead of the library's 4 s. which = 0: the grid barrier of
   the persistent kernels, entered by one CTA of a two-CTA barrier; which = 1: the mbarrier
   wait of the tensor-core kernels on a barrier nothing arrives on. Synchronises cuda_stream.
   Returns ENKF_ERR_TIMEOUT when the wait ended at its limit and raised the timeout status, as
   it must (the context stays usable); ENKF_ERR_CUDA if it was released or reported nothing;
   ENKF_ERR_INVALID_ARG for bad arguments. Allocates 16 bytes of device memory per call. */
enkf_status enkf_selftest_wait_timeout(int32_t which, double timeout_ms, void* cuda_stream);

/* The planner alone, on the host (no GPU needed). A problem costs c = m N^2 (N + 8) + 2 n N^2;
   a team of k CTAs is estimated to take c / k^alpha (0 < alpha <= 1). For a target makespan
   T every problem with c > T gets the smallest team (2 <= k <= ceil(m / floor)) that meets T,
   floor = row_floors[class of N] (classes N <= 16, <= 32, <= 64, <= 128; HOST array of 4, or
   NULL for 64 rows in every class);
   the others form a shared queue, longest first, from which the launch hands the next
   problem to whichever CTA is free (the CTAs outside teams from the start, a team's CTAs
   once its problem is done), each solving it alone; T must hold for that schedule too. The
   plan is the one for the smallest feasible T (bisection); CTAs the queue cannot keep busy
   join the slowest teams. For `count` problem shapes (only n, m, N of cfgs are read) and a
   grid of at most max_grid CTAs, fill HOST arrays cta_team[grid], cta_rank[grid] (team of
   each CTA and its rank in it; a team's CTAs are contiguous), team_size[teams],
   team_first[teams + 1] (offsets into order; a team of one CTA has an empty list) and
   order[count] (every problem exactly once: the teams' problems, then from
   order[team_first[teams]] on the queue). Arrays of max_grid, max_grid, max_grid,
   max_grid + 1 and count entries are always large enough; any may be NULL. *grid and *teams
   receive the sizes. ENKF_ERR_INVALID_ARG for alpha outside (0, 1], a floor < 1 or bad
   shapes. */
enkf_status enkf_batch_plan(int32_t count, const enkf_config* cfgs, int32_t max_grid, double alpha,
                            const int32_t* row_floors, int32_t* cta_team, int32_t* cta_rank,
                            int32_t* team_size, int32_t* team_first, int32_t* order, int32_t* grid,
                            int32_t* teams);

/* ---------------------------------------------------------------- learned warm start
   The paper's CG starts from zero. Every solution column of S Z = D has the form
   z_j = R^{-1}(d_j - HA c_j) with c_j = W e_j, W = HA^T Z/(N-1) (rearranging S Z = D), so a
   small MLP predicts c_j per column from features f_j = [d_j(sketch)/s_j, g_j/s_j]: a
   sketch of K rows i_k = floor(k m / K), s_j the RMS of d_j over the sketch (1 if 0),
   g_j = HA^T R^{-1} d_j/(N-1). The prediction is decoded into the start
   z0_j = R^{-1}(d_j - HA c_j), whose residual is HA e_j with
   e_j = c_j + (HA^T R^{-1} HA c_j - HA^T R^{-1} d_j)/(N-1) (so no extra pass over S is needed);
   a column whose start residual is non-finite or larger than that of z_j = 0 (that is, ||d_j||)
   starts from 0 instead. The refreshes of the solve then measure the true residual as usual. The network: inputs standardised per feature, `layers` hidden layers of
   width `hidden` with GELU (x Phi(x)), linear output of the standardised c_j/s_j; trained
   with mean squared error and Adam (Kingma & Ba 2015). All of it runs in this library's
   kernels (FP32). */
typedef struct enkf_mlp_shape {
  int32_t in_dim;   /* K + N                     */
  int32_t hidden;   /* hidden width (e.g. 512)   */
  int32_t layers;   /* hidden layers, 1..7       */
  int32_t out_dim;  /* N                         */
} enkf_mlp_shape;

/* Number of FP32 parameters. Layout: for each layer (hidden layers, then the output) the
   weight [out][in] row-major followed by the bias [out]; then mu_in [in_dim], sd_in [in_dim],
   mu_out [out_dim], sd_out [out_dim] (standardisation, set by enkf_mlp_standardize, not
   trained). The trained prefix is the count minus 2 (in_dim + out_dim). -1 for a bad shape. */
int64_t enkf_mlp_param_count(const enkf_mlp_shape* shape);

/* Device scratch bytes the MLP calls need for `batch` rows (-1 for bad arguments). */
int64_t enkf_mlp_work_bytes(const enkf_mlp_shape* shape, int32_t batch);

/* Y [batch][out_dim] = mu_out + sd_out * MLP((X[rows[b]] - mu_in) / sd_in), all DEVICE FP32
   (d_rows: DEVICE int32 [batch] row indices into X, NULL for rows 0..batch-1); d_work of
   enkf_mlp_work_bytes(shape, batch) bytes. Enqueued on cuda_stream. */
enkf_status enkf_mlp_forward(const enkf_mlp_shape* shape, const float* d_params, const float* d_X,
                             const int32_t* d_rows, int32_t batch, float* d_Y, void* d_work,
                             void* cuda_stream);

/* Loss L = mean over the batch x out_dim entries of (y_std - (T[rows[b]] - mu_out)/sd_out)^2
   into d_loss (DEVICE float, may be NULL) and its gradient into d_grad (DEVICE, the trained
   prefix of the parameter layout is overwritten). Enqueued on cuda_stream. */
enkf_status enkf_mlp_loss_grad(const enkf_mlp_shape* shape, const float* d_params, const float* d_X,
                               const float* d_T, const int32_t* d_rows, int32_t batch,
                               float* d_grad, float* d_loss, void* d_work, void* cuda_stream);

/* One Adam step (Kingma & Ba 2015, Algorithm 1, with bias correction at step >= 1) on the
   first `count` entries of d_params with gradient d_grad and moments d_m, d_v (DEVICE FP32,
   zero before step 1). */
enkf_status enkf_mlp_adam(int64_t count, float* d_params, const float* d_grad, float* d_m,
                          float* d_v, int32_t step, float lr, float beta1, float beta2, float eps,
                          void* cuda_stream);

/* One training epoch: for each of floor(rows / batch) minibatches (rows d_perm[q batch ..]
   of d_X [rows][in_dim] and d_T [rows][out_dim]) a loss/gradient pass and an Adam step
   (lr, beta1 0.9, beta2 0.999, eps 1e-8, step numbers step0 + 1, ...). d_losses (DEVICE,
   may be NULL) receives each minibatch's loss; d_grad holds param_count floats; d_work
   enkf_mlp_work_bytes(shape, batch) bytes. */
enkf_status enkf_mlp_train_epoch(const enkf_mlp_shape* shape, float* d_params, float* d_m, float* d_v,
                                 const float* d_X, const float* d_T, const int32_t* d_perm,
                                 int64_t rows, int32_t batch, int32_t step0, float lr,
                                 float* d_losses, float* d_grad, void* d_work, void* cuda_stream);

/* Set the standardisation entries of d_params to the per-column mean and standard
   deviation (population form, 1 where 0) of d_X [rows][in_dim] and d_T [rows][out_dim]. */
enkf_status enkf_mlp_standardize(const enkf_mlp_shape* shape, float* d_params, const float* d_X,
                                 const float* d_T, int64_t rows, void* cuda_stream);

/* Training pairs from the handle's last analysis (ENKF_CGD, ENKF_FP32): d_F [N][K + N]
   features of its N innovation columns for a sketch of K >= 1 rows and, if d_T is not NULL,
   d_T [N][N] the targets c_j / s_j with c_j = W e_j of the solve (DEVICE FP32). */
enkf_status enkf_warm_features(enkf_handle h, int32_t K, float* d_F, float* d_T);

/* Attach a model to the handle (d_params DEVICE, caller-owned, must stay valid while
   analyses with cfg.warm_start = 1 run; NULL detaches). shape->out_dim must be N and
   in_dim = K + N. Allocates the handle's feature and activation buffers (analyses allocate
   nothing). */
enkf_status enkf_set_warm_model(enkf_handle h, const enkf_mlp_shape* shape, const float* d_params);

/* Release the handle and all device memory it owns (synchronises its stream first).
   NULL is accepted. */
enkf_status enkf_destroy(enkf_handle h);

/* Static description of a status code. */
const char* enkf_status_str(enkf_status s);

/* Message for the last failing call on h (h == NULL: the last failing enkf_create on the
   calling thread). Valid until the next call on h. */
const char* enkf_last_error(enkf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* ENKF_H */
