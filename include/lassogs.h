/*
 * lassogs -- Lasso paths by cyclic coordinate descent with GAP SAFE sphere
 * screening on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Fercoq, Gramfort, Salmon, "Mind the duality gap: safer rules for
 * the Lasso", ICML 2015 (arXiv:1505.03410).  The solver is Algorithm 1 of
 * Sec. 4.1: coordinate descent over the safe-active set, a GAP SAFE sphere
 * check (Eq. (10)) every f passes, warm starts along the geometric grid of
 * Sec. 3.3, stop when the duality gap (Sec. 3.2) is <= eps.
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are device pointers (global memory of the current
 *     CUDA device); pointers named *_host are host pointers.
 *   - The caller owns every buffer.  The library allocates no memory: the
 *     scratch it needs is the caller-provided workspace, whose size is given
 *     by the matching *_workspace_size function.
 *   - Designs are column-major: element (i, j) of X is X[i + j*ldx].
 *   - Calls that take a stream enqueue their work on it and return without
 *     waiting; results are valid once the stream has been synchronised.
 *     The return value reports argument and launch errors only.  Per-lambda
 *     convergence and device-side errors are written into the stats records.
 *   - No call aborts, exits or traps.  On error the call returns a non-zero
 *     lasso_status and lasso_last_error() describes it (thread-local).
 *   - The mask of safe-active features uses one bit per feature: bit (j % 32)
 *     of 32-bit word j / 32; words = ceil(p / 32).
 */
#ifndef LASSOGS_H
#define LASSOGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LASSOGS_ABI_VERSION 1

typedef enum lasso_status {
  LASSO_OK = 0,
  LASSO_ERR_INVALID_ARG = 1,  /* a size, pointer, alignment or option is invalid */
  LASSO_ERR_NONFINITE = 2,    /* X or y holds NaN or Inf (detected by the precompute) */
  LASSO_ERR_WORKSPACE = 3,    /* workspace NULL, misaligned or smaller than required */
  LASSO_ERR_CUDA = 4,         /* a CUDA runtime call failed (message in lasso_last_error) */
  LASSO_ERR_NOT_CONVERGED = 5,/* a lambda reached the pass cap K before gap <= eps */
  LASSO_ERR_TIMEOUT = 6       /* a device-side wait hit its time limit (never expected) */
} lasso_status;

typedef enum lasso_dtype {
  LASSO_F64 = 0,   /* IEEE binary64.  lasso_path splits an FP64 design once into two FP32
                      planes (x = hi + lo), so X enters the solver with about 48 significand
                      bits, not 53; y and the objectives stay FP64 */
  LASSO_F32 = 1,   /* IEEE binary32 */
  LASSO_BF16 = 2   /* bfloat16 */
} lasso_dtype;

/* Solver options.  Fill with lasso_default_opts() and override fields. */
typedef struct lasso_opts {
  int32_t screen_period; /* f: passes between two GAP SAFE checks (Sec. 4.1 uses 10); >= 1 */
  int32_t dual_point;    /* 0: theta = rho / max(lambda, ||X^T rho||_inf) (default);
                            1: the clipped optimal scaling of Eq. (8) */
  int32_t xtr_scope;     /* 0: X^T rho over all p features at every check (default);
                            1: over the safe-active features only (the O(nq) check of Sec. 4.1) */
  int32_t warm_start;    /* 1: beta carried from lambda_{t-1} to lambda_t (Sec. 3.3, default);
                            0: every lambda starts from beta0 (or 0) */
  int64_t max_epochs;    /* K: passes allowed per lambda (Algorithm 1 INPUT), default 100000 */
  double gap_tol_rel;    /* eps / ||y||^2: stop when gap <= gap_tol_rel * ||y||^2, default 1e-6 */
  int32_t gemm_dtype;    /* batched solver: input type of the tensor-core X^T R product at the
                            first check of each lambda (LASSO_BF16 default; LASSO_F32 = exact
                            CUDA-core product); ignored by lasso_path */
  int32_t batch_ctas_per_sm; /* batched solver: resident CTAs per SM, 1 or 2 (0 = 2, the default).
                                With 1 the kernel may use up to 255 registers per thread */
  int32_t gemm_tile_n;   /* lockstep batches: N tile of the tensor-core product, 64, 128 or 256
                            (0 = 128) */
  int32_t batch_group;   /* batched solver with gemm_dtype = LASSO_F32: CTAs per problem, 1..64
                            (0 = 1).  A group solves its problem as lasso_path does with the
                            grid: feature slices per CTA, and, when the group has more than
                            ceil(n/256) CTAs, the coordinate chain in Gram form (a cache of
                            x_i^T x_k over the support per group, at most max(512, n) features).
                            lasso_batch_tune picks this, batch_ctas_per_sm, gemm_tile_n and
                            gemm_dtype */
  int32_t screen_rule;   /* 0: GAP SAFE sphere, Eq. (10) (default); 1: sphere and GAP SAFE dome,
                            Eq. (11) with the appendix's parameters: a feature is screened when
                            either test screens it.  The dome lies inside the sphere, so it screens
                            at least as much; each check then evaluates x_j^T rho exactly for the
                            features the sphere keeps */
  int32_t refined_radius; /* 0: sphere radius sqrt(2 gap)/lambda, Eq. (10) (default); 1: the radius
                            of Thm. 2, (R^2 - r(beta)^2)^(1/2) with R = ||theta - y/lambda||, which
                            is the smaller of sqrt(2 gap)/lambda and R; it differs only for iterates
                            whose primal value exceeds P(0) = ||y||^2/2 (a poor starting point) */
  double enet_alpha;     /* a in (0, 1]: 1 is the Lasso (default).  Below 1, lasso_path solves the
                            Elastic-Net 1/2 ||X beta - y||^2 + lambda a ||beta||_1
                            + lambda (1 - a)/2 ||beta||^2 (the paper's appendix) as the Lasso on
                            [X; sqrt((1 - a) lambda) I], [y; 0] with penalty a lambda, the augmented
                            rows implicit; lambda_max = ||X^T y||_inf / a and the stats report lambda.
                            Both solvers, both design types and both screening rules take it (the
                            dome is then the dome of the augmented problem) */
  int32_t audit_bounds;  /* 0: off (default).  1: every check also computes x_j^T rho exactly for
                            every feature of the X^T rho scope and records, per lambda, the largest
                            |c~_j - x_j^T rho| / E_j of the reduced-precision correlations c~ against
                            their forward-error bounds E_j (bound_ratio and bound_ratio_tc of the
                            stats; <= 1 when every bound holds).  A diagnostic: it adds one exact
                            dot product per feature to every check and changes no result */
  int32_t lockstep_pass; /* lockstep batches (gemm_dtype = LASSO_BF16): 0 (default) advances every
                            problem by one lambda per launch, the product serving the first check
                            of each lambda; 1 advances every problem by one coordinate pass per
                            launch, with a product before every launch: every check reads it,
                            and so does every pass, whose zero coefficients get their
                            certificates anew from it (few column reads then remain).  The
                            number of launches then depends on the data: lasso_batch reads a
                            device counter of unfinished problems every 4 launches
                            (synchronising `stream`), so such a call cannot be captured in a
                            CUDA graph.  Without row_mask, the last 8 unfinished problems stop
                            at their next lambda and finish on lasso_path's solver, one after
                            the other (same results; the workspace holds its region) */
} lasso_opts;

/* Per-lambda record written by the solvers (device memory, one per lambda). */
typedef struct lasso_path_stats {
  double lambda;     /* lambda_t = lambda_max * ratio_t */
  double primal;     /* P_lambda(beta) at the last check, Eq. (1) */
  double dual;       /* D_lambda(theta) at the last check, Eq. (2) */
  double gap;        /* primal - dual at the last check (Sec. 3.2) */
  double radius;     /* GAP SAFE sphere radius of the last check: sqrt(2 (max(gap, 0) + tau))/lambda
                        (Prop. 1, Eq. (10)), where tau >= 0 bounds the FP64 rounding of the gap
                        (2 (n + p + 8) 2^-53 times the sum of the magnitudes of its terms, so the
                        sphere stays safe under rounding); with refined_radius = 1, the smaller of
                        that and (||lambda theta - y||^2 + tau)^(1/2)/lambda (Thm. 2) */
  double alpha;      /* dual scaling of the last check: theta = alpha * rho */
  int64_t epochs;    /* coordinate-descent passes run at this lambda */
  int64_t checks;    /* GAP SAFE checks run at this lambda */
  int64_t n_active;  /* features kept by the last check (|A|, Eq. (6)) */
  int64_t n_nonzero; /* nonzero coefficients of the returned beta */
  int64_t x_columns; /* columns of X the method reads at this lambda: the X^T rho scope of
                        every check plus the safe-active set of every pass (algorithmic work) */
  int32_t converged; /* 1 if gap <= eps was reached */
  int32_t status;    /* lasso_status of this lambda (OK, NOT_CONVERGED, TIMEOUT, NONFINITE) */
  double bound_ratio;    /* with audit_bounds = 1: the largest |c~_j - x_j^T rho| / E_j over the FP32
                            CUDA-core correlations of this lambda's checks (0 otherwise) */
  double bound_ratio_tc; /* with audit_bounds = 1, lockstep lasso_batch: the same over the first
                            checks taken from the split-BF16 tensor-core product (0 otherwise) */
} lasso_path_stats;

/* Fills *opts with the defaults listed above.  opts must not be NULL. */
void lasso_default_opts(lasso_opts* opts);

/* The geometric grid of Sec. 3.3 as ratios to lambda_max:
 * ratios_host[t] = 10^(-delta * t / (T - 1)), t = 0..T-1 (ratios_host[0] = 1;
 * T == 1 gives {1}).  Host-only, synchronous.  INVALID_ARG if T < 1,
 * delta < 0 or ratios_host is NULL. */
lasso_status lasso_lambda_grid(int32_t T, double delta, double* ratios_host);

/* Bytes of device workspace lasso_path needs for these sizes (0 when the
 * sizes are invalid).  The workspace must be 256-byte aligned. */
size_t lasso_path_workspace_size(int64_t n, int64_t p, lasso_dtype x_dtype, const lasso_opts* opts);

/* One Lasso path by Algorithm 1 (CD with GAP SAFE sphere rules).
 *
 *   X_dev        n x p design, column-major, leading dimension ldx.
 *                x_dtype LASSO_F32: ldx % 4 == 0 and X_dev 16-byte aligned.
 *                x_dtype LASSO_F64: ldx >= n, X_dev 8-byte aligned; the design is held
 *                as two FP32 planes (about 48 significand bits, see LASSO_F64).
 *   n, p         1 <= n <= 2048, 1 <= p < 2^31.
 *   y_dev        n responses, FP64.
 *   lambda_ratios_dev  T ratios lambda_t / lambda_max, each in (0, 1]
 *                (lambda_max = ||X^T y||_inf is computed on the device);
 *                lasso_lambda_grid gives the grid of Sec. 3.3.
 *   beta0_dev    p starting coefficients (FP64) or NULL for zeros.
 *   opts         NULL for the defaults.
 *   beta_out_dev p x T FP64, column t = solution at lambda_t.
 *   mask_out_dev words x T uint32: the safe-active set of the last check at
 *                lambda_t, or NULL.
 *   stats_dev    T lasso_path_stats records.
 *   workspace_dev, workspace_bytes  device scratch of at least
 *                lasso_path_workspace_size(n, p, x_dtype, opts) bytes.
 *   stream       a cudaStream_t (NULL = the legacy default stream).
 *
 * Arithmetic: the per-check X^T rho pass runs in FP32 with a rigorous
 * forward-error bound; features whose test or maximum the bound leaves
 * undecided are recomputed exactly.  Coordinate updates keep beta and rho
 * in double-float (pairs of FP32, about 48 significand bits) with exact
 * integer reductions; objectives, gap and radius are FP64.
 *
 * Returns LASSO_OK once the work is enqueued.  The work uses every SM of the
 * device for its duration (one cooperative launch). */
lasso_status lasso_path(const void* X_dev, lasso_dtype x_dtype, int64_t n, int64_t p, int64_t ldx,
                        const double* y_dev, const double* lambda_ratios_dev, int32_t T,
                        const double* beta0_dev, const lasso_opts* opts,
                        double* beta_out_dev, uint32_t* mask_out_dev, lasso_path_stats* stats_dev,
                        void* workspace_dev, size_t workspace_bytes, void* stream);

/* Bytes of device workspace lasso_batch needs for these sizes on the current
 * device (0 when the sizes are invalid); 256-byte alignment required. */
size_t lasso_batch_workspace_size(int64_t n, int64_t p, int64_t B, const lasso_opts* opts);

/* B independent Lasso paths over one design (Algorithm 1 for each): problem b
 * uses the rows i of X with row_mask_dev[i + b*ldm] != 0 (all rows when
 * row_mask_dev is NULL) and the responses Y_dev[i + b*ldy] on those rows --
 * the row-subsampled replicates of stability selection, or many right-hand
 * sides.  Each problem has its own lambda_max over its rows and follows the
 * shared grid lambda_t = lambda_max(b) * ratio_t.
 *
 *   X_dev        n x p FP32, column-major, ldx % 4 == 0, 16-byte aligned.
 *   Y_dev        FP64, column b holds problem b's responses (ldy >= n).
 *   row_mask_dev uint8 n x B (ldm >= n) or NULL.
 *   beta_out_dev p x T x B FP64 (problem b's solution at lambda_t in
 *                column t + b*T), mask_out_dev words x T x B uint32 or NULL,
 *                stats_dev T x B records (index t + b*T).
 *   beta0_dev    p x B FP64 starting points (column b = problem b's, leading
 *                dimension ldb0 >= p) or NULL for the zero start; entries on
 *                the problem's rows only enter through rho = y - X beta0.
 *                With warm_start = 0 every lambda restarts from it.
 *   Other arguments as for lasso_path.
 *
 * opts->gemm_dtype selects how the first check of every lambda gets X^T rho:
 *   LASSO_F32   one persistent launch; each resident CTA takes problems from
 *               a queue and runs a whole path per problem with FP32 CUDA-core
 *               passes (workspace: one region per resident CTA);
 *   LASSO_BF16  lockstep over lambda (default): per lambda one tensor-core
 *               product C = X^T R for all problems in split BF16 (x ~ xh + xl,
 *               r ~ rh + rl, three BF16 GEMM terms, FP32 accumulation, error
 *               <= (3 2^-16 + 2^-20 + 3L 2^-24) |x||r|, L = n rounded up to 8),
 *               then one launch that advances every problem by one lambda
 *               (workspace: one region per problem plus the packed operands);
 *               with opts->lockstep_pass = 1, one product and one launch per
 *               coordinate pass instead.
 * Either way the test decisions equal the exact ones: features the error
 * bound leaves undecided are recomputed exactly.  Results equal B calls of
 * lasso_path on the row-restricted problems, up to rounding. */
lasso_status lasso_batch(const float* X_dev, int64_t n, int64_t p, int64_t ldx, const double* Y_dev, int64_t ldy,
                         const uint8_t* row_mask_dev, int64_t ldm, int64_t B, const double* lambda_ratios_dev,
                         int32_t T, const double* beta0_dev, int64_t ldb0, const lasso_opts* opts,
                         double* beta_out_dev, uint32_t* mask_out_dev, lasso_path_stats* stats_dev,
                         void* workspace_dev, size_t workspace_bytes, void* stream);

/* One Lasso path on a sparse design in compressed sparse column (CSC)
 * storage -- the sparse variant of the solver of Sec. 4.1 (the paper's
 * implementation runs on a dense Fortran-ordered or a sparse CSC design).
 * Algorithm 1 as lasso_path computes it, with every option of lasso_opts
 * except the batched solver's fields; the arithmetic is FP64 throughout (on
 * sparse data the cost is gathers over the nonzeros, not flops).
 *
 *   colptr_dev   p + 1 int64: column j holds entries colptr[j] .. colptr[j+1]-1
 *                (colptr[0] = 0, non-decreasing)
 *   rowidx_dev   int32 row index of every entry, in [0, n) (any order within a column)
 *   values_dev   FP64 value of every entry
 *   n, p         1 <= n <= 16384, 1 <= p < 2^31
 *   workspace    lasso_path_csc_workspace_size(n, p, opts) bytes, 256-byte aligned
 *   Other arguments, outputs, asynchrony and errors as for lasso_path.  Row
 *   indices out of range, NaN/Inf values or a decreasing colptr are found on
 *   the device and reported as LASSO_ERR_INVALID_ARG in every record.  The
 *   checks use all SMs; the coordinate passes run on one CTA, with the
 *   residual in its shared memory. */
size_t lasso_path_csc_workspace_size(int64_t n, int64_t p, const lasso_opts* opts);
lasso_status lasso_path_csc(const int64_t* colptr_dev, const int32_t* rowidx_dev, const double* values_dev,
                            int64_t n, int64_t p, const double* y_dev, const double* lambda_ratios_dev, int32_t T,
                            const double* beta0_dev, const lasso_opts* opts, double* beta_out_dev,
                            uint32_t* mask_out_dev, lasso_path_stats* stats_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream);

/* Launch-shape autotuner for lasso_batch.  Times every candidate shape
 * (lasso_batch_tune_candidates() of them: per-CTA FP32 checks or lockstep
 * split-BF16 products, 1 or 2 solver CTAs per SM, for lockstep an N tile of
 * 128 or 256 and a product per lambda or per pass, for FP32 checks groups of
 * 8, 16 or 32 CTAs per problem) on the
 * first `sample` problems over the first `lambdas`
 * ratios of the grid -- a warm-up run, then a run timed with CUDA events on
 * `stream` -- and writes *opts with the fastest gemm_dtype,
 * batch_ctas_per_sm, gemm_tile_n, batch_group and lockstep_pass to *tuned.  Every candidate makes the
 * same screening decisions (each equal to the FP64 test's), so the choice
 * changes the time, not the results.  Arguments as for lasso_batch;
 * 1 <= sample <= B, 1 <= lambdas <= T; times_ms (host, one float per
 * candidate) may be NULL.  Synchronises `stream`.  workspace: at least
 * lasso_batch_tune_workspace_size(n, p, sample, lambdas) bytes, 256-byte
 * aligned (it also holds the sample's outputs). */
int32_t lasso_batch_tune_candidates(void);
size_t lasso_batch_tune_workspace_size(int64_t n, int64_t p, int64_t sample, int32_t lambdas);
lasso_status lasso_batch_tune(const float* X_dev, int64_t n, int64_t p, int64_t ldx, const double* Y_dev, int64_t ldy,
                              const uint8_t* row_mask_dev, int64_t ldm, int64_t B, const double* lambda_ratios_dev,
                              int32_t T, const double* beta0_dev, int64_t ldb0, const lasso_opts* opts, int32_t sample,
                              int32_t lambdas, lasso_opts* tuned, float* times_ms_host, void* workspace_dev,
                              size_t workspace_bytes, void* stream);

/* The correlation pass of one GAP SAFE check on its own: c = X^T r and
 * m = ||c||_inf (Eq. (7) needs every |x_j^T rho|, the rescaling of Eq. (8)
 * the maximum).  FP32 products accumulated in FP32, one HBM stream over X.
 *
 *   X     n x p FP32, column-major (column j at X + j*ldx), ldx >= n,
 *         ldx % 4 == 0, 16-byte aligned; rows n..ldx-1 are ignored
 *   r     n FP32 (16-byte aligned; entries past n are not read)
 *   c     p FP32 out: c[j] = x_j^T r, each within
 *         (4 ceil(n/128) + 6) 2^-24 sum_i |x_ij r_i| of the exact value
 *   cmax  1 FP32 out (may be NULL): max_j |c[j]|
 * 1 <= n <= 2048.  Asynchronous on `stream`; errors as for lasso_path. */
lasso_status lasso_correlations_f32(const float* X_dev, int64_t n, int64_t p, int64_t ldx, const float* r_dev,
                                    float* c_dev, float* cmax_dev, void* stream);

/* Batched correlations C = X^T R for B residuals at once -- the first GAP
 * SAFE check of every problem of a batch is this product (Eq. (8) needs
 * ||X^T rho_b||_inf, Eq. (7) every |x_j^T rho_b|).  Runs on the tensor cores
 * (tcgen05, BF16 inputs, FP32 accumulation).
 *
 *   X_bf16  n x p BF16, column-major, ldx >= n, ldx % 8 == 0, 16-byte aligned
 *   R_bf16  n x B BF16, column-major, ldr >= n, ldr % 8 == 0, 16-byte aligned
 *   C       p x B FP32, column-major, ldc >= p (C[j + b*ldc] = x_j^T r_b)
 *   workspace  >= 256 bytes, 256-byte aligned; its first int receives a
 *              device-side error code (0 = none, 6 = a wait timed out)
 * The products of BF16 values are exact in FP32; the sum of n of them carries
 * the FP32 rounding of the accumulation.  Asynchronous on stream. */
lasso_status lasso_correlations_bf16(const void* X_bf16, int64_t n, int64_t p, int64_t ldx, const void* R_bf16,
                                     int64_t ldr, int64_t B, float* C, int64_t ldc, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* lasso_path without a workspace argument, for callers that cannot allocate
 * device memory where they solve: plug-ins under a host application that
 * owns the device heap through its own pool, or real-time code whose hot path
 * must not pay for (or risk the failure of) an allocation.  The paper has no
 * counterpart: this is a deployment variant of lasso_path with identical
 * results.
 *
 * Scratch comes from one static device array of 32 MiB that the library
 * holds on every GPU that loads it, until the process exits.  Problems whose
 * workspace (as lasso_path computes it for these sizes) exceeds 32 MiB return
 * LASSO_ERR_INVALID_ARG.  The
 * first call on a device looks up the array's address (cudaGetSymbolAddress)
 * and should come before any stream capture.  All calls on a device share the
 * array: calls whose GPU work overlaps race and must be serialised by the
 * caller.  Each call clears what must start at zero before its kernels run.
 * No memory is allocated.  Other arguments and the return value are as for
 * lasso_path. */
lasso_status lasso_path_static(const void* X_dev, lasso_dtype x_dtype, int64_t n, int64_t p, int64_t ldx,
                               const double* y_dev, const double* lambda_ratios_dev, int32_t T,
                               const double* beta0_dev, const lasso_opts* opts,
                               double* beta_out_dev, uint32_t* mask_out_dev, lasso_path_stats* stats_dev,
                               void* stream);

/* Where the last lasso_path run on this workspace spent its time: SM clock
 * cycles counted by one thread of the first CTA, by phase of Algorithm 1 as
 * the kernel runs it, written to cycles_host[0..7]:
 *   [0] GAP SAFE checks (X^T rho, gap, sphere test, compaction)
 *   [1] coordinate chains (the sequential updates of the nonzero coefficients)
 *   [2] verification that the zero coefficients stay zero
 *   [3] acceptance or rollback of a round, and the planning of the next one
 *   [4] end of a pass (the next pass's support list)
 *   [5] chain entries processed (a count, not cycles)
 *   [6] rollbacks (a count)
 *   [7] other set-up (per-lambda tables, waits before a check)
 * The counters accumulate over the whole path.  Synchronises `stream` (the
 * stream the path ran on) before it returns.  A diagnostic for tuning; the
 * paper has no counterpart. */
lasso_status lasso_path_phase_cycles(const void* workspace_dev, uint64_t* cycles_host, void* stream);

/* Thread-local description of the last error returned on this thread
 * ("" if none).  The pointer stays valid until the next call on the thread. */
const char* lasso_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LASSOGS_H */
