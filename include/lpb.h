/*
 * lpb.h -- C ABI of the batched PDHG LP solver for NVIDIA GB300 (sm_103a).
 *
 * Solves many linear programs that share one sparse constraint matrix A
 * ("Batched First-Order Methods for Parallel LP Solving in MIP", Sec. 3-5):
 *
 *     min  c_q^T x   s.t.   l <= A x <= u,   xlo_q <= x <= xhi_q,   q = 1..N
 *
 * where LP q differs from the base LP only by one override record: a bound
 * change on one variable (strong branching, Sec. 5.1) or an objective +-e_j
 * (optimization-based bound tightening, Sec. 5.2).  The method is restarted
 * reflected-Halpern PDHG (Sec. 4, Eq. mainiter) run on the whole batch at
 * once (Sec. 5, Eq. batched_iter) with per-LP step sizes, a batch-averaged
 * restart test, relative KKT termination (Eq. stopping), infeasibility
 * detection (Eq. primal-infeas, dual-infeas) and compaction of finished LPs.
 *
 * Conventions for every entry point:
 *  - Pointers without a _dev suffix are HOST pointers.  Inputs are copied
 *    during the call; the caller keeps ownership and may free them after.
 *  - Infinite bounds are +-HUGE_VAL (IEEE infinity).
 *  - Indices are 0-based.  CSR row_ptr has m+1 entries, row_ptr[0] == 0.
 *  - Every function returns an lpb_err; the library never aborts, traps or
 *    prints.  lpb_last_error() gives a message for the calling thread.
 *  - A handle is not thread-safe; distinct handles are independent.  The
 *    handles of one lpb_solve_multi call are used by that call until it
 *    returns.
 *  - All device work of a handle runs on the stream given in lpb_options
 *    (NULL: a stream the handle creates and owns), except the joint
 *    intervals of lpb_solve_multi, which run on its first handle's stream.
 */
#ifndef LPB_H
#define LPB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpb_ctx* lpb_handle;     /* one A plus base c, l, u, xlo, xhi on the device */
typedef struct lpb_batch* lpb_batch_t;  /* the results of one lpb_solve */

typedef enum {
    LPB_OK = 0,
    LPB_ERR_INVALID_ARG = 1,   /* bad size, pointer, NaN/Inf data, l > u, unsorted row_ptr ... */
    LPB_ERR_OOM = 2,           /* device or pinned host allocation failed */
    LPB_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    LPB_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    LPB_ERR_DEVICE_CHECK = 5,  /* a kernel's own bounds check fired */
    LPB_ERR_BAD_INDEX = 6      /* an override names a variable outside [0, n) */
} lpb_err;

typedef enum {
    LPB_OPTIMAL = 0,           /* rel. primal, dual and gap residuals <= tol (Eq. stopping) */
    LPB_PRIMAL_INFEASIBLE = 1, /* Eq. primal-infeas held, or the override emptied the box */
    LPB_DUAL_INFEASIBLE = 2,   /* Eq. dual-infeas held (the LP is unbounded if feasible) */
    LPB_ITERATION_LIMIT = 3,   /* max_iter reached; the result is the last evaluated point */
    LPB_NUMERICAL = 4          /* a NaN appeared in the LP's residuals */
} lpb_lp_status;

typedef enum { LPB_FP64 = 0, LPB_MIXED = 1 } lpb_precision;

typedef struct {
    int32_t precision;              /* LPB_FP64: FP64 iterates and checks; LPB_MIXED: FP32 iterates and
                                       SpMM, with the KKT residuals, gap, certificates and the fixed-point
                                       residual summed in double-float arithmetic (a pair of FP32 values,
                                       about 48 significand bits, FP32 exponent range); the restart tests,
                                       primal weights and scaling factors are FP64 */
    int32_t check_every;            /* iterations between residual evaluations (default 64) */
    int32_t ruiz_iters;             /* Ruiz infinity-norm passes (default 10) */
    int32_t pock_chambolle;         /* 1: one Pock-Chambolle (alpha = 1) pass after Ruiz */
    double beta_s, beta_n, beta_a;  /* restart conditions of Sec. 4 (0.2, 0.8, 0.36) */
    double theta;                   /* primal-weight smoothing (0.5) */
    double mnorm_sign;              /* sign of the A terms of the M-norm, Eq. residual (-1) */
    int32_t restart_to_pdhg_output; /* 1: the new anchor is T(z) at the check; 0: the Halpern iterate */
    int32_t power_max_iter;         /* power iteration for ||A||_2 (5000) */
    double power_tol;               /* relative change that stops it (1e-10) */
    uint64_t power_seed;            /* SplitMix64 seed of its start vector */
    double eps_infeas;              /* infeasibility tolerance; < 0 uses the solve's tol */
    int32_t detect_infeasibility;   /* 1: evaluate Eq. primal-infeas and dual-infeas */
    int32_t profile;                /* 1: time every iteration kernel with CUDA events */
    void* cuda_stream;              /* cudaStream_t to run on, or NULL */
    int32_t device;                 /* CUDA device ordinal, or -1 for the current device */
    int32_t fp64_polish;            /* LPB_MIXED only: 1 (default) widens the remaining batch to
                                       FP64-accurate iterates once an LP stalls at FP32 resolution */
    int32_t polish_stall_checks;    /* an LP stalls when its KKT error has not halved over this many
                                       checks (default 32) */
    int32_t polish_arith;           /* arithmetic of the polish iterates: LPB_POLISH_DFLOAT (default;
                                       double-float pairs on the FP32 pipe, 8 bytes per value) or
                                       LPB_POLISH_FP64 (native FP64) */
    double eps_dual;                /* tolerance of the relative dual residual alone; < 0 (default)
                                       uses the solve's tol.  Bound tightening (Sec. 6 OBBT) uses 1e-8
                                       so that the dual bound is safe */
    int32_t use_graphs;             /* 1 (default): each interval (check_every iterations and the check)
                                       is a CUDA graph, captured once per batch shape and replayed;
                                       not used when profile = 1 */
    int32_t use_pdl;                /* 1 (default): the step kernels of an interval are launched as
                                       programmatic dependents, so each one's launch and parameter
                                       staging overlap the end of the previous one; not used when
                                       profile = 1 */
    int32_t stream_priority;        /* priority of the stream lpb_create makes when cuda_stream is NULL
                                       (CUDA's scale: lower is more urgent; clamped to the device's
                                       range; default 0): on a shared GPU the blocks of more urgent
                                       handles are scheduled first, e.g. small LPs served beside
                                       large ones */
    int32_t reduced_cost;           /* the reduced cost r of the stopping test (Sec. 4, Eq. stopping):
                                       LPB_RC_BARRIER (default) r = Pi_B(-c - A^T y) as printed;
                                       LPB_RC_ROBUST, the variant the paper's implementation uses
                                       (PDLP's Appendix A): a component counts against a finite bound
                                       only where the primal point lies no farther from that bound
                                       than from zero, and otherwise stays in the dual residual, so
                                       that large finite bounds do not swamp the dual objective and
                                       the gap.  The infeasibility tests keep Pi_B in both modes */
} lpb_options;

/* Values of lpb_options.polish_arith. */
enum { LPB_POLISH_DFLOAT = 0, LPB_POLISH_FP64 = 1 };
/* Values of lpb_options.reduced_cost. */
enum { LPB_RC_BARRIER = 0, LPB_RC_ROBUST = 1 };

/* One override record (Sec. 5.1, 5.2). */
typedef struct {
    int32_t kind;  /* 0: base LP; 1: bound change on var; 2: objective sign * e_var */
    int32_t var;   /* variable index for kinds 1 and 2 */
    double lo, hi; /* kind 1: the child's box for var is [max(xlo[var], lo), min(xhi[var], hi)];
                      pass -HUGE_VAL / +HUGE_VAL to keep a side.  lo > hi after that
                      intersection makes the LP PRIMAL_INFEASIBLE with 0 iterations. */
    double sign;   /* kind 2: +1 minimises x_var, -1 maximises it (objective -x_var) */
} lpb_lp_spec;

typedef struct {
    int32_t status;      /* lpb_lp_status */
    int32_t restarts;    /* batch restarts taken while this LP was active */
    int64_t iters;       /* PDHG iterations applied to this LP */
    double obj;          /* c^T x at the returned point */
    double dual_obj;     /* -phi_[xlo,xhi](r) - phi_[l,u](y) (Sec. 3), r as lpb_options.reduced_cost */
    double rel_primal;   /* ||Ax - Pi_[l,u](Ax)|| / (1 + ||Ax||) */
    double rel_dual;     /* ||c + A^T y + r|| / (1 + ||c||) */
    double rel_gap;      /* |c^T x + phi + phi| / (1 + |c^T x| + |phi + phi|) */
    double safe_bound;   /* dual_obj - tol (1 + |c^T x| + |phi + phi|): the paper's OBBT bound on the
                            optimal objective, shifted by its Delta (Sec. 6 "OBBT results") */
} lpb_lp_result;

/* Per-kernel timing gathered when lpb_options.profile = 1 (CUDA events on the
 * handle's stream).  bytes = algorithmic bytes: A's values and indices, its
 * row pointers and every dense operand counted once per launch. */
typedef struct {
    int64_t launches[4];  /* 0: A^T Y primal step, 1: A X dual step, 2: FP64 check SpMMs,
                             3: check reductions + restart */
    double ms[4];
    double bytes[4];
    double setup_ms;      /* lpb_create device work */
    int64_t checks, compactions;
    int64_t kernels;      /* every kernel the solve launched */
    int64_t fp64_switch_iter;  /* iteration at which the batch moved to FP64 iterates, -1 if never */
} lpb_profile;

/* Fills *opt with the defaults listed above. */
void lpb_default_options(lpb_options* opt);

/* Builds a handle (Sec. 3 problem data; Sec. 4 step size).  Copies A (CSR,
 * FP64 values, m x n, nnz < 2^31), c (n), row bounds l, u (m) and variable
 * bounds xlo, xhi (n) to the device, then on the device: transposes A,
 * equilibrates it (Ruiz then Pock-Chambolle; A~ = D_r A D_c), estimates
 * ||A~||_2 by power iteration and fixes eta = 0.998 / ||A~||_2.
 * Rejects (LPB_ERR_INVALID_ARG): m < 0, n < 1, negative nnz, a non-monotone
 * row_ptr, a column index outside [0, n), a non-finite value or cost, NaN
 * bounds, l > u, xlo > xhi, l = +inf or u = -inf.  opt may be NULL. */
lpb_err lpb_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* vals, const double* c, const double* row_lo, const double* row_hi,
                   const double* var_lo, const double* var_hi, const lpb_options* opt, lpb_handle* out);

/* Solves num_lps LPs (Sec. 5).  specs: num_lps host records.  tol: relative
 * KKT tolerance of Eq. stopping (> 0).  max_iter >= 1 caps the PDHG
 * iterations.  warm_x (n x num_lps, LP q at offset q*n) and warm_y (m x
 * num_lps) are optional warm starts (NULL: x = projection of 0, y = 0).
 * On LPB_OK *out owns the results until lpb_batch_free. */
lpb_err lpb_solve(lpb_handle h, int32_t num_lps, const lpb_lp_spec* specs, double tol, int64_t max_iter,
                  const double* warm_x, const double* warm_y, lpb_batch_t* out);

/* As lpb_solve, with specs_dev, warm_x_dev and warm_y_dev in device memory
 * of the handle's device (layouts as above; warm pointers may be NULL).
 * The override records are validated on the device: a variable index out
 * of range returns LPB_ERR_BAD_INDEX. */
lpb_err lpb_solve_dev(lpb_handle h, int32_t num_lps, const lpb_lp_spec* specs_dev, double tol,
                      int64_t max_iter, const double* warm_x_dev, const double* warm_y_dev,
                      lpb_batch_t* out);

/* Most handles in one lpb_solve_multi call. */
enum { LPB_MAX_JOINT = 64 };

/* Solves count batches on count different handles together (Sec. 5, the
 * batched iteration of Eq. batched_iter, run over LPs of several matrices,
 * i.e. LPs of uneven size and iteration count in one launch).  Batch i is
 * num_lps[i] LPs of handles[i] with the host override records specs[i]
 * (as lpb_solve, no warm start).  Every iteration runs the primal steps of
 * all batches still iterating as one kernel launch, then their dual steps
 * as one launch (one launch per row-group width among the batches and per
 * 8 batches), and each batch's check after the interval, all on the first
 * handle's stream; with the first handle's use_graphs each interval is one
 * CUDA graph.  A batch that finishes leaves the joint launches; one that
 * stalls at FP32 resolution (LPB_MIXED with fp64_polish) leaves them and is
 * polished on its own handle and stream.  Each result is bitwise the one
 * lpb_solve gives for that batch alone.  Event timing (profile = 1) is not
 * taken; each batch's lpb_profile counts its share of the launches as if
 * solved alone.
 * Rejects (LPB_ERR_INVALID_ARG): count outside [1, LPB_MAX_JOINT], a NULL
 * array, a handle twice, handles on different devices or with different
 * precision or check_every, and whatever lpb_solve rejects for a batch.
 * On LPB_OK out[i] owns batch i's results until lpb_batch_free; on an error
 * every out[i] is NULL. */
lpb_err lpb_solve_multi(int32_t count, const lpb_handle* handles, const int32_t* num_lps,
                        const lpb_lp_spec* const* specs, double tol, int64_t max_iter, lpb_batch_t* out);

/* Result of LP lp of a batch: *res, and optionally x (n doubles) and y (m
 * doubles) in the original, unscaled space (x = D_c x~, y = D_r y~). */
lpb_err lpb_result(lpb_batch_t b, int32_t lp, lpb_lp_result* res, double* x, double* y);

/* All num_lps results at once (host array of num_lps records). */
lpb_err lpb_results(lpb_batch_t b, lpb_lp_result* res);

/* Device pointers to the batch's x (n x num_lps) and y (m x num_lps); owned by
 * the batch. */
lpb_err lpb_result_device(lpb_batch_t b, const double** x_dev, const double** y_dev);

/* Kernel timing of a batch solved with profile = 1 (zeros otherwise). */
lpb_err lpb_batch_profile(lpb_batch_t b, lpb_profile* p);

/* Scalars fixed by lpb_create: eta = 0.998/||A~||_2 and the power-iteration
 * estimate of ||A~||_2 with the number of products it took. */
lpb_err lpb_handle_info(lpb_handle h, double* eta, double* norm_est, int32_t* power_iters);

/* Scaling factors D_r (m) and D_c (n) of A~ = D_r A D_c, copied to the host. */
lpb_err lpb_scaling(lpb_handle h, double* d_row, double* d_col);

/* Equilibration factors without allocating anything.  The paper has no
 * counterpart; this serves callers that cannot call cudaMalloc: code running
 * while a CUDA graph is being captured, latency-critical callers that must
 * not trigger the allocator's device-wide synchronization, and hosts whose
 * device memory is owned by their own pool allocator.  It computes the same
 * factors as lpb_create (ruiz_iters Ruiz infinity-norm passes, then one
 * Pock-Chambolle pass when pock_chambolle != 0; A~ = D_r A D_c) for an m x n
 * CSR matrix already in device memory: row_ptr_dev (m+1 int32), col_idx_dev
 * (nnz int32) and vals_dev (nnz finite doubles) are read, d_row_dev (m) and
 * d_col_dev (n) are written; all are device pointers owned by the caller.
 * Work is queued on cuda_stream (NULL: the default stream); the factors are
 * valid once that stream reaches this point.  The scratch is a fixed
 * device-resident array of 2^21 doubles in this library, held by every GPU
 * that loads it until the process exits: m + n above 2097152 returns
 * LPB_ERR_INVALID_ARG.  A device's first call looks up that array's address
 * (make it before any stream capture); calls share the array, so calls that
 * overlap on the GPU race on it.  The column sums of the last pass come from
 * atomic updates, so they may differ from lpb_create's in the last bits. */
lpb_err lpb_scaling_noalloc(int32_t m, int32_t n, int32_t nnz, const int32_t* row_ptr_dev,
                            const int32_t* col_idx_dev, const double* vals_dev, int32_t ruiz_iters,
                            int32_t pock_chambolle, double* d_row_dev, double* d_col_dev, void* cuda_stream);

/* Bound tightening from a solved OBBT batch (Sec. 5.2, Sec. 6 "OBBT
 * results").  For each LP q of kind 2 that ended LPB_OPTIMAL: sign +1
 * (min x_var) gives the lower bound safe_bound, sign -1 (max x_var) the
 * upper bound -safe_bound.  new_lo / new_hi (n doubles, host) start as
 * var_lo / var_hi (n, host; the base box) and take a candidate only where it
 * improves the current value by more than min_gain (the paper uses 1e-4)
 * and stays inside the box; *updated counts the bounds changed.  specs are
 * the batch's num_lps host records. */
lpb_err lpb_obbt_tighten(lpb_batch_t b, const lpb_lp_spec* specs, const double* var_lo, const double* var_hi,
                         double min_gain, double* new_lo, double* new_hi, int32_t* updated);

/* Launch shapes of the two step kernels (Sec. 5 batched SpMMs).  A row of
 * A~^T (primal step) or A~ (dual step) with more nonzeros than the
 * long_row_* threshold is reduced by a whole thread block; shorter rows by a
 * row group of lanes, whose number follows from the batch width and is
 * halved lane_shift_* times (more column tiles per row).  Defaults: 32, 32,
 * 0, 0.  Results depend on the shapes only through the order in which long
 * rows are summed. */
typedef struct {
    int32_t long_row_primal;
    int32_t long_row_dual;
    int32_t lane_shift_primal;
    int32_t lane_shift_dual;
} lpb_tuning;

lpb_err lpb_get_tuning(lpb_handle h, lpb_tuning* t);
/* thresholds >= 1, shifts in [0, 5]; LPB_ERR_INVALID_ARG otherwise */
lpb_err lpb_set_tuning(lpb_handle h, const lpb_tuning* t);

/* Autotuner: times the primal and dual steps on num_lps copies of the base
 * LP for every threshold in {8, 16, 32, 64, 128, 256} and shift in {0, ..., 4},
 * applies the fastest shape of each step to the handle and returns it in
 * *chosen (may be NULL).  Takes a few hundred step launches. */
lpb_err lpb_autotune(lpb_handle h, int32_t num_lps, lpb_tuning* chosen);

/* Batch size by timing (Sec. 5: pick the N that maximises mat-vec products
 * per second): for each of count batch widths, the time of one iteration
 * (primal + dual step) on that many copies of the base LP, in microseconds,
 * into us_per_iter[i]; *best = the index with the most LP iterations per
 * second.  Widths must be in [1, 65536]. */
lpb_err lpb_tune_batch(lpb_handle h, const int32_t* widths, int32_t count, double* us_per_iter, int32_t* best);

void lpb_batch_free(lpb_batch_t b);
void lpb_destroy(lpb_handle h);

/* Message for the last non-OK return on the calling thread ("" if none). */
const char* lpb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LPB_H */
