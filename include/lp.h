/*
 * lp.h -- C ABI of the B300 restarted reflected-Halpern PDHG solver for LP.
 *
 * Method: cuPDLPx (Lu, Peng, Yang; arXiv 2507.14051).
 *   Problem, Section 2.1 eq. (lp):  min c^T x  s.t.  l_c <= A x <= u_c,  l_v <= x <= u_v,
 *     bounds may be +-INFINITY (+inf only in an upper bound, -inf only in a lower one).
 *   Iteration, Section 2.2 eq. (pdhg) with tau = eta/omega, sigma = eta*omega, wrapped in the
 *     reflected Halpern scheme of Section 3, restarted by the fixed-point-residual rule of
 *     Section 3 ("Adaptive restart"), with constant step eta = 0.998/||A||_2 (Section 3,
 *     "Stepsize") and the PID primal-weight update (Section 3, "Primal weight update").
 *   Termination, Section 4 ("Optimality termination criteria"): relative KKT error <= tol,
 *     evaluated on the original LP.
 *
 * Every call returns an lp_status: LP_OK (0) or a negative error code.  The library
 * never aborts and never prints; lp_last_error() gives a message for the calling thread.
 * All entry points are thread-compatible (one handle must not be used by two threads at once).
 *
 * Device: one CUDA device, the one current on the calling thread at lp_create; later calls
 * on the handle make that device current themselves.
 */
#ifndef PDHG_LP_H
#define PDHG_LP_H

#include <stdint.h>

#if defined(__GNUC__)
#define LP_API __attribute__((visibility("default")))
#else
#define LP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lp_status;
enum {
  LP_OK = 0,
  LP_ERR_INVALID_ARG = -1,   /* null pointer, negative size, unknown flag, bad parameter value */
  LP_ERR_INVALID_INPUT = -2, /* bad CSR (row_ptr not monotone, column out of range), NaN or inf in
                                A or c, NaN bound, l > u, +inf lower bound or -inf upper bound */
  LP_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the CUDA error string) */
  LP_ERR_OUT_OF_MEMORY = -4, /* device or host allocation failed */
  LP_ERR_NOT_SOLVED = -5,    /* lp_get before any lp_solve */
  LP_ERR_TOO_LARGE = -6      /* nnz >= 2^31 (the device CSR uses 32-bit offsets) */
};

/* Outcome of a solve (lp_get's solve_status). */
enum {
  LP_SOLVE_OPTIMAL = 1,    /* relative KKT error <= tol at a check iteration (Section 4) */
  LP_SOLVE_ITER_LIMIT = 2, /* max_iter iterations done without meeting tol */
  LP_SOLVE_NUMERICAL = 3,  /* the fixed-point residual became NaN or infinite */
  LP_SOLVE_INFEASIBLE = 4, /* reserved: the paper gives no infeasibility test; never returned */
  LP_SOLVE_STALLED = 5,    /* precision 2 only: the FP32 solve stopped improving (fp32_patience) */
  LP_SOLVE_INTERNAL_ERROR = 6 /* the device loop outran max_iter (a library fault); not expected */
};

/* Where lp_create's input arrays live. */
enum { LP_HOST = 0, LP_DEVICE = 1 };

/*
 * Solver parameters.  The paper prints the reflection range gamma in [0,1], the stepsize
 * factor 0.998, the initial primal weight 1.0 and the termination tolerance; the restart
 * thresholds and PID gains are named but not given a value, so their defaults are readings
 * (see lp_default_params).  All fields are copied at lp_create / lp_set_params.
 */
typedef struct {
  double gamma;            /* reflection coefficient of (1+gamma)PDHG - gamma*id, Section 3; [0,1] */
  double beta_sufficient;  /* restart when r(z^{n,k}) <= beta_sufficient * r(z^{n,0}), Section 3 */
  double beta_necessary;   /* ... or r <= beta_necessary * r0 and r > r(z^{n,k-1}), Section 3 */
  double beta_artificial;  /* ... or k >= beta_artificial * T, T = total iterations, Section 3 */
  double k_p, k_i, k_d;    /* PID gains on e^n = log(omega |dx| / |dy|), Section 3 */
  double eta;              /* > 0: step size used as given; <= 0: 0.998 / ||A~||_2 (power iteration
                              on the preconditioned matrix A~), Section 3 "Stepsize" */
  double omega0;           /* initial primal weight, Section 3 (1.0) */
  int64_t check_every;     /* KKT test at iterations t with (t+1) % check_every == 0 and at the last */
  int32_t restart_enabled; /* 0: no restarts (plain reflected Halpern) */
  int32_t pid_enabled;     /* 0: omega stays omega0 */
  double power_tol;        /* power iteration stops when |lambda - lambda_prev| <= tol * lambda */
  int64_t power_max_iter;
  uint64_t power_seed;     /* start vector v_j = uniform[-1,1) from splitmix64(seed, j) */
  int32_t ruiz_iters;      /* diagonal preconditioning: Ruiz l_inf passes (0: none) */
  int32_t pc_enabled;      /* then one Pock-Chambolle pass with exponent pc_alpha (0: none) */
  double pc_alpha;
  int64_t trace_cap;       /* > 0: record (r_t, omega_t, restart_t, k_t) for t < trace_cap */
  int32_t unroll;          /* iterations per body of the device-side loop (1..64) */
  int32_t lane_target;     /* SpMV schedule: at most this many nonzeros per lane and task (1..64);
                              0: automatic (32: rows of up to 32 entries are read one lane per
                              row, in sliced tiles, and longer rows take fewer FP64 butterfly
                              additions) */
  int32_t persistent;      /* 1: one cooperative kernel runs `unroll` iterations per launch with
                              grid-wide barriers between phases; 2: the same loop as one
                              thread-block cluster of up to 16 CTAs (cluster barriers; for LPs
                              of a few dozen tiles per phase); 3: the loop as one cluster whose
                              CTAs hold the whole LP in shared memory for the length of a launch
                              (gamma = 1 and an LP that fits: no row or column longer than 128
                              entries, and each CTA's slices plus replicas of the gathered
                              vectors, about 8 (3n + 2m) bytes, within its shared memory);
                              0: one kernel per phase; -1: 3 when it applies, else 2 when each
                              phase has at most 4 tiles per warp of a 16-CTA cluster, else 1
                              when every block of both phases fits on the GPU at once, else 0.
                              3 on an LP where it does not apply chooses as -1 does. */
  int32_t precision;       /* 0: FP64 throughout.  1: mixed -- matrix and iterates in FP32 with
                              FP32 SpMV accumulation (reductions, restart test, PID and KKT test in
                              FP64) until the relative KKT error is <= max(tol, switch_tol) or
                              max_iter iterations, then an FP64 refinement phase anchored at the
                              FP32 point, up to max_iter further iterations.  2: FP32 phase only.
                              Fixed at lp_create. */
  double switch_tol;       /* precision 1: KKT level at which the FP32 phase hands over */
  int32_t fp32_patience;   /* FP32 phase: at a check iteration whose relative KKT error is no new
                              best for the fp32_patience-th time in a row, or is above 100 times
                              the best, the phase stops (precision 1: hands over to FP64 with
                              omega and the PID state of the best check; precision 2: ends with
                              LP_SOLVE_STALLED).  0 disables the guard. */
  int32_t rescale;         /* 1: bound/objective rescaling after the diagonal preconditioning --
                              objective / ||c~||_2, bounds / ||finite (l_c~, u_c~)||_2.  This change
                              of variables maps every PDHG step, restart decision and PID error
                              onto those of the unrescaled iteration started from
                              omega0 * ||c~|| / ||b~||, which is how it is applied.  0: off */
  int32_t tile_rows;       /* rows per warp tile (1..32, rounded down to a power of two): a tile
                              of R rows, each read by G lanes (G from lane_target), takes R G / 32
                              passes and runs its R row epilogues in R lanes at once; 0: automatic
                              (lp_solve: 32 when A and A^T each give at least 8 tiles of 32 rows
                              per resident warp of the loop kernel, else 1, since latency-bound
                              sizes want short tasks; the batch: 8, since its long rows would
                              otherwise spend one warp's FP64 issue on each row's epilogue) */
  int64_t batch_local_nnz; /* lp_batch_* only: instances with at most this many nonzeros are
                              solved by one cluster of 8 CTAs each (cluster barriers only)
                              instead of by the grid-wide loop; 0 puts every instance on the grid
                              loop */
} lp_params;

/* Fills p with the defaults: gamma 1, betas 0.2 / 0.8 / 0.36, K_P 0.5, K_I 0.001, K_D 0,
 * eta 0 (power iteration), omega0 1, check_every 64, restarts and PID on, power_tol 1e-7,
 * power_max_iter 10000, seed 0, Ruiz 10 + Pock-Chambolle alpha 1, no trace, unroll 32,
 * lane_target 0 (automatic), persistent -1, precision 0, switch_tol 1e-5, fp32_patience 32, rescale 0,
 * tile_rows 0, batch_local_nnz 16384.  Returns LP_ERR_INVALID_ARG if p is NULL. */
LP_API lp_status lp_default_params(lp_params* p);

typedef struct lp_solver* lp_handle;

/*
 * Creates a solver for the LP of Section 2.1 eq. (lp).
 *   m, n      rows and columns of A (>= 0).
 *   nnz       stored entries; row_ptr[m] must equal nnz.
 *   row_ptr   int64[m+1], 0-based CSR offsets, non-decreasing, row_ptr[0] = 0.
 *   col_idx   int32[nnz], in [0, n); order inside a row is free; duplicates are summed.
 *   val       double[nnz], finite.
 *   c         double[n], finite objective.
 *   l_c, u_c  double[m] row bounds,  l_v, u_v  double[n] column bounds; +-INFINITY allowed
 *             (-inf lower / +inf upper only), l <= u, no NaN.
 *   where     LP_HOST: all arrays are host memory; LP_DEVICE: all are device memory of the
 *             current device.
 *   p         parameters, or NULL for lp_default_params.
 *   out       receives the handle.
 * Ownership: every input is deep-copied; the caller may free its arrays on return.  The
 * handle owns its device memory until lp_destroy.  Setup here: validation, the stored
 * transpose, the row/column length binning, diagonal preconditioning and the power
 * iteration.  Synchronous (returns when setup is complete).
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_INVALID_INPUT, LP_ERR_TOO_LARGE, LP_ERR_CUDA,
 * LP_ERR_OUT_OF_MEMORY; *out is left NULL on error.
 */
LP_API lp_status lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                    const int32_t* col_idx, const double* val, const double* c,
                    const double* l_c, const double* u_c, const double* l_v, const double* u_v,
                    int32_t where, const lp_params* p, lp_handle* out);

/* Replaces the parameters of h.  Takes effect at the next lp_solve.  With eta <= 0 the step
 * size comes from the power iteration, re-run only when power_seed, power_tol or
 * power_max_iter changed; the preconditioning fields and lane_target are fixed at lp_create
 * and ignored here.  Synchronous.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA. */
LP_API lp_status lp_set_params(lp_handle h, const lp_params* p);

/*
 * Enqueues one solve from the all-zero start (Section 4, "Initialization") on `stream`
 * (a cudaStream_t; NULL means the legacy default stream) and returns without waiting.
 *   tol       relative KKT tolerance (Section 4); 0 runs exactly max_iter iterations.
 *   max_iter  >= 1.
 * The whole loop runs on the device as one CUDA graph with a conditional while node; the
 * host is not involved between iterations.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
LP_API lp_status lp_solve(lp_handle h, double tol, int64_t max_iter, void* stream);

/*
 * Waits for the last lp_solve and returns its result: the PDHG output zhat = (xhat, yhat)
 * of the final iteration, in the original (unscaled, unpermuted) variables.
 *   x            double[n] or NULL; host or device memory (any address CUDA can reach).
 *   y            double[m] or NULL; y_i >= 0 on an active lower row bound (set Y, Section 2.1).
 *   solve_status LP_SOLVE_* or NULL.
 *   kkt          double[4] or NULL: relative gap, primal residual, dual residual and their
 *                maximum (Section 4), from the final check iteration.
 *   iters        iterations performed, or NULL.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED, LP_ERR_CUDA.
 */
LP_API lp_status lp_get(lp_handle h, double* x, double* y, int32_t* solve_status, double* kkt,
                 int64_t* iters);

/* Extra scalars of the last solve (host doubles): out[0] eta, out[1] final omega,
 * out[2] restarts, out[3] ||A~||_2 from the power iteration (0 if eta was given),
 * out[4] power-iteration steps, out[5] primal objective c^T x, out[6] dual objective,
 * out[7] 1 if the cooperative loop kernel runs the solve, 2 if the cluster loop does, 3 if the
 * shared-memory cluster loop does, 0 if one kernel per phase does,
 * out[8] iterations done in FP32 (precision 1 or 2; 0 for FP64).
 * Waits like lp_get.  Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED, LP_ERR_CUDA. */
LP_API lp_status lp_get_info(lp_handle h, double* out9);

/* Copies up to cap rows of the per-iteration trace (r_t, omega_t, restart_t, k_t) into the
 * host array trace[4*cap]; *rows receives the number written.  Needs trace_cap > 0. */
LP_API lp_status lp_get_trace(lp_handle h, double* trace, int64_t cap, int64_t* rows);

/* Frees everything the handle owns.  NULL is ignored. */
LP_API void lp_destroy(lp_handle h);

/* Message of the last error on the calling thread ("" if none). */
LP_API const char* lp_last_error(void);

/*
 * Kernel timing for roofline reports: runs at least `iters` iterations of the same solve that
 * lp_solve would (tolerance 0, from the all-zero start), launching the iteration kernels one
 * by one on `stream` with CUDA events around each launch instead of through the graph.  The
 * kernels are those of the solve's first stage: FP64 for precision 0, FP32 for precision 1 and
 * 2 (after which the handle holds no result: lp_get returns LP_ERR_NOT_SOLVED until the next
 * lp_solve).
 *   persistent = 0: ms_out[0] / ms_out[1] mean duration of the row kernel (A x, dual step,
 *     restart control) and of the column kernel (A^T y, primal step, KKT test), ms_out[2] = 1;
 *   a loop kernel (persistent 1, 2 or 3, or -1 choosing one): ms_out[0] mean duration of one
 *     launch of the loop kernel, ms_out[1] = 0, ms_out[2] = iterations per launch (unroll).
 * ms_out[3] = launches timed.  Synchronous.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
LP_API lp_status lp_time_kernels(lp_handle h, int64_t iters, void* stream, double* ms_out);

/*
 * Standalone device SpMV with the solver's binned schedule: y = A x for a CSR matrix that
 * the handle holds (which = 0: A, which = 1: A^T), in the handle's permuted and scaled
 * storage order.  x, y are device arrays of the permuted length.  Used by tests of the SpMV
 * schedule.  Synchronous.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
LP_API lp_status lp_debug_spmv(lp_handle h, int32_t which, const double* x_dev, double* y_dev);

/*
 * Handle internals for tests: copies the permutations and scale factors to host arrays.
 * row_perm[i'] = original row of permuted row i' (int32[m]); col_perm likewise (int32[n]);
 * d_r (double[m]) and d_c (double[n]) are the preconditioning factors in ORIGINAL order.
 * Any pointer may be NULL.  Errors: LP_ERR_INVALID_ARG, LP_ERR_CUDA.
 */
LP_API lp_status lp_debug_layout(lp_handle h, int32_t* row_perm, int32_t* col_perm, double* d_r,
                          double* d_c);

/*
 * ||A||_2 by power iteration, for callers that cannot allocate device memory.  The paper has
 * no counterpart to this entry point.
 *
 * Some callers must not call cudaMalloc: code whose device memory is owned entirely by its
 * own pool allocator, or latency-critical code that cannot afford the implicit device
 * synchronisation an allocation may cause.  This entry point allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call): it computes the same estimate as the
 * power iteration of lp_create (start vector uniform[-1,1) from splitmix64(seed, j),
 * w = A v, lambda = |w|^2, v = A^T w / |A^T w|, stop when |lambda - lambda_prev| <= tol *
 * lambda or after max_iter steps; result sqrt(lambda)) on the caller's matrix as given (no
 * preconditioning), with all scratch in one static device array of about 6.3 MB that the
 * library holds on every device that loads it until the process exits.
 *   m, n       at most 262144 each; larger sizes return LP_ERR_TOO_LARGE.
 *   row_ptr, col_idx, val   CSR of A in device memory of the current device (int64 offsets,
 *              0-based int32 column indices, doubles; row_ptr has m + 1 entries, col_idx and
 *              val nnz).  The kernels check every offset and column index as they read it:
 *              an offset outside [0, nnz], decreasing offsets or a column index outside
 *              [0, n) is never dereferenced, and the call returns LP_ERR_INVALID_INPUT.
 *   tol, max_iter, seed     stopping rule and start vector as in lp_params.
 *   stream     cudaStream_t (NULL: legacy default stream); the call is synchronous.  Steps are
 *              queued 16 at a time with one host synchronisation per 16 steps.
 *   norm_out   receives the estimate (0 for an empty matrix); iters_out (may be NULL) the steps.
 * Every call looks up the device address of the static scratch in the current device's
 * context (cudaGetSymbolAddress, which allocates nothing), so the address stays valid across a
 * cudaDeviceReset.  The first call on a device may load the library's device code; make that
 * first call before any stream capture.  Every call on a device shares the same scratch:
 * calls that overlap on the GPU (other threads, other streams) race and give wrong results.
 * The transposed product uses atomic adds, so the last bits of the estimate can differ from
 * run to run.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_INVALID_INPUT, LP_ERR_TOO_LARGE, LP_ERR_CUDA.
 */
LP_API lp_status lp_power_norm_noalloc(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                                       const int32_t* col_idx, const double* val, double tol,
                                       int64_t max_iter, uint64_t seed, void* stream,
                                       double* norm_out, int64_t* iters_out);

#ifdef __cplusplus
}
#endif

#endif /* PDHG_LP_H */
