/*
 * Batched solver: many independent LPs of the form of Section 2.1, eq. (lp), solved by the same
 * method as lp_solve (restarted reflected-Halpern PDHG with the fixed-point-residual restarts and
 * the PID primal weight of Sections 2.2 and 3, the relative KKT test of Section 4) in one
 * persistent device loop.  Every instance keeps its own iteration count t, epoch step k, primal
 * weight omega, restart reference r0, PID state, step size eta and status; an instance that
 * meets the tolerance stops while the others go on.  The paper solves one LP at a time; the
 * batch is an extension of this library with no counterpart in the paper.
 *
 * All entry points return LP_OK (0) or a negative lp_status from lp.h; the message is in
 * lp_last_error().  Nothing aborts or prints.
 */
#ifndef PDHG_LP_BATCH_H
#define PDHG_LP_BATCH_H

#include "lp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_batch* lp_batch_handle;

/* Largest number of instances in one batch. */
#define LP_BATCH_MAX_INSTANCES 2048

/*
 * Creates a batch of `count` (1..LP_BATCH_MAX_INSTANCES) LPs from HOST memory.  Instance k is
 * given exactly as to lp_create: m[k], n[k], nnz[k] and the arrays row_ptr[k] (int64[m+1]),
 * col_idx[k] (int32[nnz]), val[k], c[k], l_c[k], u_c[k], l_v[k], u_v[k] (double), with the same
 * validation (an invalid instance fails the whole call with LP_ERR_INVALID_INPUT; the message
 * names the instance).  The arrays are copied; the caller keeps ownership.
 *   eta   NULL: instance k uses p->eta if > 0, else 0.998 / ||A~_k||_2 from a power iteration
 *         on its own preconditioned matrix (Section 3, "Stepsize"); or double[count], each > 0,
 *         the step size of each instance.
 *   tiles NULL: p->lane_target and p->tile_rows for every instance (0, the default: lane_target
 *         32 and tile_rows 8); or int32[2 * count], the
 *         tile schedule of each instance as (lane_target in [1, 64], tile_rows in [1, 32]),
 *         e.g. from lp_tune_schedule.
 *   p     shared parameters (NULL: lp_default_params).  precision 0, 1 and 2 as for lp_solve;
 *         in a batch the FP32 phase of every instance ends before the FP64 phase of any
 *         instance starts.  trace_cap, unroll and persistent are ignored (no trace; the batch
 *         always runs the cooperative loop kernel, 16 iterations per launch).
 * Limits: the sums over the batch of m, of n and of nnz must each be below 2^31
 * (LP_ERR_TOO_LARGE otherwise).  Every row and column is read by one warp at most (lp_solve
 * splits rows longer than 256 entries across warps; the batch does not).
 * Errors: LP_ERR_INVALID_ARG (NULL pointer, count out of range, bad parameters, eta <= 0),
 * LP_ERR_INVALID_INPUT, LP_ERR_TOO_LARGE, LP_ERR_OUT_OF_MEMORY, LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_create(int32_t count, const int32_t* m, const int32_t* n,
                                 const int64_t* nnz, const int64_t* const* row_ptr,
                                 const int32_t* const* col_idx, const double* const* val,
                                 const double* const* c, const double* const* l_c,
                                 const double* const* u_c, const double* const* l_v,
                                 const double* const* u_v, const double* eta,
                                 const int32_t* tiles, const lp_params* p, lp_batch_handle* out);

/*
 * Enqueues one solve of every instance from the zero start on `stream` (a cudaStream_t, NULL for
 * the legacy default stream) and returns.  Each instance stops at its own first check iteration
 * with relative KKT error <= tol, or after max_iter iterations (per phase for precision 1), or
 * on a non-finite residual.  Errors: LP_ERR_INVALID_ARG (NULL handle, tol < 0, max_iter < 1),
 * LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_solve(lp_batch_handle h, double tol, int64_t max_iter, void* stream);

/*
 * Waits for the last solve and copies instance k's result to HOST memory: x (double[n[k]]) and
 * y (double[m[k]]) in the original variables (either may be NULL), the status (LP_SOLVE_*),
 * kkt4 = {relative gap, relative primal residual, relative dual residual, their maximum} of the
 * last check, and the iteration count (both phases).  Errors: LP_ERR_INVALID_ARG (NULL handle,
 * k out of range), LP_ERR_NOT_SOLVED, LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_get(lp_batch_handle h, int32_t k, double* x, double* y,
                              int32_t* status, double* kkt4, int64_t* iters);

/*
 * Waits and copies per-instance summaries to HOST arrays (any may be NULL): status[count],
 * kkt4[4 * count], iters[count], iters_fp32[count] (iterations of the FP32 phase; 0 for
 * precision 0), eta[count] (step size used).  Errors as lp_batch_get.
 */
LP_API lp_status lp_batch_get_all(lp_batch_handle h, int32_t* status, double* kkt4,
                                  int64_t* iters, int64_t* iters_fp32, double* eta);

/*
 * Times the batch loop kernel: runs `iters` iterations of every instance from the zero start
 * (no termination test can stop them: tolerance 0) in FP64 (precision64 != 0) or FP32 and
 * returns the mean device time of one launch (16 iterations) in ms_out[0] and the
 * number of iterations per launch in ms_out[1].  CUDA events on `stream`.  The handle's last
 * solve result is overwritten.  Errors: LP_ERR_INVALID_ARG (FP32 requested on a batch created
 * with precision 0), LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_time_loop(lp_batch_handle h, int64_t iters, int32_t precision64,
                                    void* stream, double* ms_out);

/*
 * Tile-schedule tuner (this library's own; the paper has no counterpart).  For the HOST CSR
 * matrix (row_ptr int64[m+1], col_idx int32[nnz], val double[nnz], validated as in lp_create)
 * it times the batch loop kernel (lp_batch_time_loop, 32 FP64 iterations, CUDA events) on a
 * batch of copies of the matrix (about 4M nonzeros in all, at most 256 copies, all on the grid
 * loop, box bounds [-1, 1] and a fixed objective so that every clamp is exercised) for each
 * schedule (lane_target, tile_rows) in {8, 16, 32} x {1, 8, 32}, and returns the fastest.
 * Results are cached per shape class -- the size classes of m, n, nnz and the share of nonzeros
 * in each row-length and column-length class -- in the process and, if cache_path is not NULL,
 * in that text file (one "class 100*lane_target+tile_rows" line per entry, appended).  A cached
 * class returns without timing unless ms_out is given; ms_out (NULL or double[9]) receives the
 * time per iteration of each candidate, in the order above with lane_target varying fastest.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_INVALID_INPUT, LP_ERR_TOO_LARGE, LP_ERR_OUT_OF_MEMORY,
 * LP_ERR_CUDA.
 */
LP_API lp_status lp_tune_schedule(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                                  const int32_t* col_idx, const double* val, const char* cache_path,
                                  int32_t* lane_target, int32_t* tile_rows, double* ms_out);

/*
 * Where each instance runs, fixed at lp_batch_create: where[k] (HOST int32[count]) is 0 for the
 * cooperative grid loop (nnz[k] > p->batch_local_nnz).  The small instances (the others) run,
 * with gamma = 1 and when every one of them fits it (no row or column longer than 128 entries,
 * each CTA's slices and replicas of the gathered vectors within its shared memory), on the
 * shared-memory cluster loop: 3, clusters of 4 (else 8, 16) blocks holding an instance in shared
 * memory, each claiming instances until all are done.  Otherwise 1 for a cluster of 8 blocks and
 * 2 for a single block (a small instance with at most two row tiles and two column tiles per
 * warp of a block), in two kernels launched side by side.  The schedule solve of the
 * differentiable layer (lp_diff.h) runs small instances on the loops of codes 1 and 2.
 * Errors: LP_ERR_INVALID_ARG (NULL handle or where).
 */
LP_API lp_status lp_batch_schedule(lp_batch_handle h, int32_t* where);

/* Frees the batch (waits for its work first).  NULL is a no-op. */
LP_API void lp_batch_destroy(lp_batch_handle h);

#ifdef __cplusplus
}
#endif

#endif /* PDHG_LP_BATCH_H */
