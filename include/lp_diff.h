/*
 * Differentiable unrolled solve over a batch (extension of this library; the paper has no
 * counterpart).  The forward map is K iterations of the method of Sections 2.2 and 3 (primal
 * step, dual step of eq. (pdhg), reflected Halpern update or restart) from the zero start, with
 * the restart schedule and the primal weight frozen: a solve with tolerance 0 and max_iter K
 * records, per instance and iteration t, omega_t, the restart flag and the epoch step k_t; the
 * unrolled map then uses tau_t = eta/omega_t, sigma_t = eta*omega_t and the Halpern weights of
 * k_t.  Between restarts the map is piecewise affine in (c, l_c, u_c, l_v, u_v); its
 * derivative follows the clamp of each step (inside the bounds: derivative 1 in the argument;
 * clamped to a bound: derivative 1 in that bound).  The output is the last step's
 * zhat = (xhat, yhat) in the original variables, as lp_batch_get returns it.
 *
 * Layout of every vector argument: the instances' vectors concatenated in instance order, each
 * in its original variable order (column vectors: sum of n entries; row vectors: sum of m).
 * Pointers are DEVICE memory except where `where` says otherwise.  FP64 only.  A handle keeps
 * the checkpoints of its last lp_batch_unroll; lp_batch_unroll_vjp differentiates that call.
 */
#ifndef PDHG_LP_DIFF_H
#define PDHG_LP_DIFF_H

#include "lp_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Replaces the objective and the bounds of every instance (any argument may be NULL: kept).
 * where = LP_HOST or LP_DEVICE for all five.  The values are scaled and permuted like
 * lp_batch_create's and the KKT denominators are recomputed.  Validation: c finite,
 * l <= u, no +inf lower / -inf upper bound, no NaN (LP_ERR_INVALID_INPUT, host data only;
 * device data is not read back).  Errors: LP_ERR_INVALID_ARG, LP_ERR_INVALID_INPUT, LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_set_data(lp_batch_handle h, const double* c, const double* l_c,
                                   const double* u_c, const double* l_v, const double* u_v,
                                   int32_t where);

/*
 * Forward: records the schedule (a solve of K iterations with tolerance 0) and runs the K
 * unrolled iterations on `stream`, keeping the state (x, y and the Halpern anchors x0, y0)
 * every checkpoint_every iterations.  x (sum n) and y (sum m), device, receive the output
 * zhat; either may be NULL.  Memory: 4 * 8 * (sum n + sum m) bytes per checkpoint and
 * checkpoint_every * (sum n + sum m) bytes of clamp codes.  Requires a batch created with
 * precision 0.  Errors: LP_ERR_INVALID_ARG (K < 1, checkpoint_every < 1, precision != 0),
 * LP_ERR_OUT_OF_MEMORY, LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_unroll(lp_batch_handle h, int64_t K, int64_t checkpoint_every, double* x,
                                 double* y, void* stream);

/*
 * Reverse mode of the last lp_batch_unroll: given dL/dx (sum n) and dL/dy (sum m) at its output
 * (either may be NULL = 0), writes dL/dc, dL/dl_c, dL/du_c, dL/dl_v, dL/du_v (device; any may
 * be NULL).  The adjoint runs backwards segment by segment: each segment's iterations are
 * recomputed from its checkpoint to get their clamp codes, then the adjoint of every
 * iteration is applied (two SpMVs with A^T and A per iteration).  Entries of infinite bounds
 * get 0.  Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED (no forward yet), LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_unroll_vjp(lp_batch_handle h, const double* dl_dx, const double* dl_dy,
                                     double* dl_dc, double* dl_dlc, double* dl_duc, double* dl_dlv,
                                     double* dl_duv, void* stream);

/*
 * The frozen schedule of the last lp_batch_unroll for instance k, to HOST memory: rows t < K of
 * (fixed-point residual r_t, omega_t, restart flag, epoch step k_t), at most cap rows; *rows
 * receives the count.  Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED, LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_get_trace(lp_batch_handle h, int32_t k, double* out, int64_t cap,
                                    int64_t* rows);

/*
 * Kernel timing for roofline reports, after an lp_batch_unroll: runs the first segment's kernels
 * `reps` (>= 1) times each on `stream` with CUDA events around each launch and returns mean
 * milliseconds per launch in ms_out (HOST double[4]): [0] the forward segment kernel without
 * clamp codes (as in lp_batch_unroll), [1] with codes (the recomputation of lp_batch_unroll_vjp),
 * [2] the adjoint segment kernel, [3] iterations per launch (min(K, checkpoint_every)).  The
 * checkpoints and the schedule are left as they were, so a following lp_batch_unroll_vjp is
 * unchanged; the adjoint state is overwritten (zeroed first).  Synchronous.
 * Errors: LP_ERR_INVALID_ARG, LP_ERR_NOT_SOLVED (no forward yet), LP_ERR_CUDA.
 */
LP_API lp_status lp_batch_time_unroll(lp_batch_handle h, int32_t reps, void* stream, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* PDHG_LP_DIFF_H */
