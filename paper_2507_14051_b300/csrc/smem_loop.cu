// k_loop_sm: the single-LP loop kernel over sm_run (smem_loop.cuh), one thread-block cluster that
// holds the whole LP in its CTAs' shared memory for the length of a launch.
#include "smem_loop.cuh"

namespace pdhg {

// One cluster of sp's CTAs (at most kSmMaxCtas; the grid is the cluster), sp.smem_bytes of
// dynamic shared memory each (the largest sm_layout over the CTAs; if that does not hold, the
// launch does nothing but end the solve with an internal error).  Runs up to `iters`
// iterations; rank 0 writes the scalar state back and (if use_cond) sets the enclosing graph's
// loop condition.
template <class V>
__global__ void __launch_bounds__(kThreads, 1)
    k_loop_sm(RowArgsT<V> ra, ColArgsT<V> ca, SmSplit sp, int32_t iters, cudaGraphConditionalHandle cond,
              int32_t use_cond) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Ctl sc;
  if (threadIdx.x == 0) sc = *ra.ctl;
  __syncthreads();
  const bool ok = (int)gridDim.x == (int)cl.num_blocks() &&
                  sm_run<V>(cl, smem, sp.smem_bytes, sc, ra, ca, sp, 0, 0, iters, ra.trace);
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    if (!ok) {
      if (!sc.done) {
        sc.status = kInternalError;
        sc.iters = sc.t;
        sc.done = 1;
      }
    } else {
      sc.bodies += 1;
      if (!sc.done && sc.bodies > sc.max_iter / (iters > 0 ? iters : 1) + 2) {
        sc.status = kInternalError;  // the loop outran max_iter: stop rather than spin
        sc.iters = sc.t + 1;
        sc.done = 1;
      }
    }
    *ra.ctl = sc;
    if (use_cond) cudaGraphSetConditional(cond, sc.done ? 0u : 1u);
  }
}

template <class V>
SmLoopFn<V> sm_loop_kernel() {
  return k_loop_sm<V>;
}
template SmLoopFn<double> sm_loop_kernel<double>();
template SmLoopFn<float> sm_loop_kernel<float>();

}  // namespace pdhg
