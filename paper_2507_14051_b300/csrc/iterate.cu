// Iteration kernels of restarted reflected-Halpern PDHG (cuPDLPx, arXiv 2507.14051).
//
// One iteration t has two streaming phases, each fused with its epilogue and followed by a
// deterministic fixed-order reduction and the scalar control:
//
//   row phase (rows of A, gathers xhat_t):
//     deferred Halpern update of the y side decided at t-1 (Section 3, reflected Halpern):
//       y  <- ha*yhat + hb*y + he*y0,  Ax <- ha*Axhat + hb*Ax + he*Ax0   (or <- yhat, Axhat
//       at a restart, which also resets the anchors);
//     v = A xhat_t; A xbar = 2v - Ax (xbar = 2xhat - x);
//     dual step of eq. (pdhg), Section 2.2, in the form yhat = sigma (proj_S(s) - s),
//       s = A xbar - y/sigma;
//     sums |y - yhat|^2, (y - yhat)^T (Ax - Axhat), |yhat - y0|^2 and, on check iterations,
//       the primal residual and the y part of the dual objective (Section 4);
//     control: fixed-point residual r_t = ||z - T z||_P (Section 2.2 P, Section 3), restart
//       test (Section 3, three conditions), PID update of omega (Section 3).
//   column phase (rows of A^T, gathers yhat_t):
//     u = A^T yhat_t; x side of the Halpern update (decided by the row phase of this
//       iteration), the maintained A^T y likewise; next primal step (eq. pdhg first line)
//       xhat_{t+1} = proj_X(x - tau (c - A^T y));
//     sums |x - xhat_{t+1}|^2, |xhat_{t+1} - x0|^2 and, on check iterations, c^T xhat_t, the
//       dual residual and the r part of the dual objective (Section 4);
//     control: relative KKT test (Section 4) -> done / status.
//
// Two drivers run these phases with the same device functions:
//   * k_loop: one cooperative (persistent) kernel that runs up to `iters` iterations, with a
//     grid-wide barrier after each phase; every block then reads all block partials in the same
//     order and computes the same control decision itself (its copy of the scalar state lives
//     in shared memory; block 0 writes it back).  No last-block serialisation, no launches
//     between phases.
//   * k1_rows / k2_cols: one kernel per phase; the block that finishes last reduces the
//     partials and runs the control on the global scalar state.
//
// A x and A^T y of the current iterate are maintained by the same affine updates as x and y
// (exact in exact arithmetic; refreshed from true products at every restart), so one SpMV
// per side per iteration suffices.
#include <cooperative_groups.h>

#include "step.cuh"

namespace cg = cooperative_groups;

namespace pdhg {

// ----------------------------------------------------------- one kernel per phase

template <class V>
__global__ void __launch_bounds__(kThreads, 3) k1_rows(RowArgsT<V> a) {
  Ctl* ctl = a.ctl;
  if (ctl->done) return;
  const RowStep st = row_step(*ctl);
  const V* __restrict__ xh = (ctl->t & 1) ? a.xh1 : a.xh0;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row_pf(a.bins, a.rp, a.ci, a.val, xh, pol, s,
                  [&](int i) {
                    row_prefetch(a, st, i);
                    return NoOperands{};
                  },
                  [&](int i, V v, const NoOperands&, double (&acc)[kNumSums]) { row_epilogue(a, st, i, v, acc); });
  const int nsums = st.check ? 5 : 3;
  if (!block_sums_last(s, nsums, a.partials, &ctl->count1)) return;
  double tot[kNumSums];
  block_totals(a.partials, gridDim.x, nsums, &a.bins, tot);
  if (threadIdx.x != 0) return;
  ctl->count1 = 0;
  row_control(*ctl, tot, st.check, a.trace);
}

template <class V>
__global__ void __launch_bounds__(kThreads, 3) k2_cols(ColArgsT<V> a) {
  Ctl* ctl = a.ctl;
  if (ctl->done) return;
  const ColStepT<V> st = col_step(*ctl, a);
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row_pf(a.bins, a.rp, a.ci, a.val, a.yh, pol, s,
                  [&](int j) {
                    col_prefetch(a, st, j);
                    return NoOperands{};
                  },
                  [&](int j, V u, const NoOperands&, double (&acc)[kNumSums]) { col_epilogue(a, st, j, u, acc); });
  const int nsums = st.check ? 5 : 2;
  if (!block_sums_last(s, nsums, a.partials, &ctl->count2)) return;
  double tot[kNumSums];
  block_totals(a.partials, gridDim.x, nsums, &a.bins, tot);
  if (threadIdx.x != 0) return;
  ctl->count2 = 0;
  col_control(*ctl, tot, st.check);
}

// ------------------------------------------------------------ persistent loop

// Sums each thread's values over the block and stores them as this block's partials.
__device__ __forceinline__ void store_block_partials(double (&s)[kNumSums], int nsums, double* part) {
  block_reduce(s, nsums);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) part[blockIdx.x * kNumSums + q] = s[q];
  }
}

// Runs up to `iters` iterations (fewer if the solve finishes) with a grid-wide barrier after
// each phase.  Must be launched cooperatively with every block resident.  Each block keeps an
// identical copy of the scalar state in shared memory: all blocks read the same partials in the
// same order and run the same control code, so their decisions agree bit for bit and every
// block leaves the loop at the same barrier.  Block 0 writes the state back, writes the trace,
// and (if use_cond) sets the device-side loop condition of the enclosing graph.  4 blocks per
// SM (64 registers) in both precisions: more warps keep more loads in flight (FP64 at 3 blocks
// per SM and 80 registers took 264 us per multicommodity iteration, at 4 with a few spilled
// registers 250 us).
// The phases do not accumulate the PID's norms |yhat - y0|^2 and |xhat - x0|^2 (two FP64
// operations per row and per column on the FP64-bound path): at a restart, which the control
// decides once every many iterations, one extra pass over the four vectors sums them
// (partials in part_pid) before the PID update.
// kRefl: the reflected form of the epilogues (gamma = 1 only; step.cuh), which gathers the
// reflected points xbar and qy instead of xhat and yhat; a restart then also recomputes
// A xhat_t by one SpMV (the next row phase takes it as A x and as the anchor's product).
// kCl: launched as one thread-block cluster (the grid is the cluster, up to 16 CTAs on as many
// SMs), for small LPs; its phase barriers are cluster barriers instead of grid-wide ones.  On
// this GPU an SM issues one FP64 warp instruction per 16 cycles, so even a 2,000-nonzero LP is
// bound by one SM's FP64 issue if one block runs it; a cluster spreads the tiles over its SMs
// and still synchronises in hardware.
template <class V, bool kRefl, bool kCl>
__global__ void __launch_bounds__(kThreads, 4)
    k_loop(RowArgsT<V> ra, ColArgsT<V> ca, double* part_rows, double* part_cols, double* part_pid, int32_t iters,
           cudaGraphConditionalHandle cond, int32_t use_cond) {
  cg::grid_group grid = cg::this_grid();
  // barrier between a phase and the totals of its partials: cluster-wide for a cluster launch
  // (the cluster barrier also orders the CTAs' global stores before their later loads)
  auto phase_sync = [&]() {
    if constexpr (kCl) cg::this_cluster().sync();
    else grid.sync();
  };
  __shared__ Ctl sc;
  __shared__ RowStep rst;
  __shared__ ColStepT<V> cst;
  __shared__ RowStepR<V> rstr;
  __shared__ ColStepR<V> cstr;
  __shared__ Halpern hw;
  __shared__ int rs;
  // whether iterations t and t + 1 are check iterations (reflected form): the 64-bit remainder
  // of the test is computed by the last warp while the row totals are added, not by thread 0 on
  // the serial path at the start of each phase
  __shared__ int chk_cur, chk_nxt;
  __shared__ RestartPre rpre;  // the restart test's thresholds, taken with the Halpern weights
  // reflected form: thread 0 prepares each phase's step scalars at the end of the control
  // before it (a phase then starts without a serial step and a block barrier)
  if (threadIdx.x == 0) {
    sc = *ra.ctl;
    chk_cur = is_check(sc, sc.t) ? 1 : 0;
    if constexpr (kRefl) rstr = row_step_r<V>(sc, chk_cur);
  }
  __syncthreads();
  const LoadPolicy pol = make_policy();
  double* trace = blockIdx.x == 0 ? ra.trace : nullptr;
  for (int32_t it = 0; it < iters && !sc.done; ++it) {
    // ---- row phase
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int check;
    if constexpr (kRefl) {
      const RowStepR<V> st = rstr;
      check = st.check;
      if (check) {  // A xhat_t for the primal residual of the KKT test
        const V* __restrict__ xc = (sc.t & 1) ? ra.xh1 : ra.xh0;
        double z[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
        auto fr1 = [&](int i, V v, double (&)[kNumSums]) { ra.ax[i] = v; };
        for_each_row<V, decltype(fr1)&, kCl>(ra.bins, ra.rp, ra.ci, ra.val, xc, pol, z, fr1);
        phase_sync();
      }
      auto pre1 = [&](int i) {
        row_prefetch_r(ra, st, i);
        return NoOperands{};
      };
      auto epi1 = [&](int i, V w, const NoOperands&, double (&acc)[kNumSums]) {
        row_epilogue_r(ra, st, i, w, acc);
      };
      for_each_row_pf<V, decltype(pre1)&, decltype(epi1)&, kCl>(ra.bins, ra.rp, ra.ci, ra.val, ra.xbar, pol, s, pre1,
                                                             epi1);
    } else {
      if (threadIdx.x == 0) rst = row_step(sc);
      __syncthreads();
      const RowStep st = rst;
      check = st.check;
      const V* __restrict__ xh = (sc.t & 1) ? ra.xh1 : ra.xh0;
      auto pre2 = [&](int i) {
        row_prefetch(ra, st, i);
        return NoOperands{};
      };
      auto epi2 = [&](int i, V v, const NoOperands&, double (&acc)[kNumSums]) {
        row_epilogue<V, false>(ra, st, i, v, acc);
      };
      for_each_row_pf<V, decltype(pre2)&, decltype(epi2)&, kCl>(ra.bins, ra.rp, ra.ci, ra.val, xh, pol, s, pre2,
                                                             epi2);
    }
    const int nr = check ? 5 : 2;
    store_block_partials(s, nr, part_rows);
    phase_sync();
    // the last warp is idle while warps 0..nr-1 add the totals: it computes the next Halpern
    // weights (two FP64 divisions), whether t + 1 is a check iteration and the restart test's
    // thresholds, so that the serial control does not
    if (threadIdx.x == kThreads - 32) {
      hw = halpern_weights(sc.k, sc.gamma);
      chk_nxt = is_check(sc, sc.t + 1) ? 1 : 0;
      rpre = restart_pre(sc);
    }
    double tot[kNumSums];
    block_totals(part_rows, gridDim.x, nr, &ra.bins, tot);
    if (threadIdx.x == 0) {
      rs = row_decide(sc, tot, check, trace, &hw, kRefl ? 1.0 : 2.0, &rpre);
      if constexpr (kRefl)
        if (rs != 1) cstr = col_step_r(sc, ca, chk_cur);
    }
    __syncthreads();
    if (rs == 1) {  // the same decision in every block
      const V* __restrict__ xc = (sc.t & 1) ? ca.xh1 : ca.xh0;  // xhat of this iteration
      double q[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (sc.pid_enabled) {
        const int stride = gridDim.x * kThreads;
        for (int j = blockIdx.x * kThreads + threadIdx.x; j < ca.n; j += stride) {
          const V d = xc[j] - ca.x0[j];
          acc_fma(q[0], d, d);
        }
        for (int i = blockIdx.x * kThreads + threadIdx.x; i < ra.m; i += stride) {
          const V d = ra.yh[i] - ra.y0[i];
          acc_fma(q[1], d, d);
        }
        store_block_partials(q, 2, part_pid);
        phase_sync();
        block_totals(part_pid, gridDim.x, 2, nullptr, q);
      }
      if (threadIdx.x == 0) {
        row_restart_weight(sc, q[0], q[1]);
        if constexpr (kRefl) cstr = col_step_r(sc, ca, chk_cur);  // with the new tau
      }
      if constexpr (kRefl) {
        // A xhat_t, which the next row phase takes as A x and as the new anchor's product (read
        // there after the column phase's barrier)
        double z[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for_each_row(ra.bins, ra.rp, ra.ci, ra.val, xc, pol, z,
                     [&](int i, V v, double (&)[kNumSums]) { ra.axh[i] = v; });
      }
      __syncthreads();
    }
    if (sc.done) break;
    // ---- column phase
    double s2[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if constexpr (kRefl) {
      const ColStepR<V> cs = cstr;
      check = cs.check;
      if (check && !cs.restart) {  // A^T yhat_t for the dual residual of the KKT test
        double z[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
        auto fr2 = [&](int j, V u, double (&)[kNumSums]) { ca.aty[j] = u; };
        for_each_row<V, decltype(fr2)&, kCl>(ca.bins, ca.rp, ca.ci, ca.val, ca.yh, pol, z, fr2);
        phase_sync();
      }
      const V* __restrict__ gy = cs.restart ? ca.yh : ca.qy;
      auto pre3 = [&](int j) {
        col_prefetch_r(ca, cs, j);
        return NoOperands{};
      };
      auto epi3 = [&](int j, V u, const NoOperands&, double (&acc)[kNumSums]) {
        col_epilogue_r(ca, cs, j, u, acc);
      };
      for_each_row_pf<V, decltype(pre3)&, decltype(epi3)&, kCl>(ca.bins, ca.rp, ca.ci, ca.val, gy, pol, s2, pre3,
                                                             epi3);
    } else {
      if (threadIdx.x == 0) cst = col_step(sc, ca);
      __syncthreads();
      const ColStepT<V> cs = cst;
      check = cs.check;
      auto pre4 = [&](int j) {
        col_prefetch(ca, cs, j);
        return NoOperands{};
      };
      auto epi4 = [&](int j, V u, const NoOperands&, double (&acc)[kNumSums]) {
        col_epilogue<V, false>(ca, cs, j, u, acc);
      };
      for_each_row_pf<V, decltype(pre4)&, decltype(epi4)&, kCl>(ca.bins, ca.rp, ca.ci, ca.val, ca.yh, pol, s2, pre4,
                                                             epi4);
    }
    const int nc = check ? 5 : 1;
    store_block_partials(s2, nc, part_cols);
    phase_sync();
    double tot2[kNumSums];
    block_totals(part_cols, gridDim.x, nc, &ca.bins, tot2);
    if (threadIdx.x == 0) {
      col_control(sc, tot2, check);
      chk_cur = chk_nxt;
      if constexpr (kRefl) rstr = row_step_r<V>(sc, chk_cur);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc.bodies += 1;
    if (!sc.done && sc.bodies > sc.max_iter / (iters > 0 ? iters : 1) + 2) {
      sc.status = kInternalError;  // the loop outran max_iter: stop rather than spin
      sc.iters = sc.t + 1;
      sc.done = 1;
    }
    *ra.ctl = sc;
    if (use_cond) cudaGraphSetConditional(cond, sc.done ? 0u : 1u);
  }
}

// ----------------------------------------------------------------- start / misc

// Installs the scalar state of a new solve (built on the host, passed by value so that
// back-to-back solves on one stream cannot race on a host staging buffer).
__global__ void k_init_ctl(Ctl* dst, Ctl src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = src;
}

// First primal step from z = 0: xhat_0 = proj_X(-tau c); zeroes the iterate, the anchors and
// the maintained products; sums |0 - xhat_0|^2 and |xhat_0 - 0|^2 for r_0.
template <class V>
__global__ void __launch_bounds__(kThreads) k_init_cols(int32_t n, const V* __restrict__ c,
                                                        const V* __restrict__ lv,
                                                        const V* __restrict__ uv, V* xh0, V* x,
                                                        V* x0, V* aty, V* aty0, V* xbar, Ctl* ctl,
                                                        double* partials) {
  const V tau = (V)ctl->tau;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const V xn = clampd(-tau * c[j], lv[j], uv[j]);
    xh0[j] = xn;
    if (xbar) xbar[j] = V(2) * xn;  // 2 xhat_0 - x_0 with x_0 = 0
    x[j] = V(0);
    x0[j] = V(0);
    aty[j] = V(0);
    aty0[j] = V(0);
    acc_fma(s[0], xn, xn);
  }
  if (!block_sums_last(s, 1, partials, &ctl->count0)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, nullptr, tot);
  if (threadIdx.x != 0) return;
  ctl->sxx = tot[0];
  ctl->sx0 = tot[0];
  ctl->count0 = 0;
}

template <class V>
__global__ void k_init_rows(int32_t m, V* y, V* y0, V* yh, V* ax, V* ax0, V* axh) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    y[i] = V(0);
    y0[i] = V(0);
    yh[i] = V(0);
    ax[i] = V(0);
    ax0[i] = V(0);
    axh[i] = V(0);
  }
}

// ------------------------------------------------------------- mixed precision

__global__ void k_to_float(int64_t len, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Hand-over kernel of the single-instance solve (switch_ctl in step.cuh).
__global__ void k_switch_ctl(Ctl* ctl, double tol, int64_t max_iter_fp64) {
  switch_ctl(*ctl, tol, max_iter_fp64);
}

// Copies the FP32 phase's returned point to FP64: zhat_T of its last iteration T = iters - 1
// (xhat in the ping-pong buffer of T's parity), or after a stall the best check's zhat from the
// stall guard's slot buffers.  Destination: x and x0 (refinement start) or, for an FP32-only
// solve (or an FP32 phase that ended NUMERICAL, which ends the solve), the FP64 xhat buffer of
// T's parity and yhat.  An FP32-only solve that stalled also reports the best check's KKT values.
// Runs on the FP32 phase's final state, before k_switch_ctl.
__global__ void k_switch_vectors(int32_t n, int32_t m, Ctl* ctl, const float* __restrict__ xh0f,
                                 const float* __restrict__ xh1f, const float* __restrict__ yhf,
                                 const float* __restrict__ xb0, const float* __restrict__ xb1,
                                 const float* __restrict__ yb0, const float* __restrict__ yb1,
                                 double* x, double* x0, double* yh, double* xh0, double* xh1,
                                 int32_t fp32_only) {
  if (ctl->status == kNumerical) fp32_only = 1;
  const int64_t last = ctl->iters - 1;
  const bool best = ctl->status == kStalled && ctl->best_slot >= 0 && xb0 != nullptr;
  const float* xs = best ? (ctl->best_slot ? xb1 : xb0) : ((last & 1) ? xh1f : xh0f);
  const float* ys = best ? (ctl->best_slot ? yb1 : yb0) : yhf;
  double* xo = fp32_only ? ((last & 1) ? xh1 : xh0) : x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)xs[j];
    xo[j] = v;
    if (!fp32_only) x0[j] = v;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    yh[i] = (double)ys[i];
  if (best && fp32_only && blockIdx.x == 0 && threadIdx.x == 0)
    for (int q = 0; q < 8; ++q) ctl->kkt[q] = ctl->kkt_best[q];
}

// FP64 refinement start: xhat = proj_X(x - tau (c - A^T y)) for the given x and A^T y (both
// FP64 already), aty0 = aty, and the sums |x - xhat|^2 = |xhat - x0|^2 (x0 = x).
__global__ void __launch_bounds__(kThreads) k_warm_cols(int32_t n, const double* __restrict__ c,
                                                        const double* __restrict__ lv,
                                                        const double* __restrict__ uv, double* xh0,
                                                        double* xh1, const double* __restrict__ x,
                                                        const double* __restrict__ aty,
                                                        double* __restrict__ aty0, double* xbar,
                                                        Ctl* ctl, double* partials) {
  if (ctl->done) return;  // the FP32 phase ended the solve (NUMERICAL)
  const double tau = ctl->tau;
  double* xh = (ctl->t & 1) ? xh1 : xh0;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double xj = x[j];
    const double xn = clampd(fma(-tau, c[j] - aty[j], xj), lv[j], uv[j]);
    xh[j] = xn;
    if (xbar) xbar[j] = fma(2.0, xn, -xj);
    aty0[j] = aty[j];
    const double d = xj - xn;
    s[0] = fma(d, d, s[0]);
  }
  if (!block_sums_last(s, 1, partials, &ctl->count0)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, nullptr, tot);
  if (threadIdx.x != 0) return;
  ctl->sxx = tot[0];
  ctl->sx0 = tot[0];
  ctl->count0 = 0;
}

// Sets the device-side loop condition of the split-kernel graph: keep iterating while the solve
// is not done.  Guard: each body performs at most `unroll` iterations, so more than
// max_iter/unroll + 2 bodies means the control logic failed to finish the solve; stop with an
// internal-error status instead of looping.
__global__ void k_set_cond(cudaGraphConditionalHandle h, Ctl* ctl, int32_t unroll) {
  ctl->bodies += 1;
  if (!ctl->done && ctl->bodies > ctl->max_iter / unroll + 2) {
    ctl->status = kInternalError;
    ctl->iters = ctl->t + 1;
    ctl->done = 1;
  }
  cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
}

// out[perm[i]] = v[i] * d[i]: permuted, scaled vector back to original order and scale.
__global__ void k_unpermute_scale(int32_t len, const int32_t* __restrict__ perm,
                                  const double* __restrict__ v, const double* __restrict__ d,
                                  double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    out[perm[i]] = v[i] * d[i];
}

// y = A x with the binned schedule (no epilogue), for tests of the SpMV itself.
__global__ void __launch_bounds__(kThreads) k_spmv(const int32_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci,
                                                   const double* __restrict__ val,
                                                   const double* __restrict__ x,
                                                   double* __restrict__ y, BinTable bins) {
  const LoadPolicy pol = make_policy();
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for_each_row(bins, rp, ci, val, x, pol, s, [&](int i, double v, double (&)[kNumSums]) { y[i] = v; });
}

// explicit instantiations for both precisions
template <class V>
IterKernels<V> iter_kernels() {
  IterKernels<V> k;
  k.rows = k1_rows<V>;
  k.cols = k2_cols<V>;
  k.loop = k_loop<V, false, false>;
  k.loop_refl = k_loop<V, true, false>;
  k.loop_one = k_loop<V, false, true>;
  k.loop_refl_one = k_loop<V, true, true>;
  k.init_cols = k_init_cols<V>;
  k.init_rows = k_init_rows<V>;
  return k;
}
template IterKernels<double> iter_kernels<double>();
template IterKernels<float> iter_kernels<float>();

}  // namespace pdhg
