// Batched solver (include/lp_batch.h): many independent LPs, each solved by restarted
// reflected-Halpern PDHG with its own restart and PID state (Sections 2.2, 3, 4), in one
// persistent cooperative kernel.
//
// Layout.  The instances are concatenated: global rows, columns and nonzeros, with A and A^T
// stored as block-diagonal CSR matrices (32-bit offsets; column indices of A and row indices
// of A^T are global, so a gather needs no per-instance base).  Inside each instance the rows
// (columns) are permuted by decreasing length class as in the single-instance solver.  Each
// instance's rows are cut into warp tasks (tiles of R rows with G = 32/R lanes per row, about
// lane_target entries per lane); the task lists of all instances are concatenated.
//
// One iteration of the loop kernel:
//   row phase     every warp takes tasks of the instances still running (a prefix sum over
//                 their task counts, rebuilt only when an instance finishes, maps a task number
//                 to its instance); tile SpMV A xhat + row epilogue of step.cuh; the task's
//                 sums go to its slot of a per-task partial array;
//   grid barrier
//   row control   block b handles the running instances b, b + grid, ...: sums its task
//                 partials in a fixed order, runs the restart test and the PID update on a
//                 shared-memory copy of the instance's scalar state;
//   grid barrier, column phase, grid barrier, column control (KKT test), grid barrier.
// Every instance advances by one iteration per loop trip; finished instances drop out of the
// task space.  Results are deterministic (fixed summation orders everywhere).  Instances with
// at most batch_local_nnz nonzeros skip the grid loop: each runs on a cluster of kLocalCtas CTAs
// (kb_cluster_loop) with cluster barriers and distributed-shared-memory totals, or, if it has at
// most two warp tasks per warp of one CTA in each phase, on a single CTA.
//
// The CUDA graph of each precision is a conditional while node around one cooperative launch
// of kBatchUnroll iterations, so a solve needs no host synchronisation.  Mixed precision runs
// the FP32 stage for every instance, then a batched hand-over, then the FP64 stage.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "batch.cuh"
#include "smem_loop.cuh"

namespace cg = cooperative_groups;

namespace pdhg {

// Largest k < nact with pref[k] <= j (pref non-decreasing, pref[0] = 0 <= j).
__device__ __forceinline__ int find_act(const int32_t* pref, int nact, int j) {
  int lo = 0, hi = nact - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Builds in shared memory the running instances (done == 0) in index order with the exclusive
// prefix sums of their row-task and column-task counts.  The whole block calls it.
__device__ void build_active(const int32_t* __restrict__ done, const BInst* __restrict__ inst,
                             int count, int32_t* s_act, int32_t* s_pa, int32_t* s_pt,
                             int32_t* s_nact) {
  __shared__ int32_t wsum[3][kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (count + kThreads - 1) / kThreads;
  const int b = min(count, tid * per), e = min(count, b + per);
  int na = 0, ta = 0, tt = 0;
  for (int i = b; i < e; ++i)
    if (!done[i]) {
      ++na;
      ta += inst[i].nta;
      tt += inst[i].ntt;
    }
  int xa = na, xta = ta, xtt = tt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int ya = __shfl_up_sync(kFull, xa, off);
    const int yta = __shfl_up_sync(kFull, xta, off);
    const int ytt = __shfl_up_sync(kFull, xtt, off);
    if (lane >= off) {
      xa += ya;
      xta += yta;
      xtt += ytt;
    }
  }
  if (lane == 31) {
    wsum[0][warp] = xa;
    wsum[1][warp] = xta;
    wsum[2][warp] = xtt;
  }
  __syncthreads();
  int oa = xa - na, ota = xta - ta, ott = xtt - tt;
  for (int w = 0; w < warp; ++w) {
    oa += wsum[0][w];
    ota += wsum[1][w];
    ott += wsum[2][w];
  }
  for (int i = b; i < e; ++i)
    if (!done[i]) {
      s_act[oa] = i;
      s_pa[oa] = ota;
      s_pt[oa] = ott;
      ++oa;
      ota += inst[i].nta;
      ott += inst[i].ntt;
    }
  if (tid == kThreads - 1) {
    *s_nact = oa;
    s_pa[oa] = ota;
    s_pt[oa] = ott;
  }
  __syncthreads();
}

// Cooperative copies of one instance's scalar state between global and shared memory.
__device__ __forceinline__ void ctl_load(Ctl* dst, const Ctl* src) {
  static_assert(sizeof(Ctl) % 8 == 0, "Ctl is copied as 8-byte words");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int w = threadIdx.x; w < (int)(sizeof(Ctl) / 8); w += blockDim.x) d[w] = s[w];
}

__device__ __forceinline__ BCol make_bcol(const Ctl& c) {
  BCol b;
  b.restart = c.restart;
  b.check = is_check(c, c.t) ? 1 : 0;
  b.cand = c.cand_slot;
  b.par = (int32_t)(c.t & 1);
  b.ha = c.ha;
  b.hb = c.hb;
  b.he = c.he;
  b.tau = c.tau;
  return b;
}

__device__ __forceinline__ BRow make_brow(const Ctl& c) {
  BRow b;
  b.st = row_step(c);
  b.par = (int32_t)(c.t & 1);
  return b;
}

// Sums the first ns partials of tasks [t0, t0 + nt) in a fixed order (thread-strided, then the
// block tree); totals in thread 0.
__device__ __forceinline__ void sum_task_partials(const double* __restrict__ part, int t0, int nt, int ns,
                                                  double (&s)[kNumSums]) {
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) s[q] = 0.0;
  for (int t = threadIdx.x; t < nt; t += kThreads) {
    const double* p = part + (size_t)(t0 + t) * kNumSums;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q)
      if (q < ns) s[q] += p[q];
  }
  block_reduce(s, ns);
}

template <class V>
__device__ __forceinline__ void row_phase(const BatchArgs<V>& a, const int32_t* s_act, const int32_t* s_pa,
                                          int nact, const LoadPolicy& pol) {
  const int lane = threadIdx.x & 31;
  const int total = s_pa[nact];
  const int nw = gridDim.x * kWarps;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < total; j += nw) {
    const int k = find_act(s_pa, nact, j);
    const int ii = s_act[k];
    const int tix = a.inst[ii].ta0 + (j - s_pa[k]);
    const int4 td = a.tasksA[tix];
    const BRow br = a.rstep[ii];
    const V* __restrict__ xg = br.par ? a.ra.xh1 : a.ra.xh0;
    if (lane < td.y) row_prefetch(a.ra, br.st, td.x + lane);
    const V v = tile_spmv(a.ra.rp, a.ra.ci, a.ra.val, xg, td.x, td.y, task_lanes(td), task_per_lane(td),
                          lane, pol);
    double acc[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (lane < td.y) row_epilogue(a.ra, br.st, td.x + lane, v, acc);
    const int ns = br.st.check ? 5 : 3;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q)
      if (q < ns) acc[q] = warp_sum(acc[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < kNumSums; ++q)
        if (q < ns) a.tpartA[(size_t)tix * kNumSums + q] = acc[q];
    }
  }
}

template <class V>
__device__ __forceinline__ void col_phase(const BatchArgs<V>& a, const int32_t* s_act, const int32_t* s_pt,
                                          int nact, const LoadPolicy& pol) {
  const int lane = threadIdx.x & 31;
  const int total = s_pt[nact];
  const int nw = gridDim.x * kWarps;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < total; j += nw) {
    const int k = find_act(s_pt, nact, j);
    const int ii = s_act[k];
    const int tix = a.inst[ii].tt0 + (j - s_pt[k]);
    const int4 td = a.tasksT[tix];
    const BCol bc = a.cstep[ii];
    ColStepT<V> st;
    st.restart = bc.restart;
    st.check = bc.check;
    st.cand = bc.cand;
    st.ha = bc.ha;
    st.hb = bc.hb;
    st.he = bc.he;
    st.tau = bc.tau;
    st.xc = bc.par ? a.ca.xh1 : a.ca.xh0;
    st.xn = bc.par ? a.ca.xh0 : a.ca.xh1;
    if (lane < td.y) col_prefetch(a.ca, st, td.x + lane);
    const V u = tile_spmv(a.ca.rp, a.ca.ci, a.ca.val, a.ca.yh, td.x, td.y, task_lanes(td),
                          task_per_lane(td), lane, pol);
    double acc[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (lane < td.y) col_epilogue(a.ca, st, td.x + lane, u, acc);
    const int ns = bc.check ? 5 : 2;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q)
      if (q < ns) acc[q] = warp_sum(acc[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < kNumSums; ++q)
        if (q < ns) a.tpartT[(size_t)tix * kNumSums + q] = acc[q];
    }
  }
}

// Re-reads the batch's finished count after a grid barrier and rebuilds the running list if it
// changed.  Every block sees the same count (nothing writes it between a barrier and the next
// control phase), so every block builds the same list.
template <class V>
__device__ __forceinline__ void refresh_active(const BatchArgs<V>& a, int32_t* s_act, int32_t* s_pa,
                                               int32_t* s_pt, int32_t* s_nact, unsigned* s_seen) {
  __shared__ unsigned now;
  if (threadIdx.x == 0) now = *(volatile unsigned*)&a.bc->n_done;
  __syncthreads();
  if (now != *s_seen) {
    build_active(a.done, a.inst, a.count, s_act, s_pa, s_pt, s_nact);
    if (threadIdx.x == 0) *s_seen = now;
    __syncthreads();
  }
}

// The batch loop: up to `iters` iterations of every running instance.  Cooperative launch with
// every block resident.  Block 0 counts the launch and (if use_cond) sets the graph's loop
// condition: continue while an instance is running, unless the launches outran max_iter.
// 3 blocks per SM in both precisions (4 for FP32 measured slower: more blocks at each barrier).
template <class V>
__global__ void __launch_bounds__(kThreads, 3)
    kb_loop(BatchArgs<V> a, int32_t iters, cudaGraphConditionalHandle cond, int32_t use_cond) {
  cg::grid_group grid = cg::this_grid();
  __shared__ int32_t s_act[kMaxInst];
  __shared__ int32_t s_pa[kMaxInst + 1];
  __shared__ int32_t s_pt[kMaxInst + 1];
  __shared__ int32_t s_nact;
  __shared__ unsigned s_seen;
  __shared__ Ctl sc;
  const LoadPolicy pol = make_policy();
  if (threadIdx.x == 0) s_seen = 0xFFFFFFFFu;
  __syncthreads();
  for (int32_t it = 0; it < iters; ++it) {
    refresh_active(a, s_act, s_pa, s_pt, &s_nact, &s_seen);
    const int nact = s_nact;
    if (nact == 0) break;
    // ---- row phase
    row_phase(a, s_act, s_pa, nact, pol);
    grid.sync();
    // ---- row control: restart test and PID update per instance
    for (int k = blockIdx.x; k < nact; k += gridDim.x) {
      const int ii = s_act[k];
      const BInst I = a.inst[ii];
      const int check = a.rstep[ii].st.check;
      double tot[kNumSums];
      sum_task_partials(a.tpartA, I.ta0, I.nta, check ? 5 : 3, tot);
      ctl_load(&sc, a.ctl + ii);
      __syncthreads();
      if (threadIdx.x == 0) {
        row_control(sc, tot, check != 0, trace_of(a, ii));
        a.cstep[ii] = make_bcol(sc);
        if (sc.done) {
          a.done[ii] = 1;
          atomicAdd(&a.bc->n_done, 1u);
        }
      }
      __syncthreads();
      ctl_load(a.ctl + ii, &sc);
      __syncthreads();
    }
    grid.sync();
    refresh_active(a, s_act, s_pa, s_pt, &s_nact, &s_seen);
    const int nact2 = s_nact;
    if (nact2 == 0) break;
    // ---- column phase
    col_phase(a, s_act, s_pt, nact2, pol);
    grid.sync();
    // ---- column control: KKT test per instance
    for (int k = blockIdx.x; k < nact2; k += gridDim.x) {
      const int ii = s_act[k];
      const BInst I = a.inst[ii];
      const int check = a.cstep[ii].check;
      double tot[kNumSums];
      sum_task_partials(a.tpartT, I.tt0, I.ntt, check ? 5 : 2, tot);
      ctl_load(&sc, a.ctl + ii);
      __syncthreads();
      if (threadIdx.x == 0) {
        col_control(sc, tot, check != 0);
        a.rstep[ii] = make_brow(sc);
        if (sc.done) {
          a.done[ii] = 1;
          atomicAdd(&a.bc->n_done, 1u);
        }
      }
      __syncthreads();
      ctl_load(a.ctl + ii, &sc);
      __syncthreads();
    }
    grid.sync();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    BatchCtl* b = a.bc;
    b->bodies += 1;
    bool more = *(volatile unsigned*)&b->n_done < (unsigned)a.count;
    if (more && b->bodies > b->max_bodies) {
      b->overrun = 1;  // the control failed to finish the stage: stop rather than spin
      more = false;
    }
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

// Start of a stage: every instance's scalar state from its template (step size, omega0, KKT
// denominators, parameters), with the stage's tolerance, iteration limit and stall guard.
// The small (cluster-loop) instances are marked done for the grid loop (n_local of them).
__global__ void kb_init_ctl(int32_t count, const Ctl* __restrict__ init, const BInst* __restrict__ inst,
                            Ctl* ctl, int32_t* done, BRow* rstep, BatchCtl* bc, double tol,
                            int64_t max_iter, int32_t patience, int64_t max_bodies, int32_t n_local,
                            int64_t trace_cap) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    Ctl c = init[k];
    c.tol = tol;
    c.max_iter = max_iter;
    c.patience = patience;
    c.trace_cap = trace_cap;
    c.best_kkt = INFINITY;
    c.cand_slot = 0;
    c.best_slot = -1;
    ctl[k] = c;
    done[k] = inst[k].local;  // the grid loop skips the small (cluster-local) instances
    rstep[k] = make_brow(c);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    bc->n_done = (unsigned)n_local;
    bc->overrun = 0;
    bc->bodies = 0;
    bc->max_bodies = max_bodies;
  }
}

// First primal step of every instance from z = 0 (block per instance): xhat_0 = proj_X(-tau c),
// the other vectors zeroed, |xhat_0|^2 summed for r_0.
template <class V>
__global__ void __launch_bounds__(kThreads) kb_init(BatchArgs<V> a) {
  for (int k = blockIdx.x; k < a.count; k += gridDim.x) {
    const BInst I = a.inst[k];
    const V tau = (V)a.ctl[k].tau;
    for (int i = I.row0 + threadIdx.x; i < I.row0 + I.m; i += kThreads) {
      a.ra.y[i] = V(0);
      a.ra.y0[i] = V(0);
      a.ra.yh[i] = V(0);
      a.ra.ax[i] = V(0);
      a.ra.ax0[i] = V(0);
      a.ra.axh[i] = V(0);
      a.ra.qy[i] = V(0);
      a.ra.w[i] = V(0);
    }
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = I.col0 + threadIdx.x; j < I.col0 + I.n; j += kThreads) {
      const V xn = clampd(-tau * a.ca.c[j], a.ca.lv[j], a.ca.uv[j]);
      a.ca.xh0[j] = xn;
      a.ca.xbar[j] = V(2) * xn;  // 2 xhat_0 - x_0 (x_0 = 0), for the shared-memory loop
      a.ca.x[j] = V(0);
      a.ca.x0[j] = V(0);
      a.ca.aty[j] = V(0);
      a.ca.aty0[j] = V(0);
      s[0] += (double)xn * (double)xn;
    }
    block_reduce(s, 1);
    if (threadIdx.x == 0) {
      a.ctl[k].sxx = s[0];
      a.ctl[k].sx0 = s[0];
    }
    __syncthreads();
  }
}

// End of the FP32 stage (block per instance): the stage's returned point (its last zhat, or
// after a stall the best check's zhat) goes to the FP64 buffers -- as x and anchor x0 of the
// FP64 stage (mixed), or as the FP64 output xhat / yhat (FP32 only, or an instance that ended
// NUMERICAL).  For the mixed solve the scalar state is then handed over (switch_ctl).
__global__ void __launch_bounds__(kThreads) kb_switch(BatchArgs<float> f, BatchArgs<double> d, double tol,
                                                      int64_t max_iter, int32_t fp32_only) {
  __shared__ int32_t s_final, s_best;
  __shared__ int64_t s_last;
  for (int k = blockIdx.x; k < d.count; k += gridDim.x) {
    const BInst I = d.inst[k];
    if (threadIdx.x == 0) {
      const Ctl& c = d.ctl[k];
      s_final = fp32_only || c.status == kNumerical;
      s_best = (c.status == kStalled && c.best_slot >= 0) ? c.best_slot : -1;
      s_last = c.iters - 1;
    }
    __syncthreads();
    const int fin = s_final, best = s_best;
    const int64_t last = s_last;
    const float* xs = best >= 0 ? (best ? f.ca.xb1 : f.ca.xb0) : ((last & 1) ? f.ca.xh1 : f.ca.xh0);
    const float* ys = best >= 0 ? (best ? f.ra.yb1 : f.ra.yb0) : f.ra.yh;
    double* xo = fin ? ((last & 1) ? d.ca.xh1 : d.ca.xh0) : d.ca.x;
    for (int j = I.col0 + threadIdx.x; j < I.col0 + I.n; j += kThreads) {
      const double v = (double)xs[j];
      xo[j] = v;
      if (!fin) d.ca.x0[j] = v;
    }
    for (int i = I.row0 + threadIdx.x; i < I.row0 + I.m; i += kThreads) d.ra.yh[i] = (double)ys[i];
    if (threadIdx.x == 0) {
      Ctl& c = d.ctl[k];
      if (fp32_only) {
        if (best >= 0)
          for (int q = 0; q < 8; ++q) c.kkt[q] = c.kkt_best[q];
      } else {
        switch_ctl(c, tol, max_iter);
        const int32_t skip = (c.done || I.local) ? 1 : 0;  // the grid loop skips both
        d.done[k] = skip;
        if (skip) atomicAdd(&d.bc->n_done, 1u);
      }
    }
    __syncthreads();
  }
}

// First FP64 primal step after the hand-over (block per instance): xhat = proj_X(x - tau (c -
// A^T y)) from the FP64 x and A^T yhat, aty0 = aty, |x - xhat|^2; the row step of the first FP64
// iteration.
__global__ void __launch_bounds__(kThreads) kb_warm(BatchArgs<double> d, int64_t max_bodies) {
  for (int k = blockIdx.x; k < d.count; k += gridDim.x) {
    if (d.ctl[k].done) continue;  // block-uniform: ended NUMERICAL in the FP32 stage
    const BInst I = d.inst[k];
    const Ctl& c = d.ctl[k];
    const double tau = c.tau;
    double* xh = (c.t & 1) ? d.ca.xh1 : d.ca.xh0;
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = I.col0 + threadIdx.x; j < I.col0 + I.n; j += kThreads) {
      const double xj = d.ca.x[j], atyj = d.ca.aty[j];
      const double xn = clampd(fma(-tau, d.ca.c[j] - atyj, xj), d.ca.lv[j], d.ca.uv[j]);
      xh[j] = xn;
      d.ca.xbar[j] = fma(2.0, xn, -xj);  // for the shared-memory loop (reflected form)
      d.ca.aty0[j] = atyj;
      const double df = xj - xn;
      s[0] = fma(df, df, s[0]);
    }
    block_reduce(s, 1);
    if (threadIdx.x == 0) {
      Ctl& cw = d.ctl[k];
      cw.sxx = s[0];
      cw.sx0 = s[0];
      d.rstep[k] = make_brow(cw);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.bc->bodies = 0;
    d.bc->overrun = 0;
    d.bc->max_bodies = max_bodies;
  }
}

// Loop for the small instances: a cluster of kCtas CTAs (on kCtas SMs) runs every iteration of
// one instance, then claims the next unclaimed instance of the list (`next`, zeroed before the
// launch): the instances' iteration counts are unknown and uneven, so a static assignment could
// queue two long ones on one cluster.  Which cluster runs an instance does not change its bits.  Each CTA takes every kCtas-th of the instance's warp tasks and sums its
// threads' epilogue sums (block tree); the CTAs' totals meet in distributed shared memory after
// a cluster barrier, every CTA adds them in rank order and runs the same control on its own
// shared-memory copy of the scalar state, so all copies agree bit for bit and the CTAs leave
// the loop together.  Two cluster barriers per iteration; the iteration's arithmetic is spread
// over kCtas SMs' FP64 units instead of one.  It continues from the instance's current state
// until it is done; `cap` bounds the iterations of one launch (a guard: the control ends every
// solve by max_iter).
template <int kCtas>
__device__ __forceinline__ void cluster_barrier() {
  if (kCtas > 1) cg::this_cluster().sync();
  else __syncthreads();
}

template <int kCtas>
__device__ __forceinline__ void cluster_totals(const double* part, int nsums, double (&tot)[kNumSums]) {
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) tot[q] = 0.0;
  for (int r = 0; r < kCtas; ++r) {
    const double* p = kCtas > 1 ? cg::this_cluster().map_shared_rank(const_cast<double*>(part), r) : part;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q)
      if (q < nsums) tot[q] += p[q];
  }
}

template <class V, int kCtas>
__global__ void __launch_bounds__(kThreads, 2) kb_cluster_loop(BatchArgs<V> a, const int32_t* __restrict__ list,
                                                               int32_t nlist, int32_t* next, int64_t cap) {
  __shared__ Ctl sc;
  __shared__ int32_t claim;  // the list entry this cluster runs next
  __shared__ RowStep rst;
  __shared__ ColStepT<V> cst;
  __shared__ double part[2][kNumSums];  // this CTA's row-phase and column-phase totals
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = (int)(blockIdx.x % kCtas);
  const int w0 = rank * kWarps + warp, wstep = kCtas * kWarps;
  for (;;) {
    // rank 0 claims an entry and hands it to every CTA of the cluster (each CTA finished the
    // previous instance before the barrier that ended it, so no CTA still reads `claim`)
    if (rank == 0 && threadIdx.x == 0) {
      const int32_t q = atomicAdd(next, 1);
      for (int r = 0; r < kCtas; ++r) {
        int32_t* dst = kCtas > 1 ? cg::this_cluster().map_shared_rank(&claim, r) : &claim;
        *dst = q;
      }
    }
    cluster_barrier<kCtas>();
    const int q = claim;
    if (q >= nlist) break;
    const int ii = list[q];
    const BInst I = a.inst[ii];
    ctl_load(&sc, a.ctl + ii);
    __syncthreads();
    int64_t guard = 0;
    while (!sc.done && guard < cap) {
      ++guard;
      if (threadIdx.x == 0) rst = row_step(sc);
      __syncthreads();
      const RowStep st = rst;
      const V* __restrict__ xg = (sc.t & 1) ? a.ra.xh1 : a.ra.xh0;
      double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = w0; j < I.nta; j += wstep) {
        const int4 td = a.tasksA[I.ta0 + j];
        const V v = tile_spmv<V, true>(a.ra.rp, a.ra.ci, a.ra.val, xg, td.x, td.y, task_lanes(td),
                                       task_per_lane(td), lane, pol);
        if (lane < td.y) row_epilogue(a.ra, st, td.x + lane, v, s);
      }
      const int nr = st.check ? 5 : 3;
      block_reduce(s, nr);
      if (threadIdx.x == 0)
        for (int k = 0; k < kNumSums; ++k) part[0][k] = s[k];
      cluster_barrier<kCtas>();
      if (threadIdx.x == 0) {
        double tot[kNumSums];
        cluster_totals<kCtas>(part[0], nr, tot);
        row_control(sc, tot, st.check != 0, rank == 0 ? trace_of(a, ii) : nullptr);
      }
      __syncthreads();
      if (sc.done) break;
      if (threadIdx.x == 0) cst = col_step(sc, a.ca);
      __syncthreads();
      const ColStepT<V> cs = cst;
      double s2[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = w0; j < I.ntt; j += wstep) {
        const int4 td = a.tasksT[I.tt0 + j];
        const V u = tile_spmv<V, true>(a.ca.rp, a.ca.ci, a.ca.val, a.ca.yh, td.x, td.y, task_lanes(td),
                                       task_per_lane(td), lane, pol);
        if (lane < td.y) col_epilogue(a.ca, cs, td.x + lane, u, s2);
      }
      const int nc = cs.check ? 5 : 2;
      block_reduce(s2, nc);
      if (threadIdx.x == 0)
        for (int k = 0; k < kNumSums; ++k) part[1][k] = s2[k];
      cluster_barrier<kCtas>();
      if (threadIdx.x == 0) {
        double tot[kNumSums];
        cluster_totals<kCtas>(part[1], nc, tot);
        col_control(sc, tot, cs.check != 0);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && !sc.done) {  // the guard tripped: stop with an internal error
      sc.status = kInternalError;
      sc.iters = sc.t + 1;
      sc.done = 1;
    }
    __syncthreads();
    if (rank == 0) ctl_load(a.ctl + ii, &sc);
    cluster_barrier<kCtas>();  // every CTA has read this instance's totals before the next one
  }
}

// The small instances in shared memory: a cluster of sm_ctas CTAs claims an entry of the list
// (`next`, zeroed before the launch), runs its instance to the end with sm_run (the single-LP
// shared-memory loop, reflected form) from its current state, writes the instance's scalar
// state back and claims the next entry.  splits[q]: the row / column split of entry q.  An
// instance's bits do not depend on which cluster runs it.  A split that does not fit, or an
// instance the control did not end within `cap` iterations, ends with an internal error.
template <class V>
__global__ void __launch_bounds__(kThreads, 1)
    kb_sm_loop(BatchArgs<V> a, const int32_t* __restrict__ list, int32_t nlist, int32_t* next,
               const SmSplit* __restrict__ splits, int32_t smem_bytes, int64_t cap) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Ctl sc;
  __shared__ int32_t claim;
  const int rank = (int)cl.block_rank(), nct = (int)cl.num_blocks();
  const int32_t iters = cap > (int64_t)0x7fffffff ? 0x7fffffff : (int32_t)cap;
  for (;;) {
    // every CTA finished the previous instance before the barrier that ended it
    if (rank == 0 && threadIdx.x == 0) {
      const int32_t q = atomicAdd(next, 1);
      for (int r = 0; r < nct; ++r) *cl.map_shared_rank(&claim, (unsigned)r) = q;
    }
    cl.sync();
    const int q = claim;
    if (q >= nlist) break;
    const int ii = list[q];
    const BInst I = a.inst[ii];
    if (threadIdx.x == 0) sc = a.ctl[ii];
    __syncthreads();
    if (!sc.done) {  // the same in every CTA
      RowArgsT<V> ra = a.ra;
      ColArgsT<V> ca = a.ca;
      const int r0 = I.row0, c0 = I.col0;
      ra.rp += r0;
      ra.xh0 += c0;
      ra.xh1 += c0;
      ra.y += r0;
      ra.y0 += r0;
      ra.yh += r0;
      ra.ax += r0;
      ra.ax0 += r0;
      ra.axh += r0;
      ra.lc += r0;
      ra.uc += r0;
      ra.inv_dr += r0;
      if (ra.yb0) ra.yb0 += r0;
      if (ra.yb1) ra.yb1 += r0;
      ra.qy += r0;
      ra.w += r0;
      ra.xbar += c0;
      ra.m = I.m;
      ca.rp += c0;
      ca.yh += r0;
      ca.xh0 += c0;
      ca.xh1 += c0;
      ca.x += c0;
      ca.x0 += c0;
      ca.aty += c0;
      ca.aty0 += c0;
      ca.c += c0;
      ca.lv += c0;
      ca.uv += c0;
      ca.inv_dc += c0;
      if (ca.xb0) ca.xb0 += c0;
      if (ca.xb1) ca.xb1 += c0;
      ca.xbar += c0;
      ca.qy += r0;
      ca.n = I.n;
      const bool ok = sm_run<V>(cl, smem, smem_bytes, sc, ra, ca, splits[q], r0, c0, iters, trace_of(a, ii));
      if (threadIdx.x == 0 && (!ok || !sc.done)) {
        sc.status = kInternalError;
        sc.iters = ok ? sc.t + 1 : sc.t;
        sc.done = 1;
      }
    }
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) a.ctl[ii] = sc;
    cl.sync();
  }
}

// Power iteration (Section 3, "Stepsize"), every instance at once: u = start vector / |.|,
// then repeatedly w = s A u, lambda = |w|^2, u = A^T w, s = 1/|u|, with the single-instance
// solver's stopping rule per instance.
__global__ void __launch_bounds__(kThreads) kb_pw_start(const BInst* __restrict__ inst, int32_t count,
                                                        const int32_t* __restrict__ col_perm, uint64_t seed,
                                                        double* __restrict__ u, BPw* pw) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const BInst I = inst[k];
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = I.col0 + threadIdx.x; j < I.col0 + I.n; j += kThreads) {
      const double v = start_entry(seed, (uint64_t)col_perm[j]);
      u[j] = v;
      s[0] = fma(v, v, s[0]);
    }
    block_reduce(s, 1);
    if (threadIdx.x == 0) {
      BPw p;
      p.lam = 0.0;
      p.prev = 0.0;
      p.s = s[0] > 0.0 ? 1.0 / sqrt(s[0]) : 0.0;
      p.done = (I.m == 0 || I.n == 0) ? 1 : 0;
      p.iters = 0;
      pw[k] = p;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) kb_pw_rows(const BInst* __restrict__ inst, int32_t count,
                                                       double* __restrict__ w, BPw* pw, double tol) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    if (pw[k].done) continue;  // block-uniform
    const BInst I = inst[k];
    const double sc = pw[k].s;
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = I.row0 + threadIdx.x; i < I.row0 + I.m; i += kThreads) {
      const double v = w[i] * sc;
      w[i] = v;
      s[0] = fma(v, v, s[0]);
    }
    block_reduce(s, 1);
    if (threadIdx.x == 0) {
      BPw& p = pw[k];
      const double lam = s[0];
      p.iters += 1;
      p.lam = lam;
      if (lam == 0.0) p.done = 1;
      else if (p.iters > 1 && fabs(lam - p.prev) <= tol * lam) p.done = 1;
      else p.prev = lam;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) kb_pw_cols(const BInst* __restrict__ inst, int32_t count,
                                                       const double* __restrict__ u, BPw* pw) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    if (pw[k].done) continue;
    const BInst I = inst[k];
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = I.col0 + threadIdx.x; j < I.col0 + I.n; j += kThreads) s[0] = fma(u[j], u[j], s[0]);
    block_reduce(s, 1);
    if (threadIdx.x == 0) pw[k].s = s[0] > 0.0 ? 1.0 / sqrt(s[0]) : 0.0;
    __syncthreads();
  }
}

// y = A x over the tasks of the instances whose power iteration is still running (a finished
// instance's vectors are no longer read).
__global__ void __launch_bounds__(kThreads) kb_pw_spmv(const int4* __restrict__ tasks, int32_t ntasks,
                                                       const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ x, double* __restrict__ y,
                                                       const BPw* __restrict__ pw) {
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < ntasks; j += gridDim.x * kWarps) {
    const int4 td = tasks[j];
    if (pw[td.w].done) continue;  // warp-uniform
    const double v = tile_spmv(rp, ci, val, x, td.x, td.y, task_lanes(td), task_per_lane(td), lane, pol);
    if (lane < td.y) y[td.x + lane] = v;
  }
}

__global__ void kb_pw_count(const BPw* __restrict__ pw, int32_t count, BatchCtl* bc) {
  __shared__ unsigned int left;
  if (threadIdx.x == 0) left = 0;
  __syncthreads();
  unsigned mine = 0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) mine += pw[k].done ? 0u : 1u;
  atomicAdd(&left, mine);
  __syncthreads();
  if (threadIdx.x == 0) bc->pw_left = left;
}

}  // namespace pdhg

using namespace pdhg;
using namespace pdhg_host;

// ====================================================================== host side

namespace {

// Tiles of rows already sorted by decreasing length class, shaped by tile_shape (the
// single-instance schedule without chunks: a row of any length gets at most one warp).
void make_tasks(const std::vector<int32_t>& rp, int lane_target, int tile_rows, int32_t row_base, int32_t inst,
                std::vector<int4>& out) {
  const int32_t rows = (int32_t)rp.size() - 1;
  int32_t r = 0;
  while (r < rows) {
    const int cls = length_class(rp[r + 1] - rp[r]);
    int32_t e = r + 1;
    while (e < rows && length_class(rp[e + 1] - rp[e]) == cls) ++e;
    const TileShape ts = tile_shape(int64_t(1) << cls, lane_target, tile_rows);
    const int32_t pl = ts.per_lane < 0xFFFFFF ? ts.per_lane : 0xFFFFFF;
    for (int32_t q = r; q < e; q += ts.rows)
      out.push_back(make_int4(row_base + q, std::min<int32_t>(ts.rows, e - q), (ts.lanes << 24) | pl, inst));
    r = e;
  }
}

// One instance's host-side structure: permutations, permuted CSR of A and A^T (global indices),
// tasks, KKT denominators.
struct Built {
  std::vector<int32_t> row_perm, col_perm;
  std::vector<int32_t> rlen_perm, clen_perm;
  std::vector<int4> tA, tT;
  double c_norm = 0.0, lu_norm = 0.0;
};

template <class V>
cudaError_t launch_batch_loop(const lp_batch* h, const BatchArgs<V>& a, int32_t iters,
                              cudaGraphConditionalHandle cond, int32_t use_cond, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(sizeof(V) == sizeof(float) ? h->grid32 : h->grid));
  cfg.blockDim = dim3((unsigned)kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kb_loop<V>, a, iters, cond, use_cond);
}

// The small instances' loop: clusters of kLocalCtas CTAs over the clustered list, and single
// CTAs over the tiny instances, the two launches running side by side (a second stream, joined
// back into s by an event).
template <class V, int kCtas>
cudaError_t launch_cluster_loop(const lp_batch* h, const BatchArgs<V>& a, const int32_t* list, int32_t n,
                                int64_t cap, cudaStream_t s) {
  const int clusters = std::max(1, std::min(n, 2 * h->num_sms / kCtas));
  int32_t* next = h->local_next + (kCtas == 1 ? 1 : 0);
  const cudaError_t e0 = cudaMemsetAsync(next, 0, sizeof(int32_t), s);
  if (e0 != cudaSuccess) return e0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(clusters * kCtas));
  cfg.blockDim = dim3((unsigned)kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kb_cluster_loop<V, kCtas>, a, list, n, next, cap);
}

// The clustered small instances on clusters of k CTAs (8, 4 or 2).
template <class V>
cudaError_t launch_wide(const lp_batch* h, const BatchArgs<V>& a, int k, int64_t cap, cudaStream_t s) {
  if (k == 4) return launch_cluster_loop<V, 4>(h, a, h->local_list, h->n_wide, cap, s);
  if (k == 2) return launch_cluster_loop<V, 2>(h, a, h->local_list, h->n_wide, cap, s);
  return launch_cluster_loop<V, kLocalCtas>(h, a, h->local_list, h->n_wide, cap, s);
}

// The small instances on the shared-memory loop: as many clusters of sm_ctas CTAs as fit on the
// device at once, each claiming instances until the list is done.
template <class V>
cudaError_t launch_sm_loop(const lp_batch* h, const BatchArgs<V>& a, int64_t cap, cudaStream_t s) {
  const int C = h->sm_ctas;
  const int32_t bytes = h->sm_bytes[sizeof(V) == sizeof(float) ? 1 : 0];
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3((unsigned)kThreads);
  cfg.dynamicSmemBytes = (size_t)bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)C);
  int fit = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&fit, kb_sm_loop<V>, &cfg);
  if (e != cudaSuccess) return e;
  const int clusters = std::max(1, std::min(h->n_local, fit));
  cfg.gridDim = dim3((unsigned)(clusters * C));
  e = cudaMemsetAsync(h->local_next, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, kb_sm_loop<V>, a, (const int32_t*)h->local_list, h->n_local, h->local_next,
                            (const SmSplit*)h->d_splits, bytes, cap);
}

// one_wave: clusters of the most CTAs (8, 4, 2) with which every clustered instance has its own
// cluster at once.  A solve to tolerance keeps 8 (its small stragglers run longest, so each
// instance's own speed decides); the schedule solve of the differentiable map runs exactly K
// iterations of every instance, so a second wave of clusters would cost a second pass.
template <class V>
cudaError_t launch_local(const lp_batch* h, const BatchArgs<V>& a, int64_t cap, cudaStream_t s,
                         bool one_wave = false) {
  // a solve runs the small instances in shared memory when they fit; the schedule solve of the
  // differentiable map keeps the plain-form loops, whose schedule its adjoint replays
  if (h->sm_ctas > 0 && !one_wave) return launch_sm_loop<V>(h, a, cap, s);
  const int32_t n_tiny = h->n_local - h->n_wide;
  int k = kLocalCtas;
  if (one_wave)
    while (k > 2 && (int64_t)h->n_wide * k > 2 * (int64_t)h->num_sms) k >>= 1;
  cudaError_t e = cudaSuccess;
  if (h->n_wide > 0 && n_tiny > 0) {
    e = cudaEventRecord(h->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0);
    if (e == cudaSuccess) e = launch_cluster_loop<V, 1>(h, a, h->local_list + h->n_wide, n_tiny, cap, h->side_stream);
    if (e == cudaSuccess) e = launch_wide<V>(h, a, k, cap, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
    return e;
  }
  if (h->n_wide > 0) return launch_wide<V>(h, a, k, cap, s);
  return launch_cluster_loop<V, 1>(h, a, h->local_list, n_tiny, cap, s);
}

template <class V>
lp_status build_batch_graph(lp_batch* h, cudaGraph_t* graph, cudaGraphExec_t* exec) {
  BatchArgs<V> a;
  fill_batch_args<V>(h, a);
  CK(cudaGraphCreate(graph, 0));
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, *graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, *graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t s = h->setup_stream;
  CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const cudaError_t le = launch_batch_loop<V>(h, a, kBatchUnroll, cond, 1, s);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &captured);
  if (e == cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, *graph, 0);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  return LP_OK;
}

// Runs fn(k) for k in [0, count) on up to hardware_concurrency threads; returns the first
// failure by instance order.
template <class Fn>
lp_status parallel_for(int32_t count, Fn&& fn) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthreads = (int)std::min<unsigned>(hw, (unsigned)std::max(1, count));
  std::vector<lp_status> st(count, LP_OK);
  std::vector<std::string> msg(count);
  std::atomic<int32_t> next{0};
  auto worker = [&]() {
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= count) return;
      st[k] = fn(k, msg[k]);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  for (int32_t k = 0; k < count; ++k)
    if (st[k] != LP_OK) return fail(st[k], msg[k]);
  return LP_OK;
}

lp_status batch_power_iteration(lp_batch* h) {
  cudaStream_t s = h->setup_stream;
  double* u = h->x;  // scratch until the first solve
  double* w = h->y;
  kb_pw_start<<<h->gridS, kThreads, 0, s>>>(h->d_inst, h->count, h->col_perm, h->prm.power_seed, u, h->pw);
  CK(cudaGetLastError());
  const int gA = grid_for(h->ntA, kWarps, 8 * h->num_sms), gT = grid_for(h->ntT, kWarps, 8 * h->num_sms);
  unsigned left = 1;
  int64_t it = 0;
  while (left > 0 && it < h->prm.power_max_iter) {
    const int64_t rest = h->prm.power_max_iter - it;
    const int batch = rest < kPwBatch ? (int)rest : kPwBatch;
    for (int q = 0; q < batch; ++q) {
      kb_pw_spmv<<<gA, kThreads, 0, s>>>(h->tasksA, h->ntA, h->rpA, h->ciA, h->valA, u, w, h->pw);
      kb_pw_rows<<<h->gridS, kThreads, 0, s>>>(h->d_inst, h->count, w, h->pw, h->prm.power_tol);
      kb_pw_spmv<<<gT, kThreads, 0, s>>>(h->tasksT, h->ntT, h->rpT, h->ciT, h->valT, w, u, h->pw);
      kb_pw_cols<<<h->gridS, kThreads, 0, s>>>(h->d_inst, h->count, u, h->pw);
    }
    kb_pw_count<<<1, kThreads, 0, s>>>(h->pw, h->count, h->bc);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&left, &h->bc->pw_left, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    it += batch;
  }
  std::vector<BPw> pw(h->count);
  CK(cudaMemcpy(pw.data(), h->pw, sizeof(BPw) * h->count, cudaMemcpyDeviceToHost));
  for (int32_t k = 0; k < h->count; ++k) {
    const double nrm = std::sqrt(pw[k].lam);
    h->eta[k] = nrm > 0.0 ? 0.998 / nrm : 1.0;
  }
  return LP_OK;
}

// Sets up the shared-memory loop for the small instances (`local`, with their host build data B)
// if every one of them fits it (gamma = 1, the reflected form; no row or column longer than
// kSmMaxLen; each CTA's slices and replicas within its shared memory): the smallest cluster
// (4, 8 or 16 CTAs) that takes them all, their splits uploaded in list order.  Leaves
// h->sm_ctas = 0 (the cluster and single-CTA loops) otherwise.
lp_status setup_batch_sm(lp_batch* h, const std::vector<Built>& B, const std::vector<int32_t>& local) {
  h->sm_ctas = 0;
  if (local.empty() || h->prm.gamma != 1.0) return LP_OK;
  for (int32_t k : local) {
    const Built& b = B[k];
    for (size_t i = 0; i + 1 < b.rlen_perm.size(); ++i)
      if (b.rlen_perm[i + 1] - b.rlen_perm[i] > kSmMaxLen) return LP_OK;
    for (size_t j = 0; j + 1 < b.clen_perm.size(); ++j)
      if (b.clen_perm[j + 1] - b.clen_perm[j] > kSmMaxLen) return LP_OK;
  }
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
    cudaGetLastError();
    return LP_OK;
  }
  const int nprec = h->prm.precision != 0 ? 2 : 1;
  std::vector<SmSplit> sp(local.size());
  for (int C : {4, 8, 16}) {
    uint64_t mx[2] = {0, 0};
    for (size_t q = 0; q < local.size(); ++q) {
      const Built& b = B[local[q]];
      SmSplit& s = sp[q];
      s = SmSplit{};
      sm_slices(b.rlen_perm, C, s.rs);
      sm_slices(b.clen_perm, C, s.cs);
      const int64_t mk = (int64_t)b.rlen_perm.size() - 1, nk = (int64_t)b.clen_perm.size() - 1;
      for (int r = 0; r < C; ++r) {
        const int32_t a0 = s.rs[r], a1 = s.rs[r + 1], c0 = s.cs[r], c1 = s.cs[r + 1];
        for (int pr = 0; pr < nprec; ++pr) {
          const uint64_t t = sm_layout(mk, nk, a1 - a0, c1 - c0, b.rlen_perm[a1] - b.rlen_perm[a0],
                                       b.clen_perm[c1] - b.clen_perm[c0], pr == 0 ? 8 : 4).total;
          mx[pr] = t > mx[pr] ? t : mx[pr];
        }
      }
    }
    bool ok = true;
    for (int pr = 0; pr < nprec && ok; ++pr) {
      const void* kern = pr == 0 ? (const void*)kb_sm_loop<double> : (const void*)kb_sm_loop<float>;
      cudaFuncAttributes fa{};
      ok = cudaFuncGetAttributes(&fa, kern) == cudaSuccess && mx[pr] + fa.sharedSizeBytes <= (uint64_t)optin &&
           cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx[pr]) == cudaSuccess &&
           (C <= 8 || cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess);
      if (ok) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3((unsigned)kThreads);
        cfg.dynamicSmemBytes = (size_t)mx[pr];
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0;
      }
    }
    cudaGetLastError();
    if (!ok) continue;
    CK(h->alloc(&h->d_splits, sp.size()));
    CK(cudaMemcpy(h->d_splits, sp.data(), sizeof(SmSplit) * sp.size(), cudaMemcpyHostToDevice));
    h->sm_ctas = C;
    h->sm_bytes[0] = (int32_t)mx[0];
    h->sm_bytes[1] = (int32_t)mx[1];
    return LP_OK;
  }
  return LP_OK;
}

lp_status batch_create_impl(lp_batch* h, const int32_t* m, const int32_t* n, const int64_t* nnz,
                            const int64_t* const* rp, const int32_t* const* ci, const double* const* val,
                            const double* const* c, const double* const* lc, const double* const* uc,
                            const double* const* lv, const double* const* uv, const double* eta,
                            const int32_t* tiles) {
  const int32_t K = h->count;

  // ---- sizes and offsets ----
  h->inst.assign(K, BInst{});
  int64_t sm = 0, sn = 0, snz = 0;
  for (int32_t k = 0; k < K; ++k) {
    if (m[k] < 0 || n[k] < 0 || nnz[k] < 0) return fail(LP_ERR_INVALID_ARG, "negative size in instance " + std::to_string(k));
    if (m[k] > 0 && (!rp[k] || (nnz[k] > 0 && (!ci[k] || !val[k])) || !lc[k] || !uc[k]))
      return fail(LP_ERR_INVALID_ARG, "NULL array in instance " + std::to_string(k));
    if (!rp[k] || (n[k] > 0 && (!c[k] || !lv[k] || !uv[k])))
      return fail(LP_ERR_INVALID_ARG, "NULL array in instance " + std::to_string(k));
    h->inst[k].row0 = (int32_t)std::min<int64_t>(sm, INT32_MAX);
    h->inst[k].col0 = (int32_t)std::min<int64_t>(sn, INT32_MAX);
    h->inst[k].m = m[k];
    h->inst[k].n = n[k];
    sm += m[k];
    sn += n[k];
    snz += nnz[k];
  }
  if (sm >= INT32_MAX || sn >= INT32_MAX || snz >= INT32_MAX)
    return fail(LP_ERR_TOO_LARGE, "the batch's total rows, columns and nonzeros must each be below 2^31");
  h->sum_m = sm;
  h->sum_n = sn;
  h->sum_nnz = snz;
  std::vector<int64_t> nz0(K + 1, 0);
  for (int32_t k = 0; k < K; ++k) nz0[k + 1] = nz0[k] + nnz[k];

  // ---- pass 1 (host threads): validation, permutations, tasks, KKT denominators ----
  std::vector<Built> B(K);
  lp_status st = parallel_for(K, [&](int32_t k, std::string& msg) -> lp_status {
    const int32_t mk = m[k], nk = n[k];
    const int64_t zk = nnz[k];
    lp_status v = validate(mk, nk, zk, rp[k], ci[k], val[k], c[k], lc[k], uc[k], lv[k], uv[k]);
    if (v != LP_OK) {
      msg = "instance " + std::to_string(k) + ": " + lp_last_error();
      return v;
    }
    Built& b = B[k];
    double c2 = 0.0, lu2 = 0.0;
    for (int32_t j = 0; j < nk; ++j) c2 += c[k][j] * c[k][j];
    for (int32_t i = 0; i < mk; ++i) {
      if (std::isfinite(lc[k][i])) lu2 += lc[k][i] * lc[k][i];
      if (std::isfinite(uc[k][i])) lu2 += uc[k][i] * uc[k][i];
    }
    b.c_norm = std::sqrt(c2);
    b.lu_norm = std::sqrt(lu2);
    std::vector<int64_t> rlen(mk), clen(nk, 0);
    for (int32_t i = 0; i < mk; ++i) rlen[i] = rp[k][i + 1] - rp[k][i];
    for (int64_t p = 0; p < zk; ++p) clen[ci[k][p]]++;
    order_by_class(rlen, b.row_perm);
    order_by_class(clen, b.col_perm);
    std::vector<int32_t> rpl(mk + 1), cpl(nk + 1);
    rpl[0] = 0;
    for (int32_t i = 0; i < mk; ++i) rpl[i + 1] = rpl[i] + (int32_t)rlen[b.row_perm[i]];
    cpl[0] = 0;
    for (int32_t j = 0; j < nk; ++j) cpl[j + 1] = cpl[j] + (int32_t)clen[b.col_perm[j]];
    const int lt = tiles ? tiles[2 * k] : (h->prm.lane_target > 0 ? h->prm.lane_target : kBatchLaneTarget);
    const int tr = tiles ? tiles[2 * k + 1] : (h->prm.tile_rows > 0 ? h->prm.tile_rows : kBatchTileRows);
    make_tasks(rpl, lt, tr, h->inst[k].row0, k, b.tA);
    make_tasks(cpl, lt, tr, h->inst[k].col0, k, b.tT);
    b.rlen_perm.swap(rpl);
    b.clen_perm.swap(cpl);
    return LP_OK;
  });
  if (st != LP_OK) return st;
  int64_t ta = 0, tt = 0;
  for (int32_t k = 0; k < K; ++k) {
    h->inst[k].ta0 = (int32_t)ta;
    h->inst[k].nta = (int32_t)B[k].tA.size();
    h->inst[k].tt0 = (int32_t)tt;
    h->inst[k].ntt = (int32_t)B[k].tT.size();
    ta += (int64_t)B[k].tA.size();
    tt += (int64_t)B[k].tT.size();
  }
  if (ta >= INT32_MAX || tt >= INT32_MAX) return fail(LP_ERR_TOO_LARGE, "too many tasks");
  // small instances: clustered ones first, then the tiny ones (at most two warp tasks per warp
  // of one CTA in each phase), which one CTA runs with less synchronisation
  std::vector<int32_t> local, tiny;
  for (int32_t k = 0; k < K; ++k) {
    h->inst[k].local = (nnz[k] <= h->prm.batch_local_nnz) ? 1 : 0;
    if (!h->inst[k].local) continue;
    if (std::max(h->inst[k].nta, h->inst[k].ntt) <= 2 * kWarps) tiny.push_back(k);
    else local.push_back(k);
  }
  h->n_wide = (int32_t)local.size();
  local.insert(local.end(), tiny.begin(), tiny.end());
  h->n_local = (int32_t)local.size();
  h->ntA = (int32_t)ta;
  h->ntT = (int32_t)tt;

  // ---- device buffers (the first CUDA calls: bad input is refused before them) ----
  CK(cudaGetDevice(&h->device));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  CK(cudaStreamCreateWithFlags(&h->setup_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  CK(h->alloc(&h->rpA, sm + 1)); CK(h->alloc(&h->ciA, snz)); CK(h->alloc(&h->valA, snz));
  CK(h->alloc(&h->rpT, sn + 1)); CK(h->alloc(&h->ciT, snz)); CK(h->alloc(&h->valT, snz));
  CK(h->alloc(&h->row_perm, sm)); CK(h->alloc(&h->col_perm, sn));
  for (double** p : {&h->c, &h->lv, &h->uv, &h->inv_dc, &h->dc, &h->x, &h->x0, &h->xh0, &h->xh1, &h->aty, &h->aty0,
                     &h->xbar})
    CK(h->alloc(p, sn));
  for (double** p : {&h->lc, &h->uc, &h->inv_dr, &h->dr, &h->y, &h->y0, &h->yh, &h->ax, &h->ax0, &h->axh,
                     &h->qy, &h->w})
    CK(h->alloc(p, sm));
  {
    int64_t mx = 1;
    for (int32_t k = 0; k < K; ++k) mx = std::max<int64_t>(mx, std::max(m[k], n[k]));
    CK(h->alloc(&h->out_buf, mx));
  }
  CK(h->alloc(&h->tasksA, ta)); CK(h->alloc(&h->tasksT, tt));
  CK(h->alloc(&h->tpartA, (size_t)std::max<int64_t>(ta, 1) * kNumSums));
  CK(h->alloc(&h->tpartT, (size_t)std::max<int64_t>(tt, 1) * kNumSums));
  CK(h->alloc(&h->d_inst, K)); CK(h->alloc(&h->ctl, K)); CK(h->alloc(&h->ctl_init, K));
  CK(h->alloc(&h->rstep, K)); CK(h->alloc(&h->cstep, K)); CK(h->alloc(&h->done, K));
  CK(h->alloc(&h->bc, 1)); CK(h->alloc(&h->pw, K));
  CK(cudaMemset(h->ctl, 0, sizeof(Ctl) * K));
  CK(cudaMemset(h->bc, 0, sizeof(BatchCtl)));
  CK(cudaMemset(h->done, 0, sizeof(int32_t) * K));
  CK(cudaMemcpy(h->d_inst, h->inst.data(), sizeof(BInst) * K, cudaMemcpyHostToDevice));
  h->local_host = local;
  CK(h->alloc(&h->local_list, local.size()));
  CK(h->alloc(&h->local_next, 2));
  if (!local.empty()) CK(cudaMemcpy(h->local_list, local.data(), sizeof(int32_t) * local.size(), cudaMemcpyHostToDevice));

  // ---- pass 2 (host threads): permuted CSR of A and A^T with global indices, upload ----
  const int dev = h->device;
  st = parallel_for(K, [&](int32_t k, std::string& msg) -> lp_status {
    cudaError_t e = cudaSetDevice(dev);
    const Built& b = B[k];
    const BInst& I = h->inst[k];
    const int32_t mk = m[k], nk = n[k];
    const int64_t zk = nnz[k];
    const int32_t z0 = (int32_t)nz0[k];
    std::vector<int32_t> col_inv(nk);
    for (int32_t j = 0; j < nk; ++j) col_inv[b.col_perm[j]] = j;
    std::vector<int32_t> rpA(mk + 1), ciA(zk), rpT(nk + 1), ciT(zk), cursor(nk);
    std::vector<double> valA(zk), valT(zk);
    for (int32_t i = 0; i <= mk; ++i) rpA[i] = z0 + b.rlen_perm[i];
    for (int32_t j = 0; j <= nk; ++j) rpT[j] = z0 + b.clen_perm[j];
    for (int32_t i = 0; i < mk; ++i) {
      const int32_t o = b.row_perm[i];
      int32_t q = b.rlen_perm[i];
      for (int64_t p = rp[k][o]; p < rp[k][o + 1]; ++p, ++q) {
        ciA[q] = I.col0 + col_inv[ci[k][p]];
        valA[q] = val[k][p];
      }
    }
    for (int32_t j = 0; j < nk; ++j) cursor[j] = b.clen_perm[j];
    for (int32_t i = 0; i < mk; ++i)
      for (int32_t q = b.rlen_perm[i]; q < b.rlen_perm[i + 1]; ++q) {
        const int32_t pos = cursor[ciA[q] - I.col0]++;
        ciT[pos] = I.row0 + i;
        valT[pos] = valA[q];
      }
    // rp arrays: instance k writes rows [row0, row0 + m) and the entry at row0 + m (equal to
    // the next instance's first offset, so concurrent writers store the same value)
    if (e == cudaSuccess) e = cudaMemcpy(h->rpA + I.row0, rpA.data(), sizeof(int32_t) * (mk + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->rpT + I.col0, rpT.data(), sizeof(int32_t) * (nk + 1), cudaMemcpyHostToDevice);
    if (zk > 0) {
      if (e == cudaSuccess) e = cudaMemcpy(h->ciA + z0, ciA.data(), sizeof(int32_t) * zk, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(h->valA + z0, valA.data(), sizeof(double) * zk, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(h->ciT + z0, ciT.data(), sizeof(int32_t) * zk, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(h->valT + z0, valT.data(), sizeof(double) * zk, cudaMemcpyHostToDevice);
    }
    std::vector<double> tmp(std::max(mk, nk));
    auto up = [&](double* dst, const double* src, int32_t len, const std::vector<int32_t>& perm) {
      if (e != cudaSuccess || len == 0) return;
      for (int32_t q = 0; q < len; ++q) tmp[q] = src[perm[q]];
      e = cudaMemcpy(dst, tmp.data(), sizeof(double) * len, cudaMemcpyHostToDevice);
    };
    up(h->c + I.col0, c[k], nk, b.col_perm);
    up(h->lv + I.col0, lv[k], nk, b.col_perm);
    up(h->uv + I.col0, uv[k], nk, b.col_perm);
    up(h->lc + I.row0, lc[k], mk, b.row_perm);
    up(h->uc + I.row0, uc[k], mk, b.row_perm);
    if (e == cudaSuccess && mk > 0) e = cudaMemcpy(h->row_perm + I.row0, b.row_perm.data(), sizeof(int32_t) * mk, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nk > 0) e = cudaMemcpy(h->col_perm + I.col0, b.col_perm.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b.tA.empty()) e = cudaMemcpy(h->tasksA + I.ta0, b.tA.data(), sizeof(int4) * b.tA.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b.tT.empty()) e = cudaMemcpy(h->tasksT + I.tt0, b.tT.data(), sizeof(int4) * b.tT.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      msg = std::string("upload of instance ") + std::to_string(k) + ": " + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? LP_ERR_OUT_OF_MEMORY : LP_ERR_CUDA;
    }
    return LP_OK;
  });
  if (st != LP_OK) return st;
  if (sm == 0) CK(cudaMemset(h->rpA, 0, sizeof(int32_t)));
  if (sn == 0) CK(cudaMemset(h->rpT, 0, sizeof(int32_t)));

  // ---- diagonal preconditioning of the block-diagonal matrix (per row / column, so per
  //      instance) ----
  cudaStream_t s = h->setup_stream;
  const int gV = grid_for(std::max(sm, sn), kThreads, 4 * h->num_sms);
  {
    std::vector<double> ones(std::max<int64_t>(std::max(sm, sn), 1), 1.0);
    if (sn > 0) CK(cudaMemcpy(h->dc, ones.data(), sizeof(double) * sn, cudaMemcpyHostToDevice));
    if (sm > 0) CK(cudaMemcpy(h->dr, ones.data(), sizeof(double) * sm, cudaMemcpyHostToDevice));
  }
  // a copy from pageable memory returns once its source is staged, possibly before its last
  // transfer lands, and the setup stream does not wait on the default stream: wait here
  CK(cudaDeviceSynchronize());
  const int passes = h->prm.ruiz_iters + (h->prm.pc_enabled ? 1 : 0);
  if (passes > 0 && snz > 0) {
    double* fr = h->y;
    double* fc = h->x;
    const int gr = grid_for(sm * 32, 256, 8 * h->num_sms);
    const int gc = grid_for(sn * 32, 256, 8 * h->num_sms);
    for (int pass = 0; pass < passes; ++pass) {
      const int kind = (pass == h->prm.ruiz_iters) ? 1 : 0;
      // the batch's rows are not ordered by length across instances: a warp per row throughout
      if (sm > 0)
        k_row_factor<<<gr, 256, 0, s>>>((int32_t)sm, (int32_t)sm, h->rpA, h->valA, kind, 2.0 - h->prm.pc_alpha, fr);
      if (sn > 0) k_row_factor<<<gc, 256, 0, s>>>((int32_t)sn, (int32_t)sn, h->rpT, h->valT, kind, h->prm.pc_alpha, fc);
      if (sm > 0) k_apply_factors<<<gr, 256, 0, s>>>((int32_t)sm, (int32_t)sm, h->rpA, h->ciA, h->valA, fr, fc, 0);
      if (sn > 0) k_apply_factors<<<gc, 256, 0, s>>>((int32_t)sn, (int32_t)sn, h->rpT, h->ciT, h->valT, fr, fc, 1);
      if (sm > 0) k_mul_inplace<<<gV, 256, 0, s>>>((int32_t)sm, h->dr, fr);
      if (sn > 0) k_mul_inplace<<<gV, 256, 0, s>>>((int32_t)sn, h->dc, fc);
    }
    CK(cudaGetLastError());
  }
  if (sn > 0) k_scale_cols<<<gV, 256, 0, s>>>((int32_t)sn, h->dc, h->c, h->lv, h->uv, h->inv_dc);
  if (sm > 0) k_scale_rows<<<gV, 256, 0, s>>>((int32_t)sm, h->dr, h->lc, h->uc, h->inv_dr);
  CK(cudaGetLastError());

  // ---- grids ----
  int occ64 = 0, occ32 = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, kb_loop<double>, kThreads, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, kb_loop<float>, kThreads, 0));
  h->grid = std::max(1, occ64) * h->num_sms;
  h->grid32 = std::max(1, occ32) * h->num_sms;
  h->gridS = std::max(1, std::min<int>(K, 8 * h->num_sms));

  // ---- the small instances' shared-memory loop ----
  st = setup_batch_sm(h, B, local);
  if (st != LP_OK) return st;

  // ---- step sizes ----
  CK(cudaStreamSynchronize(s));  // the scaled data below is read back by the host
  h->eta.assign(K, 0.0);
  if (eta) {
    for (int32_t k = 0; k < K; ++k) h->eta[k] = eta[k];
  } else if (h->prm.eta > 0.0) {
    for (int32_t k = 0; k < K; ++k) h->eta[k] = h->prm.eta;
  } else {
    st = batch_power_iteration(h);
    if (st != LP_OK) return st;
  }

  // ---- scalar-state templates ----
  std::vector<double> ratio(K, 1.0);
  if (h->prm.rescale) {
    std::vector<double> hc(sn), hl(sm), hu(sm);
    if (sn > 0) CK(cudaMemcpy(hc.data(), h->c, sizeof(double) * sn, cudaMemcpyDeviceToHost));
    if (sm > 0) CK(cudaMemcpy(hl.data(), h->lc, sizeof(double) * sm, cudaMemcpyDeviceToHost));
    if (sm > 0) CK(cudaMemcpy(hu.data(), h->uc, sizeof(double) * sm, cudaMemcpyDeviceToHost));
    for (int32_t k = 0; k < K; ++k) {
      const BInst& I = h->inst[k];
      ratio[k] = rescale_ratio(hc.data() + I.col0, I.n, hl.data() + I.row0, hu.data() + I.row0, I.m);
    }
  }
  std::vector<Ctl> init(K);
  for (int32_t k = 0; k < K; ++k) {
    Ctl& ci0 = init[k];
    ci0 = Ctl{};
    const double e0 = h->eta[k], om = h->prm.omega0 * (h->prm.rescale ? ratio[k] : 1.0);
    ci0.eta = e0;
    ci0.omega = om;
    ci0.tau = e0 / om;
    ci0.sigma = e0 * om;
    ci0.inv_sigma = 1.0 / (e0 * om);
    ci0.w_over_eta = om / e0;
    ci0.inv_eta_w = 1.0 / (e0 * om);
    ci0.restart_enabled = h->prm.restart_enabled;
    ci0.pid_enabled = h->prm.pid_enabled;
    ci0.check_every = h->prm.check_every;
    ci0.trace_cap = 0;
    ci0.omega_used = om;
    for (int q = 0; q < 8; ++q) ci0.kkt[q] = NAN;
    ci0.lu_norm = B[k].lu_norm;
    ci0.c_norm = B[k].c_norm;
    ci0.gamma = h->prm.gamma;
    ci0.beta_s = h->prm.beta_sufficient;
    ci0.beta_n = h->prm.beta_necessary;
    ci0.beta_a = h->prm.beta_artificial;
    ci0.kp = h->prm.k_p;
    ci0.ki = h->prm.k_i;
    ci0.kd = h->prm.k_d;
  }
  CK(cudaMemcpy(h->ctl_init, init.data(), sizeof(Ctl) * K, cudaMemcpyHostToDevice));

  // ---- FP32 copies ----
  if (h->prm.precision != 0) {
    auto& f = h->f32;
    CK(h->alloc(&f.valA, snz)); CK(h->alloc(&f.valT, snz));
    for (float** q : {&f.c, &f.lv, &f.uv, &f.inv_dc, &f.x, &f.x0, &f.xh0, &f.xh1, &f.aty, &f.aty0, &f.xb0, &f.xb1,
                      &f.xbar})
      CK(h->alloc(q, sn));
    for (float** q : {&f.lc, &f.uc, &f.inv_dr, &f.y, &f.y0, &f.yh, &f.ax, &f.ax0, &f.axh, &f.yb0, &f.yb1,
                      &f.qy, &f.w})
      CK(h->alloc(q, sm));
    const int g = grid_for(std::max<int64_t>(snz, 1), 256, 8 * h->num_sms);
    k_to_float<<<g, 256, 0, s>>>(snz, h->valA, f.valA);
    k_to_float<<<g, 256, 0, s>>>(snz, h->valT, f.valT);
    for (auto pr : {std::make_pair((const double*)h->c, f.c), std::make_pair((const double*)h->lv, f.lv),
                    std::make_pair((const double*)h->uv, f.uv), std::make_pair((const double*)h->inv_dc, f.inv_dc)})
      k_to_float<<<gV, 256, 0, s>>>(sn, pr.first, pr.second);
    for (auto pr : {std::make_pair((const double*)h->lc, f.lc), std::make_pair((const double*)h->uc, f.uc),
                    std::make_pair((const double*)h->inv_dr, f.inv_dr)})
      k_to_float<<<gV, 256, 0, s>>>(sm, pr.first, pr.second);
    CK(cudaGetLastError());
  }
  CK(cudaDeviceSynchronize());  // the setup stream's work and the state templates' copy

  st = build_batch_graph<double>(h, &h->graph64, &h->exec64);
  if (st != LP_OK) return st;
  if (h->prm.precision != 0) {
    st = build_batch_graph<float>(h, &h->graph32, &h->exec32);
    if (st != LP_OK) return st;
  }
  return LP_OK;
}

int64_t bodies_for(int64_t max_iter) { return max_iter / kBatchUnroll + 2; }

template <class V>
lp_status enqueue_batch_start(lp_batch* h, double tol, int64_t max_iter, int32_t patience, cudaStream_t s) {
  const int g = grid_for(h->count, 256, 4 * h->num_sms);
  kb_init_ctl<<<g, 256, 0, s>>>(h->count, h->ctl_init, h->d_inst, h->ctl, h->done, h->rstep, h->bc, tol,
                                max_iter, patience, bodies_for(max_iter), h->n_local, 0);
  BatchArgs<V> a;
  fill_batch_args<V>(h, a);
  kb_init<V><<<h->gridS, kThreads, 0, s>>>(a);
  CK(cudaGetLastError());
  return LP_OK;
}

// One stage of precision V: the grid loop over the grid instances (graph), then the cluster
// loop over the small ones.
template <class V>
lp_status enqueue_stage(lp_batch* h, cudaGraphExec_t exec, int64_t max_iter, cudaStream_t s) {
  if (h->n_local < h->count) CK(cudaGraphLaunch(exec, s));
  if (h->n_local > 0) {
    BatchArgs<V> a;
    fill_batch_args<V>(h, a);
    CK(launch_local<V>(h, a, max_iter + 2, s));
  }
  return LP_OK;
}

lp_batch* checked(lp_batch_handle h) { return h; }

}  // namespace

// Differentiation support: a solve of exactly K FP64 iterations (tolerance 0) of every
// instance that records each instance's trace rows (r, omega, restart flag, k): the frozen
// schedule of the unrolled map.
lp_status batch_schedule_solve(lp_batch* h, int64_t K, cudaStream_t s) {
  if (h->trace_cap < K) {
    cudaFree(h->trace);
    h->trace = nullptr;
    h->trace_cap = 0;
    CK(cudaMalloc(&h->trace, sizeof(double) * 4 * (size_t)K * (size_t)h->count));
    h->trace_cap = K;
  }
  const int g = grid_for(h->count, 256, 4 * h->num_sms);
  kb_init_ctl<<<g, 256, 0, s>>>(h->count, h->ctl_init, h->d_inst, h->ctl, h->done, h->rstep, h->bc, 0.0, K, 0,
                                bodies_for(K), h->n_local, h->trace_cap);
  BatchArgs<double> a;
  fill_batch_args<double>(h, a);
  a.trace = h->trace;
  a.trace_cap = h->trace_cap;
  kb_init<double><<<h->gridS, kThreads, 0, s>>>(a);
  CK(cudaGetLastError());
  if (h->n_local < h->count) {
    const int64_t launches = (K + kBatchUnroll - 1) / kBatchUnroll;
    for (int64_t q = 0; q < launches; ++q)
      CK(launch_batch_loop<double>(h, a, kBatchUnroll, cudaGraphConditionalHandle{}, 0, s));
  }
  if (h->n_local > 0) CK(launch_local<double>(h, a, K + 2, s, true));
  h->solved = true;
  h->last_stream = s;
  return LP_OK;
}


// ------------------------------------------------------------------ schedule tuner

namespace {

// Candidate tile schedules (lane_target, tile_rows).
constexpr int kTuneLane[] = {8, 16, 32, 8, 16, 32, 8, 16, 32};
constexpr int kTuneRows[] = {1, 1, 1, 8, 8, 8, 32, 32, 32};
constexpr int kTuneN = 9;

// Length-class signature of a CSR (rows) and of its transpose (columns): the schedule depends
// on the matrix only through these, so they key the cache together with the sizes' classes.
std::string shape_class(int32_t m, int32_t n, int64_t nnz, const int64_t* rp, const int32_t* ci) {
  std::vector<int64_t> rc(34, 0), cc(34, 0), clen(n, 0);
  for (int32_t i = 0; i < m; ++i) rc[length_class(rp[i + 1] - rp[i])] += rp[i + 1] - rp[i];
  for (int64_t p = 0; p < nnz; ++p) clen[ci[p]]++;
  for (int32_t j = 0; j < n; ++j) cc[length_class(clen[j])] += clen[j];
  // the classes holding most nonzeros, in tenths of nnz
  std::string key = "m" + std::to_string(length_class(m)) + "n" + std::to_string(length_class(n)) +
                    "z" + std::to_string(length_class(nnz));
  for (auto* h : {&rc, &cc}) {
    key += nnz > 0 ? "|" : "|-";
    for (int c = 0; c < 34 && nnz > 0; ++c) {
      const int64_t tenth = (10 * (*h)[c] + nnz / 2) / nnz;
      if (tenth > 0) key += std::to_string(c) + ":" + std::to_string(tenth) + ",";
    }
  }
  return key;
}

std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

bool cache_lookup(const std::string& key, const char* path, int* best) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(key);
  if (it != g_tune_cache.end()) {
    *best = it->second;
    return true;
  }
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char kbuf[1024];
  int v = 0;
  bool found = false;
  while (std::fscanf(f, "%1023s %d", kbuf, &v) == 2) {
    g_tune_cache[kbuf] = v;
    if (key == kbuf) {
      *best = v;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const std::string& key, const char* path, int best) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), best);
  std::fclose(f);
}

}  // namespace

lp_status lp_tune_schedule(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* val, const char* cache_path, int32_t* lane_target_out,
                           int32_t* tile_rows_out, double* ms_out) {
  pdhg_set_last_error(std::string());
  if (!lane_target_out || !tile_rows_out || !row_ptr || (nnz > 0 && (!col_idx || !val)))
    return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (m < 0 || n < 0 || nnz < 0) return fail(LP_ERR_INVALID_ARG, "negative size");
  if (nnz >= INT32_MAX) return fail(LP_ERR_TOO_LARGE, "nnz must be below 2^31");
  // a box LP on the given matrix: every clamp of the iteration is exercised
  std::vector<double> zc(n, 0.0), lo_n(n, -1.0), hi_n(n, 1.0), lo_m(m, -1.0), hi_m(m, 1.0);
  for (int32_t j = 0; j < n; ++j) zc[j] = (j % 3 == 0) ? 1.0 : -0.5;
  lp_status st = validate(m, n, nnz, row_ptr, col_idx, val, zc.data(), lo_m.data(), hi_m.data(), lo_n.data(),
                          hi_n.data());
  if (st != LP_OK) return st;
  const std::string key = shape_class(m, n, nnz, row_ptr, col_idx);
  int cached = 0;
  if (!ms_out && cache_lookup(key, cache_path, &cached)) {
    *lane_target_out = cached / 100;
    *tile_rows_out = cached % 100;
    return LP_OK;
  }
  // copies of the instance, enough to fill the device (about 4M nonzeros), on the grid loop
  const int32_t rep = (int32_t)std::max<int64_t>(1, std::min<int64_t>(256, (int64_t(1) << 22) / std::max<int64_t>(nnz, 1)));
  std::vector<int32_t> vm(rep, m), vn(rep, n);
  std::vector<int64_t> vz(rep, nnz);
  std::vector<const int64_t*> vrp(rep, row_ptr);
  std::vector<const int32_t*> vci(rep, col_idx);
  std::vector<const double*> vval(rep, val), vc(rep, zc.data()), vlc(rep, lo_m.data()), vuc(rep, hi_m.data()),
      vlv(rep, lo_n.data()), vuv(rep, hi_n.data());
  lp_params prm;
  lp_default_params(&prm);
  prm.batch_local_nnz = 0;
  double best_ms = INFINITY;
  int best = 0;
  std::vector<int32_t> tiles(2 * (size_t)rep);
  for (int q = 0; q < kTuneN; ++q) {
    for (int32_t k = 0; k < rep; ++k) {
      tiles[2 * k] = kTuneLane[q];
      tiles[2 * k + 1] = kTuneRows[q];
    }
    lp_batch_handle h = nullptr;
    st = lp_batch_create(rep, vm.data(), vn.data(), vz.data(), vrp.data(), vci.data(), vval.data(), vc.data(),
                         vlc.data(), vuc.data(), vlv.data(), vuv.data(), nullptr, tiles.data(), &prm, &h);
    if (st != LP_OK) return st;
    double out[2] = {0.0, 0.0};
    st = lp_batch_time_loop(h, 32, 1, nullptr, out);
    lp_batch_destroy(h);
    if (st != LP_OK) return st;
    const double per_iter = out[0] / out[1];
    if (ms_out) ms_out[q] = per_iter;
    if (per_iter < best_ms) {
      best_ms = per_iter;
      best = q;
    }
  }
  cache_store(key, cache_path, 100 * kTuneLane[best] + kTuneRows[best]);
  *lane_target_out = kTuneLane[best];
  *tile_rows_out = kTuneRows[best];
  return LP_OK;
}

extern "C" {

lp_status lp_batch_create(int32_t count, const int32_t* m, const int32_t* n, const int64_t* nnz,
                          const int64_t* const* row_ptr, const int32_t* const* col_idx,
                          const double* const* val, const double* const* c, const double* const* l_c,
                          const double* const* u_c, const double* const* l_v,
                          const double* const* u_v, const double* eta, const int32_t* tiles,
                          const lp_params* p, lp_batch_handle* out) {
  pdhg_set_last_error(std::string());
  if (!out) return fail(LP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || count > kMaxInst)
    return fail(LP_ERR_INVALID_ARG, "count must be in [1, " + std::to_string(kMaxInst) + "]");
  if (!m || !n || !nnz || !row_ptr || !col_idx || !val || !c || !l_c || !u_c || !l_v || !u_v)
    return fail(LP_ERR_INVALID_ARG, "NULL argument");
  lp_params prm;
  if (p) prm = *p;
  else lp_default_params(&prm);
  lp_status st = check_params(prm);
  if (st != LP_OK) return st;
  if (eta)
    for (int32_t k = 0; k < count; ++k)
      if (!(eta[k] > 0.0) || !std::isfinite(eta[k]))
        return fail(LP_ERR_INVALID_ARG, "eta[" + std::to_string(k) + "] must be finite and > 0");
  if (tiles)
    for (int32_t k = 0; k < count; ++k)
      if (tiles[2 * k] < 1 || tiles[2 * k] > 64 || tiles[2 * k + 1] < 1 || tiles[2 * k + 1] > 32)
        return fail(LP_ERR_INVALID_ARG, "tiles[" + std::to_string(k) + "] must be (lane_target in [1, 64], tile_rows in [1, 32])");
  lp_batch* h = new lp_batch();
  h->count = count;
  h->prm = prm;
  st = batch_create_impl(h, m, n, nnz, row_ptr, col_idx, val, c, l_c, u_c, l_v, u_v, eta, tiles);
  if (st != LP_OK) {
    const std::string keep = lp_last_error();
    delete h;
    pdhg_set_last_error(keep);
    return st;
  }
  *out = h;
  return LP_OK;
}

lp_status lp_batch_solve(lp_batch_handle hh, double tol, int64_t max_iter, void* stream) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol >= 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be >= 0");
  if (max_iter < 1) return fail(LP_ERR_INVALID_ARG, "max_iter must be >= 1");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lp_status st;
  if (h->prm.precision == 0) {
    st = enqueue_batch_start<double>(h, tol, max_iter, 0, s);
    if (st != LP_OK) return st;
    st = enqueue_stage<double>(h, h->exec64, max_iter, s);
    if (st != LP_OK) return st;
  } else {
    const double tol32 = h->prm.precision == 1 ? std::max(tol, h->prm.switch_tol) : tol;
    st = enqueue_batch_start<float>(h, tol32, max_iter, h->prm.fp32_patience, s);
    if (st != LP_OK) return st;
    st = enqueue_stage<float>(h, h->exec32, max_iter, s);
    if (st != LP_OK) return st;
    BatchArgs<float> f;
    BatchArgs<double> d;
    fill_batch_args<float>(h, f);
    fill_batch_args<double>(h, d);
    if (h->prm.precision == 1) {
      CK(cudaMemsetAsync(&h->bc->n_done, 0, sizeof(unsigned), s));
      kb_switch<<<h->gridS, kThreads, 0, s>>>(f, d, tol, max_iter, 0);
      const int gA = grid_for(h->ntA, kWarps, 8 * h->num_sms), gT = grid_for(h->ntT, kWarps, 8 * h->num_sms);
      kb_spmv<double><<<gA, kThreads, 0, s>>>(h->tasksA, h->ntA, h->rpA, h->ciA, h->valA, h->x, h->axh);
      kb_spmv<double><<<gT, kThreads, 0, s>>>(h->tasksT, h->ntT, h->rpT, h->ciT, h->valT, h->yh, h->aty);
      kb_warm<<<h->gridS, kThreads, 0, s>>>(d, bodies_for(max_iter));
      CK(cudaGetLastError());
      st = enqueue_stage<double>(h, h->exec64, max_iter, s);
      if (st != LP_OK) return st;
    } else {
      kb_switch<<<h->gridS, kThreads, 0, s>>>(f, d, tol, max_iter, 1);
      CK(cudaGetLastError());
    }
  }
  h->solved = true;
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_batch_get_all(lp_batch_handle hh, int32_t* status, double* kkt4, int64_t* iters,
                           int64_t* iters_fp32, double* eta) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "no solve has been enqueued");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  std::vector<Ctl> ctl(h->count);
  BatchCtl bc{};
  CK(cudaMemcpy(ctl.data(), h->ctl, sizeof(Ctl) * h->count, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&bc, h->bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
  for (int32_t k = 0; k < h->count; ++k) {
    const Ctl& c = ctl[k];
    if (status) status[k] = c.done ? c.status : LP_SOLVE_INTERNAL_ERROR;
    if (kkt4)
      for (int q = 0; q < 4; ++q) kkt4[4 * k + q] = c.kkt[q];
    if (iters) iters[k] = c.iters;
    if (iters_fp32) iters_fp32[k] = h->prm.precision == 1 ? c.iters32 : (h->prm.precision == 2 ? c.iters : 0);
    if (eta) eta[k] = h->eta[k];
  }
  return LP_OK;
}

lp_status lp_batch_schedule(lp_batch_handle hh, int32_t* where) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!where) return fail(LP_ERR_INVALID_ARG, "NULL output");
  for (int32_t k = 0; k < h->count; ++k) where[k] = h->inst[k].local ? (h->sm_ctas > 0 ? 3 : 1) : 0;
  if (h->sm_ctas == 0)
    for (int32_t q = h->n_wide; q < h->n_local; ++q) where[h->local_host[q]] = 2;
  return LP_OK;
}

lp_status lp_batch_get(lp_batch_handle hh, int32_t k, double* x, double* y, int32_t* status, double* kkt4,
                       int64_t* iters) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (k < 0 || k >= h->count) return fail(LP_ERR_INVALID_ARG, "instance index out of range");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "no solve has been enqueued");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  Ctl c;
  CK(cudaMemcpy(&c, h->ctl + k, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const BInst& I = h->inst[k];
  cudaStream_t s = h->setup_stream;
  const int g = grid_for(std::max(I.m, I.n), 256, 4 * h->num_sms);
  if (x && I.n > 0) {
    const double* xh = (c.t & 1) ? h->xh1 : h->xh0;
    k_unpermute_scale<<<g, 256, 0, s>>>(I.n, h->col_perm + I.col0, xh + I.col0, h->dc + I.col0, h->out_buf);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(x, h->out_buf, sizeof(double) * I.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (y && I.m > 0) {
    k_unpermute_scale<<<g, 256, 0, s>>>(I.m, h->row_perm + I.row0, h->yh + I.row0, h->dr + I.row0, h->out_buf);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(y, h->out_buf, sizeof(double) * I.m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (status) status[0] = c.done ? c.status : LP_SOLVE_INTERNAL_ERROR;
  if (kkt4)
    for (int q = 0; q < 4; ++q) kkt4[q] = c.kkt[q];
  if (iters) *iters = c.iters;
  return LP_OK;
}

lp_status lp_batch_time_loop(lp_batch_handle hh, int64_t iters, int32_t precision64, void* stream,
                             double* ms_out) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h || !ms_out) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (!precision64 && h->prm.precision == 0) return fail(LP_ERR_INVALID_ARG, "no FP32 data (precision 0)");
  if (iters < 1) return fail(LP_ERR_INVALID_ARG, "iters must be >= 1");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t launches = (iters + kBatchUnroll - 1) / kBatchUnroll;
  const int64_t total = launches * kBatchUnroll;
  lp_status st = precision64 ? enqueue_batch_start<double>(h, 0.0, total, 0, s)
                             : enqueue_batch_start<float>(h, 0.0, total, 0, s);
  if (st != LP_OK) return st;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  for (int64_t q = 0; q < launches; ++q) {
    if (precision64) {
      BatchArgs<double> a;
      fill_batch_args<double>(h, a);
      CK(launch_batch_loop<double>(h, a, kBatchUnroll, cudaGraphConditionalHandle{}, 0, s));
    } else {
      BatchArgs<float> a;
      fill_batch_args<float>(h, a);
      CK(launch_batch_loop<float>(h, a, kBatchUnroll, cudaGraphConditionalHandle{}, 0, s));
    }
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ms_out[0] = (double)ms / (double)launches;
  ms_out[1] = (double)kBatchUnroll;
  h->solved = true;
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_batch_get_trace(lp_batch_handle hh, int32_t k, double* out, int64_t cap, int64_t* rows) {
  pdhg_set_last_error(std::string());
  lp_batch* h = checked(hh);
  if (!h || !rows || (cap > 0 && !out)) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  if (k < 0 || k >= h->count) return fail(LP_ERR_INVALID_ARG, "instance index out of range");
  if (!h->trace) return fail(LP_ERR_NOT_SOLVED, "no traced run (lp_batch_unroll) yet");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  Ctl c;
  CK(cudaMemcpy(&c, h->ctl + k, sizeof(Ctl), cudaMemcpyDeviceToHost));
  int64_t r = std::min<int64_t>(c.iters, h->trace_cap);
  if (r > cap) r = cap;
  if (r < 0) r = 0;
  if (r > 0)
    CK(cudaMemcpy(out, h->trace + (size_t)k * (size_t)h->trace_cap * 4, sizeof(double) * 4 * (size_t)r,
                  cudaMemcpyDeviceToHost));
  *rows = r;
  return LP_OK;
}

void lp_batch_destroy(lp_batch_handle h) { delete h; }

}  // extern "C"
