// The iteration loop of restarted reflected-Halpern PDHG (cuPDLPx, arXiv 2507.14051; reflected
// form, gamma = 1) for LPs small enough to live in the shared memory of one thread-block cluster:
// sm_run, which the single-LP kernel k_loop_sm (smem_loop.cu) and the batch's small-instance
// kernel (batch.cu) run.
//
// Each iteration is the one of iterate.cu's loop kernel: the same row and column epilogues
// (step.cuh), the same scalar control (restart test and PID update of Section 3, relative KKT
// test of Section 4) in the same order.  What changes is where the data sits during a launch:
//   * CTA q of the cluster owns a contiguous slice of the rows and one of the columns (host
//     split, balanced by nonzeros), with its rows of A and of A^T (local CSR) and its slices of
//     the row and column vectors, all in its shared memory;
//   * every CTA holds a replica of the vectors the SpMVs gather: xbar and xhat (xhat_t in buffer
//     t & 1, as in global memory) for the row phase, qy and yhat for the column phase.  After a
//     phase the owner of a row or column writes its new entries into every other CTA's replica
//     (distributed shared memory);
//   * each reduction sums the block (warp butterflies, then the warps in order), writes the
//     block's sums into every CTA's table of partials (row = the writer's rank; two tables used
//     alternately), passes one cluster barrier, then adds the table's rows in rank order by a
//     fixed butterfly, so every CTA runs the same control on the same bits.
// So a phase costs its shared-memory SpMV and epilogue, one cluster barrier and the control; the
// only global traffic inside the loop is the trace and the stall guard's slots.  A launch loads
// the CTA's data from global memory, runs up to `iters` iterations and writes the CTA's rows and
// columns of the state back.
//
// The SpMV gives each row (and column) up to 8 lanes, each adding its strided entries in order,
// then a fixed butterfly (sm_rows): deterministic, though not the binned kernels' order.
#pragma once
#include <cooperative_groups.h>

#include "step.cuh"

namespace cg = cooperative_groups;

namespace pdhg {

namespace {

template <class T>
__device__ __forceinline__ T* sm_at(unsigned char* base, uint32_t off) {
  return reinterpret_cast<T*>(base + off);
}

// A pointer p - off (as an address) for arrays indexed by global row or column index whose
// shared-memory copy starts at the slice's first index: only p[off .. off + len) is accessed.
template <class T>
__device__ __forceinline__ T* sm_rebase(T* p, int off) {
  return reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) - (uintptr_t)off * sizeof(T));
}

// Lanes per row of the shared-memory SpMV for a slice of cnt rows: 8, halved until the rows
// fit in the first kThreads - 32 threads (the last warp then stays free for the control's
// precomputation), down to 1.
__device__ __forceinline__ int sm_lanes(int cnt) {
  int g = 8;
  while (g > 1 && cnt * g > kThreads - 32) g >>= 1;
  return g;
}

// Rows [0, cnt) of a shared-memory CSR slice (local offsets rp) times xg, G lanes per row: lane
// sub of row li adds entries sub, sub + G, ... in order, then a fixed xor butterfly over the G
// lanes; f(li, value) runs in the row's first lane (thread li * G of a pass).  FP64 operations
// have a ~64-cycle dependent latency on this GPU, so spreading a row over lanes shortens its
// chain.  The whole block must call it (every warp runs every pass's shuffles).
template <class V, class F>
__device__ __forceinline__ void sm_rows(const int32_t* rp, const int32_t* ci, const V* val, const V* xg, int cnt,
                                        int G, F&& f) {
  const int total = cnt * G;
  for (int base = 0; base < total; base += kThreads) {
    const int slot = base + (int)threadIdx.x;
    const int li = slot / G, sub = slot - li * G;
    V acc = V(0);
    if (li < cnt) {
      const int e = rp[li + 1];
      for (int k = rp[li] + sub; k < e; k += G) acc = fmav(val[k], xg[ci[k]], acc);
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (li < cnt && sub == 0) f(li, acc);
  }
}

// One pass of sm_rows without the epilogue (cnt * G <= the calling warps' threads; the calling
// warps are whole and the first ones of the block): the value of row li = threadIdx.x / G, in
// the same order as sm_rows, ends in every lane of the row's group.
template <class V>
__device__ __forceinline__ V sm_dot(const int32_t* rp, const int32_t* ci, const V* val, const V* xg, int cnt, int G) {
  const int li = (int)threadIdx.x / G, sub = (int)threadIdx.x - li * G;
  V acc = V(0);
  if (li < cnt) {
    const int e = rp[li + 1];
    for (int k = rp[li] + sub; k < e; k += G) acc = fmav(val[k], xg[ci[k]], acc);
  }
  for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
  return acc;
}

template <class T>
__device__ __forceinline__ void copy_in(T* dst, const T* __restrict__ src, int len) {
  for (int k = threadIdx.x; k < len; k += kThreads) dst[k] = src[k];
}
template <class T>
__device__ __forceinline__ void copy_out(T* __restrict__ dst, const T* src, int len) {
  for (int k = threadIdx.x; k < len; k += kThreads) dst[k] = src[k];
}

// Writes entries [b, b + len) of the replicas a and b2 (same offsets in every CTA) into every
// other CTA of the cluster.  The caller has synchronised the block after writing them.
template <class V>
__device__ __forceinline__ void publish(cg::cluster_group& cl, V* a, V* b2, int b, int len, int me, int nctas) {
  const int work = len * (nctas - 1);
  for (int k = threadIdx.x; k < work; k += kThreads) {
    const int q0 = k / len, i = b + (k - q0 * len);
    const int q = q0 < me ? q0 : q0 + 1;
    V* ra = cl.map_shared_rank(a, (unsigned)q);
    V* rb = cl.map_shared_rank(b2, (unsigned)q);
    ra[i] = a[i];
    rb[i] = b2[i];
  }
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// Block barrier of warps 0 .. kWarps - 2 (named barrier 1; the last warp does not take part).
__device__ __forceinline__ void sync_but_last() { asm volatile("bar.sync 1, %0;" ::"r"(kThreads - 32) : "memory"); }

// Cluster-wide sums of v[0..NS), where only the first lane of each group of G lanes of the first
// `warps` warps holds nonzero values: a butterfly over those lanes per warp (xor offsets
// 16 .. G), the warps' sums added in warp order, the block's sums written into row `me` of every
// CTA's table `tab` (kSmMaxCtas x kNumSums doubles, the same offset in every CTA), one cluster
// barrier (which also publishes every store made before it), then warp 0 adds the table's rows
// 0..nctas-1 by a fixed butterfly.  The totals end in thread 0's v[]; every CTA gets the same
// bits.  The NS sums go through each step side by side (FP64 additions have a ~64-cycle
// dependent latency here; independent ones overlap).
// side(): work for thread kThreads - 32 that the caller reads after its next block barrier.
// With `detach` (the last warp holds no sums) that thread runs it between its arrival at the
// cluster barrier and its wait, off everyone's path; otherwise before the sums.  The whole
// cluster must call it, each CTA with its own table buffer in the same alternation.
// kLast: the last warp adds the table instead of warp 0 and the totals end in thread
// kThreads - 32's v[]; the other warps return right after the cluster barrier (free to work
// while the last warp adds and runs the control).
template <int NS, bool kLast = false, class Side>
__device__ __forceinline__ void cluster_sums(cg::cluster_group& cl, double (&v)[kNumSums], int G, int warps,
                                             bool detach, double* tab, int me, int nctas, Side&& side) {
  __shared__ double wsum[kWarps][kNumSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool last = warp == kWarps - 1;
  if (!detach && last && lane == 0) side();
  if (!(detach && last)) {
    if (warp < warps) {
      double t[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) t[q] = v[q];
      for (int off = 16; off >= G; off >>= 1) {
#pragma unroll
        for (int q = 0; q < NS; ++q) t[q] += __shfl_xor_sync(kFull, t[q], off);
      }
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) wsum[warp][q] = t[q];
      }
    }
    if (detach) sync_but_last();
    else __syncthreads();
    if (threadIdx.x < nctas) {
      double t[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) t[q] = warps > 0 ? wsum[0][q] : 0.0;
      for (int w = 1; w < warps; ++w) {
#pragma unroll
        for (int q = 0; q < NS; ++q) t[q] += wsum[w][q];
      }
      double* dst = cl.map_shared_rank(tab, threadIdx.x) + me * kNumSums;
#pragma unroll
      for (int q = 0; q < NS; ++q) dst[q] = t[q];
    }
  }
  cluster_arrive();
  if (detach && last && lane == 0) side();
  cluster_wait();
  if (kLast ? last : threadIdx.x < 32) {
    int width = 1;
    while (width < nctas) width <<= 1;
    double t[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) t[q] = lane < nctas ? tab[lane * kNumSums + q] : 0.0;
    for (int off = width >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < NS; ++q) t[q] += __shfl_xor_sync(kFull, t[q], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NS; ++q) v[q] = t[q];
    }
  }
}

}  // namespace

// Runs one LP on the calling cluster: its rows [0, ra.m) and columns [0, ca.n) (ra / ca point at
// its arrays; A's column indices are col_base + j and A^T's row indices row_base + i, so that
// one LP of a concatenated batch can be run), split over the cluster's CTAs by sp, with
// smem_bytes of dynamic shared memory at smem.  Loads the LP, runs up to `iters` iterations from
// the scalar state in sc (the caller's shared copy, loaded and synchronised before), writes the
// LP's rows and columns of the state back and leaves the final scalar state in sc; the trace
// (if any) is written by rank 0.  Returns false, having done nothing, if the split does not fit
// smem_bytes (the same answer in every CTA).  The whole cluster must call it.
template <class V>
__device__ __forceinline__ bool sm_run(cg::cluster_group& cl, unsigned char* smem, int32_t smem_bytes, Ctl& sc,
                                       const RowArgsT<V>& ra, const ColArgsT<V>& ca, const SmSplit& sp,
                                       int row_base, int col_base, int32_t iters, double* trace) {
  __shared__ RowStepR<V> rstr;
  __shared__ ColStepR<V> cstr;
  __shared__ Halpern hw;
  __shared__ int rs, chk_cur, chk_nxt;
  __shared__ RestartPre rpre;
  const int tid = threadIdx.x;
  const int me = (int)cl.block_rank(), nctas = (int)cl.num_blocks();
  const int m = ra.m, n = ca.n;
  // the same check in every CTA (so either all CTAs run or none does)
  bool ok = nctas <= kSmMaxCtas && sp.rs[0] == 0 && sp.cs[0] == 0 && sp.rs[nctas] == m && sp.cs[nctas] == n;
  for (int q = 0; ok && q < nctas; ++q) {
    const int a0 = sp.rs[q], a1 = sp.rs[q + 1], b0 = sp.cs[q], b1 = sp.cs[q + 1];
    ok = a0 <= a1 && b0 <= b1 &&
         sm_layout(m, n, a1 - a0, b1 - b0, ra.rp[a1] - ra.rp[a0], ca.rp[b1] - ca.rp[b0], (int)sizeof(V)).total <=
             (uint64_t)smem_bytes;
  }
  if (!ok) return false;
  const int r0 = sp.rs[me], mr = sp.rs[me + 1] - r0, c0 = sp.cs[me], nc = sp.cs[me + 1] - c0;
  const int zr0 = ra.rp[r0], nzr = ra.rp[r0 + mr] - zr0;
  const int zc0 = ca.rp[c0], nzc = ca.rp[c0 + nc] - zc0;
  const SmLayout L = sm_layout(m, n, mr, nc, nzr, nzc, (int)sizeof(V));
  double* part = sm_at<double>(smem, L.part);
  V* xbar_r = sm_at<V>(smem, L.xbar);
  V* xh_r0 = sm_at<V>(smem, L.xh0);
  V* xh_r1 = sm_at<V>(smem, L.xh1);
  V* qy_r = sm_at<V>(smem, L.qy);
  V* yh_r = sm_at<V>(smem, L.yh);
  int32_t* rp_s = sm_at<int32_t>(smem, L.rp);
  int32_t* ci_s = sm_at<int32_t>(smem, L.ci);
  V* val_s = sm_at<V>(smem, L.val);
  int32_t* rpT_s = sm_at<int32_t>(smem, L.rpT);
  int32_t* ciT_s = sm_at<int32_t>(smem, L.ciT);
  V* valT_s = sm_at<V>(smem, L.valT);
  V *y0_s = sm_at<V>(smem, L.y0), *w_s = sm_at<V>(smem, L.w), *ax0_s = sm_at<V>(smem, L.ax0);
  V *axh_s = sm_at<V>(smem, L.axh), *ax_s = sm_at<V>(smem, L.ax);
  V *lc_s = sm_at<V>(smem, L.lc), *uc_s = sm_at<V>(smem, L.uc), *idr_s = sm_at<V>(smem, L.inv_dr);
  V *x0_s = sm_at<V>(smem, L.x0), *aty0_s = sm_at<V>(smem, L.aty0), *aty_s = sm_at<V>(smem, L.aty);
  V *c_s = sm_at<V>(smem, L.c), *lv_s = sm_at<V>(smem, L.lv), *uv_s = sm_at<V>(smem, L.uv);
  V* idc_s = sm_at<V>(smem, L.inv_dc);

  // ---- load: replicas, this CTA's matrix slices (local offsets) and vector slices
  copy_in(xbar_r, ca.xbar, n);
  copy_in(xh_r0, (const V*)ca.xh0, n);
  copy_in(xh_r1, (const V*)ca.xh1, n);
  copy_in(qy_r, (const V*)ra.qy, m);
  copy_in(yh_r, (const V*)ra.yh, m);
  for (int k = tid; k <= mr; k += kThreads) rp_s[k] = ra.rp[r0 + k] - zr0;
  for (int k = tid; k < nzr; k += kThreads) ci_s[k] = ra.ci[zr0 + k] - col_base;
  copy_in(val_s, ra.val + zr0, nzr);
  for (int k = tid; k <= nc; k += kThreads) rpT_s[k] = ca.rp[c0 + k] - zc0;
  for (int k = tid; k < nzc; k += kThreads) ciT_s[k] = ca.ci[zc0 + k] - row_base;
  copy_in(valT_s, ca.val + zc0, nzc);
  copy_in(y0_s, (const V*)ra.y0 + r0, mr);
  copy_in(w_s, (const V*)ra.w + r0, mr);
  copy_in(ax0_s, (const V*)ra.ax0 + r0, mr);
  copy_in(axh_s, (const V*)ra.axh + r0, mr);
  copy_in(ax_s, (const V*)ra.ax + r0, mr);
  copy_in(lc_s, ra.lc + r0, mr);
  copy_in(uc_s, ra.uc + r0, mr);
  copy_in(idr_s, ra.inv_dr + r0, mr);
  copy_in(x0_s, (const V*)ca.x0 + c0, nc);
  copy_in(aty0_s, (const V*)ca.aty0 + c0, nc);
  copy_in(aty_s, (const V*)ca.aty + c0, nc);
  copy_in(c_s, ca.c + c0, nc);
  copy_in(lv_s, ca.lv + c0, nc);
  copy_in(uv_s, ca.uv + c0, nc);
  copy_in(idc_s, ca.inv_dc + c0, nc);
  // thread 0 prepares each phase's step scalars at the end of the control before it (so a phase
  // starts without a serial step and a block barrier)
  if (tid == 0) {
    chk_cur = is_check(sc, sc.t) ? 1 : 0;
    rstr = row_step_r<V>(sc, chk_cur);
  }
  // the epilogues' argument blocks over shared memory (the LP's row / column indices)
  RowArgsT<V> rl = ra;
  rl.xh0 = xh_r0;
  rl.xh1 = xh_r1;
  rl.qy = qy_r;
  rl.yh = yh_r;
  rl.xbar = xbar_r;
  rl.y0 = sm_rebase(y0_s, r0);
  rl.w = sm_rebase(w_s, r0);
  rl.ax0 = sm_rebase(ax0_s, r0);
  rl.axh = sm_rebase(axh_s, r0);
  rl.ax = sm_rebase(ax_s, r0);
  rl.lc = sm_rebase(lc_s, r0);
  rl.uc = sm_rebase(uc_s, r0);
  rl.inv_dr = sm_rebase(idr_s, r0);
  ColArgsT<V> cl_ = ca;
  cl_.yh = yh_r;
  cl_.qy = qy_r;
  cl_.xbar = xbar_r;
  cl_.xh0 = xh_r0;
  cl_.xh1 = xh_r1;
  cl_.x0 = sm_rebase(x0_s, c0);
  cl_.aty0 = sm_rebase(aty0_s, c0);
  cl_.aty = sm_rebase(aty_s, c0);
  cl_.c = sm_rebase(c_s, c0);
  cl_.lv = sm_rebase(lv_s, c0);
  cl_.uv = sm_rebase(uv_s, c0);
  cl_.inv_dc = sm_rebase(idc_s, c0);
  // every CTA has loaded its replicas before any CTA writes into them
  cl.sync();
  if (me != 0) trace = nullptr;
  // lanes per row and warps holding sums, per side
  const int Gr = sm_lanes(mr), Gc = sm_lanes(nc);
  const int wr = min(kWarps, (mr * Gr + 31) / 32), wc = min(kWarps, (nc * Gc + 31) / 32);
  // the last warp holds no sums of either phase: it runs the control's precomputation while the
  // cluster barrier completes
  const bool detach = wr < kWarps && wc < kWarps;
  int red = 0;  // reductions so far: table buffer red & 1
  auto sums = [&](double (&v)[kNumSums], int nsums, int G, int warps, bool det, auto&& side) {
    double* tab = part + (red & 1) * (kSmMaxCtas * kNumSums);
    if (nsums == 1) cluster_sums<1>(cl, v, G, warps, det, tab, me, nctas, side);
    else if (nsums == 2) cluster_sums<2>(cl, v, G, warps, det, tab, me, nctas, side);
    else cluster_sums<kNumSums>(cl, v, G, warps, det, tab, me, nctas, side);
    ++red;
  };
  auto nothing = []() {};
  // the same reductions with the table added by the last warp (totals in thread ctl's v[])
  auto sums_last = [&](double (&v)[kNumSums], int nsums, int G, int warps, auto&& side) {
    double* tab = part + (red & 1) * (kSmMaxCtas * kNumSums);
    if (nsums == 1) cluster_sums<1, true>(cl, v, G, warps, true, tab, me, nctas, side);
    else if (nsums == 2) cluster_sums<2, true>(cl, v, G, warps, true, tab, me, nctas, side);
    else cluster_sums<kNumSums, true>(cl, v, G, warps, true, tab, me, nctas, side);
    ++red;
  };
  if (detach) {
    // Overlapped form (every row and column slice fits one SpMV pass in the first kWarps - 1
    // warps): after each phase's cluster barrier, the last warp adds the table and its first
    // thread runs the control while the other warps already take the next phase's dot
    // products (they read only replicas the barrier published; a column phase that turns out
    // to restart recomputes its dot products from yhat).  Same operations, same order, same
    // bits as the loop below.
    const int ctl = kThreads - 32;
    const bool work = tid < ctl;
    const int lr = tid / Gr, lc = tid / Gc;
    const bool row_first = work && lr < mr && tid - lr * Gr == 0;
    const bool col_first = work && lc < nc && tid - lc * Gc == 0;
    V rv = V(0), rax = V(0);
    if (work) {
      rv = sm_dot(rp_s, ci_s, val_s, (const V*)xbar_r, mr, Gr);
      if (rstr.check) rax = sm_dot(rp_s, ci_s, val_s, (const V*)((sc.t & 1) ? xh_r1 : xh_r0), mr, Gr);
    }
    for (int32_t it = 0; it < iters && !sc.done; ++it) {
      // ---- row phase: epilogues from the dot products taken during the last control
      double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      const RowStepR<V> st = rstr;
      const int check = st.check;
      if (row_first) {
        if (check) ax_s[lr] = rax;
        row_epilogue_r(rl, st, r0 + lr, rv, s);
      }
      __syncthreads();
      publish(cl, qy_r, yh_r, r0, mr, me, nctas);
      // during the barrier: the Halpern weights, the restart test's thresholds and whether
      // t + 1 is a check iteration
      sums_last(s, check ? 5 : 2, Gr, wr, [&]() {
        hw = halpern_weights(sc.k, sc.gamma);
        rpre = restart_pre(sc);
        chk_nxt = is_check(sc, sc.t + 1) ? 1 : 0;
      });
      const int ccheck = chk_cur;
      V cv = V(0), caty = V(0);
      if (work) {  // the column phase's dot products, assuming no restart
        cv = sm_dot(rpT_s, ciT_s, valT_s, (const V*)qy_r, nc, Gc);
        if (ccheck) caty = sm_dot(rpT_s, ciT_s, valT_s, (const V*)yh_r, nc, Gc);
      } else if (tid == ctl) {
        rs = row_decide(sc, s, check, trace, &hw, 1.0, &rpre);
        if (rs != 1) cstr = col_step_r(sc, cl_, chk_cur);
      }
      __syncthreads();
      if (rs == 1) {  // the same decision in every CTA
        const V* xc = (sc.t & 1) ? xh_r1 : xh_r0;  // xhat of this iteration
        double q[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (sc.pid_enabled) {
          for (int lj = tid; lj < nc; lj += kThreads) {
            const V d = xc[c0 + lj] - x0_s[lj];
            acc_fma(q[0], d, d);
          }
          for (int li = tid; li < mr; li += kThreads) {
            const V d = yh_r[r0 + li] - y0_s[li];
            acc_fma(q[1], d, d);
          }
          sums(q, 2, 1, kWarps, false, nothing);
        }
        if (tid == 0) {
          row_restart_weight(sc, q[0], q[1]);
          cstr = col_step_r(sc, cl_, chk_cur);  // with the new primal weight's tau
        }
        // A xhat_t: the next row phase takes it as A x and as the new anchor's product
        sm_rows(rp_s, ci_s, val_s, xc, mr, Gr, [&](int li, V v) { axh_s[li] = v; });
        if (work) cv = sm_dot(rpT_s, ciT_s, valT_s, (const V*)yh_r, nc, Gc);  // a restart gathers yhat
        __syncthreads();
      }
      if (sc.done) break;
      // ---- column phase
      double s2[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      const ColStepR<V> cs = cstr;
      if (col_first) {
        if (cs.check && !cs.restart) aty_s[lc] = caty;
        col_epilogue_r(cl_, cs, c0 + lc, cv, s2);
      }
      __syncthreads();
      publish(cl, xbar_r, cs.xn, c0, nc, me, nctas);
      sums_last(s2, cs.check ? 5 : 1, Gc, wc, nothing);
      if (work) {  // the next row phase's dot products
        rv = sm_dot(rp_s, ci_s, val_s, (const V*)xbar_r, mr, Gr);
        if (chk_nxt) rax = sm_dot(rp_s, ci_s, val_s, (const V*)cs.xn, mr, Gr);
      } else if (tid == ctl) {
        col_control(sc, s2, cs.check);
        chk_cur = chk_nxt;
        rstr = row_step_r<V>(sc, chk_cur);
      }
      __syncthreads();
    }
  }
  for (int32_t it = 0; !detach && it < iters && !sc.done; ++it) {
    // ---- row phase (rows r0 .. r0 + mr)
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const RowStepR<V> st = rstr;
    const int check = st.check;
    if (check) {  // A xhat_t for the primal residual of the KKT test (read by the same lane)
      const V* xc = (sc.t & 1) ? xh_r1 : xh_r0;
      sm_rows(rp_s, ci_s, val_s, xc, mr, Gr, [&](int li, V v) { ax_s[li] = v; });
    }
    sm_rows(rp_s, ci_s, val_s, (const V*)xbar_r, mr, Gr,
            [&](int li, V wv) { row_epilogue_r(rl, st, r0 + li, wv, s); });
    __syncthreads();
    publish(cl, qy_r, yh_r, r0, mr, me, nctas);
    // the last warp computes, during the barrier, the Halpern weights that row_decide takes
    // (two FP64 divisions) and the restart test's thresholds
    sums(s, check ? 5 : 2, Gr, wr, detach, [&]() {
      hw = halpern_weights(sc.k, sc.gamma);
      rpre = restart_pre(sc);
    });
    __syncthreads();
    if (tid == 0) {
      rs = row_decide(sc, s, check, trace, &hw, 1.0, &rpre);
      if (rs != 1) cstr = col_step_r(sc, cl_, chk_cur);
    }
    __syncthreads();
    if (rs == 1) {  // the same decision in every CTA
      const V* xc = (sc.t & 1) ? xh_r1 : xh_r0;  // xhat of this iteration
      double q[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (sc.pid_enabled) {
        for (int lj = tid; lj < nc; lj += kThreads) {
          const V d = xc[c0 + lj] - x0_s[lj];
          acc_fma(q[0], d, d);
        }
        for (int li = tid; li < mr; li += kThreads) {
          const V d = yh_r[r0 + li] - y0_s[li];
          acc_fma(q[1], d, d);
        }
        sums(q, 2, 1, kWarps, false, nothing);
      }
      if (tid == 0) {
        row_restart_weight(sc, q[0], q[1]);
        cstr = col_step_r(sc, cl_, chk_cur);  // with the new primal weight's tau
      }
      // A xhat_t: the next row phase takes it as A x and as the new anchor's product
      sm_rows(rp_s, ci_s, val_s, xc, mr, Gr, [&](int li, V v) { axh_s[li] = v; });
      __syncthreads();
    }
    if (sc.done) break;
    // ---- column phase (columns c0 .. c0 + nc)
    double s2[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const ColStepR<V> cs = cstr;
    const int ccheck = cs.check;
    if (ccheck && !cs.restart)  // A^T yhat_t for the dual residual of the KKT test
      sm_rows(rpT_s, ciT_s, valT_s, (const V*)yh_r, nc, Gc, [&](int lj, V u) { aty_s[lj] = u; });
    const V* gy = cs.restart ? yh_r : qy_r;
    sm_rows(rpT_s, ciT_s, valT_s, gy, nc, Gc, [&](int lj, V u) { col_epilogue_r(cl_, cs, c0 + lj, u, s2); });
    __syncthreads();
    publish(cl, xbar_r, cs.xn, c0, nc, me, nctas);
    // ... and whether t + 1 is a check iteration (a 64-bit remainder)
    sums(s2, ccheck ? 5 : 1, Gc, wc, detach, [&]() { chk_nxt = is_check(sc, sc.t + 1) ? 1 : 0; });
    __syncthreads();
    if (tid == 0) {
      col_control(sc, s2, ccheck);
      chk_cur = chk_nxt;
      rstr = row_step_r<V>(sc, chk_cur);
    }
    __syncthreads();
  }
  // ---- write back this CTA's rows and columns of the state (every remote store into this CTA
  // came before the last cluster barrier it passed)
  copy_out((V*)ra.qy + r0, qy_r + r0, mr);
  copy_out((V*)ra.yh + r0, yh_r + r0, mr);
  copy_out((V*)ra.y0 + r0, y0_s, mr);
  copy_out((V*)ra.w + r0, w_s, mr);
  copy_out((V*)ra.ax0 + r0, ax0_s, mr);
  copy_out((V*)ra.axh + r0, axh_s, mr);
  copy_out((V*)ra.ax + r0, ax_s, mr);
  copy_out(ca.xbar + c0, xbar_r + c0, nc);
  copy_out(ca.xh0 + c0, xh_r0 + c0, nc);
  copy_out(ca.xh1 + c0, xh_r1 + c0, nc);
  copy_out(ca.x0 + c0, x0_s, nc);
  copy_out(ca.aty0 + c0, aty0_s, nc);
  copy_out(ca.aty + c0, aty_s, nc);
  return true;
}

}  // namespace pdhg
