// Differentiable unrolled solve (include/lp_diff.h): forward K iterations with the schedule
// frozen from a traced solve, and a hand-written adjoint run backwards with checkpointing.
//
// One iteration t of one instance in the scaled, permuted variables (tau = eta/omega_t,
// sigma = eta*omega_t, Section 2.2 eq. (pdhg) with the dual step written sigma (proj(s) - s)):
//   a    = x - tau (c - A^T y)          xhat = clamp(a, l_v, u_v)
//   xbar = 2 xhat - x                   s    = A xbar - y / sigma
//   p    = clamp(s, l_c, u_c)           yhat = sigma (p - s)
//   restart at t: x' = x0' = xhat, y' = y0' = yhat;
//   else (Section 3, reflected Halpern, weights of the epoch step k_t):
//     x' = al xhat + be x + ep x0,  y' = al yhat + be y + ep y0   (anchors kept).
// Adjoint of the same iteration, given the adjoints (lx, ly, lx0, ly0) of (x', y', x0', y0'):
//   restart: lxhat = lx + lx0, lyhat = ly + ly0, nothing flows to x, y, x0, y0;
//   else:    lxhat = al lx, lx_prev = be lx, lx0_prev = lx0 + ep lx (same for y);
//   ls    = sigma (inside_s - 1) lyhat;  l(l_c) += sigma [s < l_c] lyhat;  l(u_c) += sigma [s > u_c] lyhat
//   lv = ls (v = A xbar);  ly_prev -= ls / sigma;  lxbar = A^T lv
//   lxhat += 2 lxbar;  lx_prev -= lxbar
//   la = inside_a lxhat;  l(l_v) += [a < l_v] lxhat;  l(u_v) += [a > u_v] lxhat
//   lx_prev += la;  l(c) -= tau la;  ly_prev += A (tau la)
// The clamp codes (0 inside, 1 below the lower bound, 2 above the upper bound) are all the
// backward pass needs from the forward one; they are recomputed segment by segment from the
// checkpoints.
#include <cooperative_groups.h>

#include <type_traits>

#include "batch.cuh"

namespace cg = cooperative_groups;

namespace pdhg {

namespace {

using Sched = ::DiffSched;

// Frozen schedule of instance k at iteration t from its trace row (r, omega, restart, k_t).
__device__ __forceinline__ Sched sched_from_trace(const double* __restrict__ trace, int64_t cap, int k, int64_t t,
                                                  const double* __restrict__ eta, double gamma) {
  const double* r = trace + ((size_t)k * (size_t)cap + (size_t)t) * 4;
  const double om = r[1], e = eta[k];
  Sched s;
  s.tau = e / om;
  s.sigma = e * om;
  s.inv_sigma = 1.0 / (e * om);
  s.rho = r[2] != 0.0 ? 1 : 0;
  const double kk = r[3];
  const double aw = (kk + 1.0) / (kk + 2.0);
  s.al = aw * (1.0 + gamma);
  s.be = -aw * gamma;
  s.ep = 1.0 / (kk + 2.0);
  return s;
}

// The schedule of every instance and iteration t < K, once, into a table of rows (k, t): the
// per-entry kernels then read their instance's row instead of dividing for every entry.
__global__ void kd_sched_table(const double* __restrict__ trace, int64_t cap, int32_t count, int64_t K,
                               const double* __restrict__ eta, double gamma, Sched* __restrict__ table) {
  const int64_t total = (int64_t)count * K;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    table[q] = sched_from_trace(trace, cap, (int)(q / K), q % K, eta, gamma);
}

__device__ __forceinline__ uint8_t clamp_code(double v, double lo, double hi) {
  return v < lo ? 1 : (v > hi ? 2 : 0);
}

#define GRID_STRIDE(i, len) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (len); i += (int64_t)gridDim.x * blockDim.x)

// Everything one unrolled iteration touches (the batch's permuted, scaled data; the
// differentiation state).
struct DiffArgs {
  const int32_t *rpA, *ciA, *rpT, *ciT;
  const double *valA, *valT;
  const int4 *tasksA, *tasksT;
  int32_t ntA, ntT;
  int64_t n, m;
  const int32_t *irow, *icol;
  const Sched* sched;  // rows (instance, iteration), K per instance
  int64_t K;
  const double *c, *lv, *uv, *lc, *uc;
  double *x, *y, *x0, *y0, *xh, *yh, *xbar;                 // forward state
  double *lx, *ly, *lx0, *ly0, *lsv, *laty;                 // adjoint state (lsv: adjoint of s = of A xbar)
  const double *sx, *sy;                                     // seeds (at the map's last iteration)
  double *gc, *glv, *guv, *glc, *guc;                        // gradients (scaled, permuted)
  const BInst* inst;  // per instance: its rows, columns, tasks and whether it is small
  int32_t skip_local;  // grid kernels: leave the small instances to the cluster kernels
};

// Forward, column j, iteration t: the x update of iteration t - 1 (deferred to here, where the
// same lane owns x[j]), then xhat = clamp(x - tau (c - A^T y)), xbar = 2 xhat - x.
__device__ __forceinline__ void col_fwd(const DiffArgs& a, int64_t j, int64_t t, int64_t t_first, double u,
                                        uint8_t* code) {
  const int k = a.icol[j];
  double xj = a.x[j];
  if (t > t_first) {
    const Sched& p = a.sched[(size_t)k * (size_t)a.K + (size_t)(t - 1)];
    const double h = a.xh[j];
    if (p.rho) {
      xj = h;
      a.x0[j] = h;
    } else {
      xj = p.al * h + p.be * xj + p.ep * a.x0[j];
    }
    a.x[j] = xj;
  }
  const Sched& s = a.sched[(size_t)k * (size_t)a.K + (size_t)t];
  const double av = fma(-s.tau, a.c[j] - u, xj);
  const double lo = a.lv[j], hi = a.uv[j];
  const double h = clampd(av, lo, hi);
  a.xh[j] = h;
  a.xbar[j] = 2.0 * h - xj;
  if (code) code[j] = clamp_code(av, lo, hi);
}

// Forward, the x update of iteration t alone (the last iteration of a launch).
__device__ __forceinline__ void col_upd(const DiffArgs& a, int64_t j, int64_t t) {
  const Sched& p = a.sched[(size_t)a.icol[j] * (size_t)a.K + (size_t)t];
  const double h = a.xh[j];
  if (p.rho) {
    a.x[j] = h;
    a.x0[j] = h;
  } else {
    a.x[j] = p.al * h + p.be * a.x[j] + p.ep * a.x0[j];
  }
}

// Forward, row i, iteration t: yhat = sigma (clamp(s) - s), s = A xbar - y / sigma, then the y
// update (Halpern or restart).
__device__ __forceinline__ void row_fwd(const DiffArgs& a, int64_t i, int64_t t, double v, uint8_t* code) {
  const Sched& s = a.sched[(size_t)a.irow[i] * (size_t)a.K + (size_t)t];
  const double yi = a.y[i];
  const double sv = fma(-yi, s.inv_sigma, v);  // v - y / sigma, with 1/sigma from the table
  const double lo = a.lc[i], hi = a.uc[i];
  const double h = s.sigma * (clampd(sv, lo, hi) - sv);
  a.yh[i] = h;
  if (code) code[i] = clamp_code(sv, lo, hi);
  if (s.rho) {
    a.y[i] = h;
    a.y0[i] = h;
  } else {
    a.y[i] = s.al * h + s.be * yi + s.ep * a.y0[i];
  }
}

// Adjoint, row i, iteration t (first half): from (ly, ly0) of (y', y0') to lv = ls and the
// partial adjoints of (y, y0); accumulates the row-bound gradients.
__device__ __forceinline__ void row_bwd(const DiffArgs& a, int64_t i, int64_t t, int64_t K, const uint8_t* code) {
  const Sched& s = a.sched[(size_t)a.irow[i] * (size_t)a.K + (size_t)t];
  const double a_y = a.ly[i], a_y0 = a.ly0[i];
  double lyh, lyp, ly0p;
  if (s.rho) {
    lyh = a_y + a_y0;
    lyp = 0.0;
    ly0p = 0.0;
  } else {
    lyh = s.al * a_y;
    lyp = s.be * a_y;
    ly0p = a_y0 + s.ep * a_y;
  }
  if (t == K - 1) lyh += a.sy[i];
  const uint8_t cd = code[i];
  const double ls = cd == 0 ? 0.0 : -s.sigma * lyh;
  if (cd == 1) a.glc[i] += s.sigma * lyh;
  if (cd == 2) a.guc[i] += s.sigma * lyh;
  a.lsv[i] = ls;
  a.ly[i] = fma(-ls, s.inv_sigma, lyp);  // lyp - ls / sigma (the adjoint of the same product)
  a.ly0[i] = ly0p;
}

// Adjoint, column j, iteration t: from (lx, lx0) and lxbar = (A^T lv)_j to the adjoints of
// (x, x0) and laty = tau la; accumulates the gradients of c and the variable bounds.
__device__ __forceinline__ void col_bwd(const DiffArgs& a, int64_t j, int64_t t, int64_t K, double lb,
                                        const uint8_t* code) {
  const Sched& s = a.sched[(size_t)a.icol[j] * (size_t)a.K + (size_t)t];
  const double a_x = a.lx[j], a_x0 = a.lx0[j];
  double lxh, lxp, lx0p;
  if (s.rho) {
    lxh = a_x + a_x0;
    lxp = 0.0;
    lx0p = 0.0;
  } else {
    lxh = s.al * a_x;
    lxp = s.be * a_x;
    lx0p = a_x0 + s.ep * a_x;
  }
  if (t == K - 1) lxh += a.sx[j];
  lxh += 2.0 * lb;
  lxp -= lb;
  const uint8_t cd = code[j];
  const double la = cd == 0 ? lxh : 0.0;
  if (cd == 1) a.glv[j] += lxh;
  if (cd == 2) a.guv[j] += lxh;
  lxp += la;
  a.gc[j] -= s.tau * la;
  a.laty[j] = s.tau * la;
  a.lx[j] = lxp;
  a.lx0[j] = lx0p;
}

__device__ __forceinline__ int dtask_lanes(const int4& t) { return t.z >> 24; }
__device__ __forceinline__ int dtask_per_lane(const int4& t) { return t.z & 0xFFFFFF; }

// Forward: iterations t0 .. t0 + len - 1 of every instance, one cooperative launch (all blocks
// resident).  Per iteration: column phase (A^T y by column tiles, then col_fwd, which first
// applies the previous iteration's deferred x update), grid barrier, row phase (A xbar by row
// tiles, then row_fwd), grid barrier.  The last iteration's x update ends the launch, so the
// state (x, y, x0, y0) is complete between launches.  cx / cy (or NULL): where iteration
// t0 + o stores its clamp codes, at cx + o n and cy + o m.
__global__ void __launch_bounds__(kThreads, 3) kd_fwd_loop(DiffArgs a, int64_t t0, int32_t len, uint8_t* cx,
                                                           uint8_t* cy) {
  cg::grid_group grid = cg::this_grid();
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5), nw = gridDim.x * kWarps;
  for (int32_t o = 0; o < len; ++o) {
    const int64_t t = t0 + o;
    uint8_t* ccx = cx ? cx + (size_t)o * (size_t)a.n : nullptr;
    uint8_t* ccy = cy ? cy + (size_t)o * (size_t)a.m : nullptr;
    for (int j = gw; j < a.ntT; j += nw) {
      const int4 td = a.tasksT[j];
      if (a.skip_local && a.inst[td.w].local) continue;  // warp-uniform
      const double u = tile_spmv(a.rpT, a.ciT, a.valT, a.y, td.x, td.y, dtask_lanes(td), dtask_per_lane(td), lane, pol);
      if (lane < td.y) col_fwd(a, td.x + lane, t, t0, u, ccx);
    }
    grid.sync();
    for (int j = gw; j < a.ntA; j += nw) {
      const int4 td = a.tasksA[j];
      if (a.skip_local && a.inst[td.w].local) continue;
      const double v = tile_spmv(a.rpA, a.ciA, a.valA, a.xbar, td.x, td.y, dtask_lanes(td), dtask_per_lane(td), lane, pol);
      if (lane < td.y) row_fwd(a, td.x + lane, t, v, ccy);
    }
    grid.sync();
  }
  if (len > 0) {
    GRID_STRIDE(j, a.n) {
      if (!a.skip_local || !a.inst[a.icol[j]].local) col_upd(a, j, t0 + len - 1);
    }
  }
}

// Adjoint of iterations t0 + len - 1 down to t0 (codes of iteration t0 + o at cx + o n,
// cy + o m), one cooperative launch.  Per iteration: column phase (lxbar = A^T lv by column
// tiles, then col_bwd), grid barrier, row phase (A laty by row tiles, added to ly, then the
// first half of the previous iteration's adjoint, row_bwd, in the same lane), grid barrier.
// The launch starts with row_bwd of its last iteration.
__global__ void __launch_bounds__(kThreads, 3) kd_bwd_loop(DiffArgs a, int64_t t0, int64_t K, int32_t len,
                                                           const uint8_t* cx, const uint8_t* cy) {
  cg::grid_group grid = cg::this_grid();
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5), nw = gridDim.x * kWarps;
  if (len <= 0) return;
  {
    const uint8_t* ccy = cy + (size_t)(len - 1) * (size_t)a.m;
    GRID_STRIDE(i, a.m) {
      if (!a.skip_local || !a.inst[a.irow[i]].local) row_bwd(a, i, t0 + len - 1, K, ccy);
    }
  }
  grid.sync();
  for (int32_t o = len - 1; o >= 0; --o) {
    const int64_t t = t0 + o;
    const uint8_t* ccx = cx + (size_t)o * (size_t)a.n;
    for (int j = gw; j < a.ntT; j += nw) {
      const int4 td = a.tasksT[j];
      if (a.skip_local && a.inst[td.w].local) continue;
      const double lb = tile_spmv(a.rpT, a.ciT, a.valT, a.lsv, td.x, td.y, dtask_lanes(td), dtask_per_lane(td), lane, pol);
      if (lane < td.y) col_bwd(a, td.x + lane, t, K, lb, ccx);
    }
    grid.sync();
    const uint8_t* ccy = o > 0 ? cy + (size_t)(o - 1) * (size_t)a.m : nullptr;
    for (int j = gw; j < a.ntA; j += nw) {
      const int4 td = a.tasksA[j];
      if (a.skip_local && a.inst[td.w].local) continue;
      const double w = tile_spmv(a.rpA, a.ciA, a.valA, a.laty, td.x, td.y, dtask_lanes(td), dtask_per_lane(td), lane, pol);
      if (lane < td.y) {
        const int64_t i = td.x + lane;
        a.ly[i] += w;
        if (o > 0) row_bwd(a, i, t - 1, K, ccy);
      }
    }
    grid.sync();
  }
}

// The same two segment kernels for the small instances (BInst::local), one instance per cluster
// of kCtas CTAs at a time: the instance's tasks are spread over the cluster's warps and its two
// phases per iteration are separated by cluster barriers instead of grid barriers.  The
// matrix slice is re-read every iteration by the same SMs, so it is loaded through L1.
template <int kCtas>
__device__ __forceinline__ void kd_cluster_sync() {
  if (kCtas > 1) cg::this_cluster().sync();
  else __syncthreads();
}

template <int kCtas>
__global__ void __launch_bounds__(kThreads, 2) kd_fwd_cluster(DiffArgs a, const int32_t* __restrict__ list,
                                                              int32_t nlist, int64_t t0, int32_t len, uint8_t* cx,
                                                              uint8_t* cy) {
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = (int)(blockIdx.x % kCtas), cid = (int)(blockIdx.x / kCtas), ncl = (int)(gridDim.x / kCtas);
  const int w0 = rank * kWarps + warp, wstep = kCtas * kWarps;
  for (int q = cid; q < nlist; q += ncl) {
    const BInst I = a.inst[list[q]];
    for (int32_t o = 0; o < len; ++o) {
      const int64_t t = t0 + o;
      uint8_t* ccx = cx ? cx + (size_t)o * (size_t)a.n : nullptr;
      uint8_t* ccy = cy ? cy + (size_t)o * (size_t)a.m : nullptr;
      for (int j = w0; j < I.ntt; j += wstep) {
        const int4 td = a.tasksT[I.tt0 + j];
        const double u = tile_spmv<double, true>(a.rpT, a.ciT, a.valT, a.y, td.x, td.y, dtask_lanes(td),
                                                 dtask_per_lane(td), lane, pol);
        if (lane < td.y) col_fwd(a, td.x + lane, t, t0, u, ccx);
      }
      kd_cluster_sync<kCtas>();
      for (int j = w0; j < I.nta; j += wstep) {
        const int4 td = a.tasksA[I.ta0 + j];
        const double v = tile_spmv<double, true>(a.rpA, a.ciA, a.valA, a.xbar, td.x, td.y, dtask_lanes(td),
                                                 dtask_per_lane(td), lane, pol);
        if (lane < td.y) row_fwd(a, td.x + lane, t, v, ccy);
      }
      kd_cluster_sync<kCtas>();
    }
    if (len > 0)
      for (int64_t j = I.col0 + (int64_t)rank * kThreads + threadIdx.x; j < (int64_t)I.col0 + I.n;
           j += (int64_t)kCtas * kThreads)
        col_upd(a, j, t0 + len - 1);
  }
}

template <int kCtas>
__global__ void __launch_bounds__(kThreads, 2) kd_bwd_cluster(DiffArgs a, const int32_t* __restrict__ list,
                                                              int32_t nlist, int64_t t0, int64_t K, int32_t len,
                                                              const uint8_t* cx, const uint8_t* cy) {
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = (int)(blockIdx.x % kCtas), cid = (int)(blockIdx.x / kCtas), ncl = (int)(gridDim.x / kCtas);
  const int w0 = rank * kWarps + warp, wstep = kCtas * kWarps;
  if (len <= 0) return;
  for (int q = cid; q < nlist; q += ncl) {
    const BInst I = a.inst[list[q]];
    {
      const uint8_t* ccy = cy + (size_t)(len - 1) * (size_t)a.m;
      for (int64_t i = I.row0 + (int64_t)rank * kThreads + threadIdx.x; i < (int64_t)I.row0 + I.m;
           i += (int64_t)kCtas * kThreads)
        row_bwd(a, i, t0 + len - 1, K, ccy);
    }
    kd_cluster_sync<kCtas>();
    for (int32_t o = len - 1; o >= 0; --o) {
      const int64_t t = t0 + o;
      const uint8_t* ccx = cx + (size_t)o * (size_t)a.n;
      for (int j = w0; j < I.ntt; j += wstep) {
        const int4 td = a.tasksT[I.tt0 + j];
        const double lb = tile_spmv<double, true>(a.rpT, a.ciT, a.valT, a.lsv, td.x, td.y, dtask_lanes(td),
                                                  dtask_per_lane(td), lane, pol);
        if (lane < td.y) col_bwd(a, td.x + lane, t, K, lb, ccx);
      }
      kd_cluster_sync<kCtas>();
      const uint8_t* ccy = o > 0 ? cy + (size_t)(o - 1) * (size_t)a.m : nullptr;
      for (int j = w0; j < I.nta; j += wstep) {
        const int4 td = a.tasksA[I.ta0 + j];
        const double w = tile_spmv<double, true>(a.rpA, a.ciA, a.valA, a.laty, td.x, td.y, dtask_lanes(td),
                                                 dtask_per_lane(td), lane, pol);
        if (lane < td.y) {
          const int64_t i = td.x + lane;
          a.ly[i] += w;
          if (o > 0) row_bwd(a, i, t - 1, K, ccy);
        }
      }
      kd_cluster_sync<kCtas>();
    }
  }
}

// Instance of every permuted row and column.
__global__ void kd_owner(const BInst* __restrict__ inst, int32_t count, int32_t* irow, int32_t* icol) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const BInst I = inst[k];
    for (int i = threadIdx.x; i < I.m; i += blockDim.x) irow[I.row0 + i] = k;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) icol[I.col0 + j] = k;
  }
}

// Permuted/scaled <-> original/concatenated maps.  Position p of instance k holds original
// entry off_k + perm[p] (off_k = row0 or col0: the original concatenated layout has the same
// per-instance offsets).
// dst[p] = src[off + perm[p]] * mul[p]          (mode 0)
// dst[p] = src[off + perm[p]] / mul[p]          (mode 1)
__global__ void kd_gather(int64_t len, const int32_t* __restrict__ owner, const BInst* __restrict__ inst,
                          int32_t is_col, const int32_t* __restrict__ perm, const double* __restrict__ src,
                          const double* __restrict__ mul, int32_t mode, double* __restrict__ dst) {
  GRID_STRIDE(p, len) {
    const BInst I = inst[owner[p]];
    const int64_t o = (int64_t)(is_col ? I.col0 : I.row0) + perm[p];
    const double v = src[o];
    dst[p] = mode == 0 ? v * mul[p] : v / mul[p];
  }
}

// dst[off + perm[p]] = src[p] * mul[p]  (mode 0)  or  src[p] / mul[p]  (mode 1)
__global__ void kd_scatter(int64_t len, const int32_t* __restrict__ owner, const BInst* __restrict__ inst,
                           int32_t is_col, const int32_t* __restrict__ perm, const double* __restrict__ src,
                           const double* __restrict__ mul, int32_t mode, double* __restrict__ dst) {
  GRID_STRIDE(p, len) {
    const BInst I = inst[owner[p]];
    const int64_t o = (int64_t)(is_col ? I.col0 : I.row0) + perm[p];
    const double v = src[p];
    dst[o] = mode == 0 ? v * mul[p] : v / mul[p];
  }
}

// KKT denominators of every instance from the original data (block per instance): ||c||_2 and
// the 2-norm of the finite row bounds, into the scalar-state templates.
__global__ void __launch_bounds__(kThreads) kd_norms(const BInst* __restrict__ inst, int32_t count,
                                                     const double* __restrict__ c, const double* __restrict__ lc,
                                                     const double* __restrict__ uc, Ctl* init) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const BInst I = inst[k];
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < I.n; j += kThreads) s[0] = fma(c[I.col0 + j], c[I.col0 + j], s[0]);
    for (int i = threadIdx.x; i < I.m; i += kThreads) {
      const double l = lc[I.row0 + i], u = uc[I.row0 + i];
      if (isfinite(l)) s[1] = fma(l, l, s[1]);
      if (isfinite(u)) s[1] = fma(u, u, s[1]);
    }
    block_reduce(s, 2);
    if (threadIdx.x == 0) {
      init[k].c_norm = sqrt(s[0]);
      init[k].lu_norm = sqrt(s[1]);
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace pdhg

namespace {

int vgrid(const lp_batch* h, int64_t len) { return grid_for(std::max<int64_t>(len, 1), 256, 8 * h->num_sms); }

lp_status diff_buffers(lp_batch* h) {
  if (h->diff) return LP_OK;
  Diff* d = new Diff();
  h->diff = d;
  auto get = [&](auto** p, size_t count) -> cudaError_t {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(**p));
    if (e == cudaSuccess) d->own.push_back(v);
    *p = static_cast<std::remove_reference_t<decltype(*p)>>(v);
    return e;
  };
  const size_t n = (size_t)h->sum_n, m = (size_t)h->sum_m;
  CK(get(&d->irow, m)); CK(get(&d->icol, n));
  for (double** p : {&d->x, &d->x0, &d->xh, &d->xbar, &d->lx, &d->lx0, &d->lxbar, &d->laty, &d->sx,
                     &d->gc, &d->glv, &d->guv})
    CK(get(p, n));
  for (double** p : {&d->y, &d->y0, &d->yh, &d->ly, &d->ly0, &d->lv, &d->sy, &d->glc, &d->guc})
    CK(get(p, m));
  kd_owner<<<h->gridS, kThreads, 0, h->setup_stream>>>(h->d_inst, h->count, d->irow, d->icol);
  CK(cudaGetLastError());
  if (!h->d_eta) {
    CK(h->alloc(&h->d_eta, h->count));
    CK(cudaMemcpy(h->d_eta, h->eta.data(), sizeof(double) * h->count, cudaMemcpyHostToDevice));
  }
  CK(cudaDeviceSynchronize());  // the setup stream's kernel and the step sizes' copy
  return LP_OK;
}

// Resizes a buffer that only grows (contents are not kept).
template <class T>
lp_status grow(T** p, int64_t* cap, int64_t need) {
  if (*cap >= need) return LP_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  CK(cudaMalloc(p, sizeof(T) * (size_t)std::max<int64_t>(need, 1)));
  *cap = need;
  return LP_OK;
}

DiffArgs diff_args(const lp_batch* h) {
  const Diff* d = h->diff;
  DiffArgs a;
  a.rpA = h->rpA; a.ciA = h->ciA; a.rpT = h->rpT; a.ciT = h->ciT; a.valA = h->valA; a.valT = h->valT;
  a.tasksA = h->tasksA; a.tasksT = h->tasksT; a.ntA = h->ntA; a.ntT = h->ntT;
  a.n = h->sum_n; a.m = h->sum_m;
  a.irow = d->irow; a.icol = d->icol; a.sched = d->sched; a.K = d->K;
  a.c = h->c; a.lv = h->lv; a.uv = h->uv; a.lc = h->lc; a.uc = h->uc;
  a.x = d->x; a.y = d->y; a.x0 = d->x0; a.y0 = d->y0; a.xh = d->xh; a.yh = d->yh; a.xbar = d->xbar;
  a.lx = d->lx; a.ly = d->ly; a.lx0 = d->lx0; a.ly0 = d->ly0; a.lsv = d->lv; a.laty = d->laty;
  a.sx = d->sx; a.sy = d->sy;
  a.gc = d->gc; a.glv = d->glv; a.guv = d->guv; a.glc = d->glc; a.guc = d->guc;
  a.inst = h->d_inst;
  a.skip_local = h->n_local > 0 ? 1 : 0;
  return a;
}

lp_status coop_launch(lp_batch* h, const void* fn, void** args, cudaStream_t s) {
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, 0));
  if (occ < 1) occ = 1;
  CK(cudaLaunchCooperativeKernel(fn, dim3((unsigned)(occ * h->num_sms)), dim3(kThreads), args, 0, s));
  return LP_OK;
}

// Cluster launch of a small-instance segment kernel (fn<kCtas>) over the handle's small
// instances, `clusters` clusters of kCtas CTAs.
template <int kCtas, class... Args>
lp_status cluster_launch(void (*fn)(Args...), int clusters, cudaStream_t s, Args... args) {
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
  CK(cudaLaunchKernelEx(&cfg, fn, args...));
  return LP_OK;
}

// CTAs per cluster for the small instances: the most (8, 4, 2 or 1) with which every small
// instance has its own cluster resident at once (an instance's iterations are a chain of
// barriers, so a second wave of clusters costs a second pass of that chain); 1 when even single
// CTAs take more than one wave (throughput then decides, and one CTA needs no cluster barrier).
int diff_cluster_ctas(const lp_batch* h, int* clusters) {
  int occ = 0, occ_b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kd_fwd_cluster<8>, kThreads, 0) != cudaSuccess) occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, kd_bwd_cluster<8>, kThreads, 0) != cudaSuccess) occ_b = 1;
  occ = std::max(1, std::min(occ, occ_b));
  const int64_t slots = (int64_t)occ * h->num_sms;
  int k = 8;
  while (k > 1 && (int64_t)h->n_local * k > slots) k >>= 1;
  *clusters = (int)std::max<int64_t>(1, std::min<int64_t>(h->n_local, slots / k));
  return k;
}

// Forward iterations t0 .. t0 + len - 1 (codes stored when cx, cy are given): the grid kernel
// over the large instances, then the cluster kernel over the small ones.
lp_status forward_run(lp_batch* h, int64_t t0, int32_t len, uint8_t* cx, uint8_t* cy, cudaStream_t s) {
  DiffArgs a = diff_args(h);
  if (h->n_local < h->count) {
    void* args[] = {&a, &t0, &len, &cx, &cy};
    const lp_status st = coop_launch(h, reinterpret_cast<const void*>(kd_fwd_loop), args, s);
    if (st != LP_OK) return st;
  }
  if (h->n_local > 0) {
    int cl = 1;
    const int k = diff_cluster_ctas(h, &cl);
    const int32_t* list = h->local_list;
    const int32_t nl = h->n_local;
    if (k == 8) return cluster_launch<8>(kd_fwd_cluster<8>, cl, s, a, list, nl, t0, len, cx, cy);
    if (k == 4) return cluster_launch<4>(kd_fwd_cluster<4>, cl, s, a, list, nl, t0, len, cx, cy);
    if (k == 2) return cluster_launch<2>(kd_fwd_cluster<2>, cl, s, a, list, nl, t0, len, cx, cy);
    return cluster_launch<1>(kd_fwd_cluster<1>, cl, s, a, list, nl, t0, len, cx, cy);
  }
  return LP_OK;
}

// Adjoint of iterations t0 + len - 1 down to t0 of a map of K iterations.
lp_status backward_run(lp_batch* h, int64_t t0, int64_t K, int32_t len, const uint8_t* cx, const uint8_t* cy,
                       cudaStream_t s) {
  DiffArgs a = diff_args(h);
  if (h->n_local < h->count) {
    void* args[] = {&a, &t0, &K, &len, &cx, &cy};
    const lp_status st = coop_launch(h, reinterpret_cast<const void*>(kd_bwd_loop), args, s);
    if (st != LP_OK) return st;
  }
  if (h->n_local > 0) {
    int cl = 1;
    const int k = diff_cluster_ctas(h, &cl);
    const int32_t* list = h->local_list;
    const int32_t nl = h->n_local;
    if (k == 8) return cluster_launch<8>(kd_bwd_cluster<8>, cl, s, a, list, nl, t0, K, len, cx, cy);
    if (k == 4) return cluster_launch<4>(kd_bwd_cluster<4>, cl, s, a, list, nl, t0, K, len, cx, cy);
    if (k == 2) return cluster_launch<2>(kd_bwd_cluster<2>, cl, s, a, list, nl, t0, K, len, cx, cy);
    return cluster_launch<1>(kd_bwd_cluster<1>, cl, s, a, list, nl, t0, K, len, cx, cy);
  }
  return LP_OK;
}

// Checkpoint q: (x, y, x0, y0) of the diff state.
double* ck_slot(lp_batch* h, int64_t q) {
  return h->diff->ck + (size_t)q * 2 * (size_t)(h->sum_n + h->sum_m);
}

lp_status save_ck(lp_batch* h, int64_t q, cudaStream_t s) {
  Diff* d = h->diff;
  const size_t n = (size_t)h->sum_n, m = (size_t)h->sum_m;
  double* c = ck_slot(h, q);
  CK(cudaMemcpyAsync(c, d->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c + n, d->x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c + 2 * n, d->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c + 2 * n + m, d->y0, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  return LP_OK;
}

lp_status load_ck(lp_batch* h, int64_t q, cudaStream_t s) {
  Diff* d = h->diff;
  const size_t n = (size_t)h->sum_n, m = (size_t)h->sum_m;
  const double* c = ck_slot(h, q);
  CK(cudaMemcpyAsync(d->x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d->x0, c + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d->y, c + 2 * n, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d->y0, c + 2 * n + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  return LP_OK;
}

lp_status zero(double* p, int64_t len, cudaStream_t s) {
  if (len > 0) CK(cudaMemsetAsync(p, 0, sizeof(double) * (size_t)len, s));
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_batch_set_data(lp_batch_handle h, const double* c, const double* l_c, const double* u_c,
                            const double* l_v, const double* u_v, int32_t where) {
  pdhg_set_last_error(std::string());
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (where != LP_HOST && where != LP_DEVICE) return fail(LP_ERR_INVALID_ARG, "where must be LP_HOST or LP_DEVICE");
  const int64_t n = h->sum_n, m = h->sum_m;
  if (where == LP_HOST) {
    for (int64_t j = 0; c && j < n; ++j)
      if (!std::isfinite(c[j])) return fail(LP_ERR_INVALID_INPUT, "non-finite objective entry " + std::to_string(j));
    // each given bound: no NaN, no +inf lower, no -inf upper; lower <= upper when both given
    auto check = [](const double* lo, const double* hi, int64_t len, const char* what) -> lp_status {
      for (int64_t i = 0; i < len; ++i) {
        const bool bad = (lo && (std::isnan(lo[i]) || lo[i] == INFINITY)) ||
                         (hi && (std::isnan(hi[i]) || hi[i] == -INFINITY)) || (lo && hi && lo[i] > hi[i]);
        if (bad) return fail(LP_ERR_INVALID_INPUT, std::string("bad ") + what + " bounds at " + std::to_string(i));
      }
      return LP_OK;
    };
    lp_status v = check(l_v, u_v, n, "variable");
    if (v != LP_OK) return v;
    v = check(l_c, u_c, m, "row");
    if (v != LP_OK) return v;
  }
  CK(cudaSetDevice(h->device));
  lp_status st = diff_buffers(h);
  if (st != LP_OK) return st;
  cudaStream_t s = h->setup_stream;
  Diff* d = h->diff;
  // stage the original-order data on the device (host data: one copy each)
  auto stage = [&](const double* src, int64_t len, double* tmp) -> const double* {
    if (!src) return nullptr;
    if (where == LP_DEVICE) return src;
    cudaMemcpyAsync(tmp, src, sizeof(double) * (size_t)len, cudaMemcpyHostToDevice, s);
    return tmp;
  };
  // the adjoint buffers are free between calls: use them as staging space
  const double* dc_ = stage(c, n, d->lx);
  const double* dlv = stage(l_v, n, d->lx0);
  const double* duv = stage(u_v, n, d->lxbar);
  const double* dlc = stage(l_c, m, d->ly);
  const double* duc = stage(u_c, m, d->ly0);
  CK(cudaGetLastError());
  if (dc_) kd_gather<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, dc_, h->dc, 0, h->c);
  if (dlv) kd_gather<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, dlv, h->dc, 1, h->lv);
  if (duv) kd_gather<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, duv, h->dc, 1, h->uv);
  if (dlc) kd_gather<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, dlc, h->dr, 0, h->lc);
  if (duc) kd_gather<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, duc, h->dr, 0, h->uc);
  CK(cudaGetLastError());
  // KKT denominators from the original data now in force: unscale the stored scaled vectors
  // into staging space (c = c~ / d_c, l_c = l_c~ / d_r, u_c = u_c~ / d_r) and reduce per instance
  kd_scatter<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, h->c, h->dc, 1, d->gc);
  kd_scatter<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, h->lc, h->dr, 1, d->glc);
  kd_scatter<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, h->uc, h->dr, 1, d->guc);
  kd_norms<<<h->gridS, kThreads, 0, s>>>(h->d_inst, h->count, d->gc, d->glc, d->guc, h->ctl_init);
  CK(cudaGetLastError());
  if (h->prm.precision != 0) {
    auto& f = h->f32;
    k_to_float<<<vgrid(h, n), 256, 0, s>>>(n, h->c, f.c);
    k_to_float<<<vgrid(h, n), 256, 0, s>>>(n, h->lv, f.lv);
    k_to_float<<<vgrid(h, n), 256, 0, s>>>(n, h->uv, f.uv);
    k_to_float<<<vgrid(h, m), 256, 0, s>>>(m, h->lc, f.lc);
    k_to_float<<<vgrid(h, m), 256, 0, s>>>(m, h->uc, f.uc);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  d->forward_done = false;
  return LP_OK;
}

lp_status lp_batch_unroll(lp_batch_handle h, int64_t K, int64_t checkpoint_every, double* x, double* y,
                          void* stream) {
  pdhg_set_last_error(std::string());
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (K < 1 || checkpoint_every < 1) return fail(LP_ERR_INVALID_ARG, "K and checkpoint_every must be >= 1");
  if (h->prm.precision != 0) return fail(LP_ERR_INVALID_ARG, "differentiation needs a batch created with precision 0");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lp_status st = diff_buffers(h);
  if (st != LP_OK) return st;
  Diff* d = h->diff;
  // 1. the frozen schedule, and its table of step sizes and Halpern weights
  st = batch_schedule_solve(h, K, s);
  if (st != LP_OK) return st;
  st = grow(&d->sched, &d->cap_sched, (int64_t)h->count * K);
  if (st != LP_OK) return st;
  kd_sched_table<<<vgrid(h, (int64_t)h->count * K), 256, 0, s>>>(h->trace, h->trace_cap, h->count, K, h->d_eta,
                                                                  h->prm.gamma, d->sched);
  CK(cudaGetLastError());
  d->K = K;
  // 2. the unrolled iterations from zero, with checkpoints
  const int64_t C = checkpoint_every;
  const int64_t nck = (K + C - 1) / C;
  st = grow(&d->ck, &d->cap_ck, nck * 2 * (h->sum_n + h->sum_m));
  if (st != LP_OK) return st;
  for (double* p : {d->x, d->x0}) {
    st = zero(p, h->sum_n, s);
    if (st != LP_OK) return st;
  }
  for (double* p : {d->y, d->y0}) {
    st = zero(p, h->sum_m, s);
    if (st != LP_OK) return st;
  }
  for (int64_t q = 0; q < nck; ++q) {
    const int64_t t0 = q * C, len = std::min(C, K - t0);
    st = save_ck(h, q, s);
    if (st == LP_OK) st = forward_run(h, t0, (int32_t)len, nullptr, nullptr, s);
    if (st != LP_OK) return st;
  }
  // 3. the output zhat of the last iteration in the original variables
  if (x && h->sum_n > 0)
    kd_scatter<<<vgrid(h, h->sum_n), 256, 0, s>>>(h->sum_n, d->icol, h->d_inst, 1, h->col_perm, d->xh, h->dc, 0, x);
  if (y && h->sum_m > 0)
    kd_scatter<<<vgrid(h, h->sum_m), 256, 0, s>>>(h->sum_m, d->irow, h->d_inst, 0, h->row_perm, d->yh, h->dr, 0, y);
  CK(cudaGetLastError());
  d->K = K;
  d->C = C;
  d->forward_done = true;
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_batch_unroll_vjp(lp_batch_handle h, const double* dl_dx, const double* dl_dy, double* dl_dc,
                              double* dl_dlc, double* dl_duc, double* dl_dlv, double* dl_duv, void* stream) {
  pdhg_set_last_error(std::string());
  if (!h) return fail(LP_ERR_INVALID_ARG, "NULL handle");
  if (!h->diff || !h->diff->forward_done) return fail(LP_ERR_NOT_SOLVED, "no lp_batch_unroll to differentiate");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Diff* d = h->diff;
  const int64_t n = h->sum_n, m = h->sum_m, K = d->K, C = d->C;
  lp_status st = grow(&d->mx, &d->cap_mask, C * std::max<int64_t>(n + m, 1));
  if (st != LP_OK) return st;
  d->my = nullptr;  // the row codes of a segment follow its column codes in the same buffer
  // seeds: lxhat = dL/dx * d_c, lyhat = dL/dy * d_r at the permuted positions
  if (dl_dx && n > 0) kd_gather<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, dl_dx, h->dc, 0, d->sx);
  else st = zero(d->sx, n, s);
  if (st != LP_OK) return st;
  if (dl_dy && m > 0) kd_gather<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, dl_dy, h->dr, 0, d->sy);
  else st = zero(d->sy, m, s);
  if (st != LP_OK) return st;
  for (double* p : {d->lx, d->lx0, d->gc, d->glv, d->guv}) {
    st = zero(p, n, s);
    if (st != LP_OK) return st;
  }
  for (double* p : {d->ly, d->ly0, d->glc, d->guc}) {
    st = zero(p, m, s);
    if (st != LP_OK) return st;
  }
  CK(cudaGetLastError());
  for (int64_t q = (K + C - 1) / C - 1; q >= 0; --q) {
    const int64_t t0 = q * C, len = std::min(C, K - t0);
    uint8_t* cx = d->mx;
    uint8_t* cy = d->mx + (size_t)len * (size_t)n;
    st = load_ck(h, q, s);
    if (st == LP_OK) st = forward_run(h, t0, (int32_t)len, cx, cy, s);
    if (st == LP_OK) st = backward_run(h, t0, K, (int32_t)len, cx, cy, s);
    if (st != LP_OK) return st;
  }
  // gradients in the original variables: c~ = d_c c, l_v~ = l_v / d_c, l_c~ = d_r l_c
  if (dl_dc && n > 0) kd_scatter<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, d->gc, h->dc, 0, dl_dc);
  if (dl_dlv && n > 0) kd_scatter<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, d->glv, h->dc, 1, dl_dlv);
  if (dl_duv && n > 0) kd_scatter<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->d_inst, 1, h->col_perm, d->guv, h->dc, 1, dl_duv);
  if (dl_dlc && m > 0) kd_scatter<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, d->glc, h->dr, 0, dl_dlc);
  if (dl_duc && m > 0) kd_scatter<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->d_inst, 0, h->row_perm, d->guc, h->dr, 0, dl_duc);
  CK(cudaGetLastError());
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_batch_time_unroll(lp_batch_handle h, int32_t reps, void* stream, double* ms_out) {
  pdhg_set_last_error(std::string());
  if (!h || !ms_out || reps < 1) return fail(LP_ERR_INVALID_ARG, "bad argument");
  if (!h->diff || !h->diff->forward_done) return fail(LP_ERR_NOT_SOLVED, "no lp_batch_unroll to time");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Diff* d = h->diff;
  const int64_t n = h->sum_n, m = h->sum_m;
  const int32_t len = (int32_t)std::min(d->C, d->K);
  lp_status st = grow(&d->mx, &d->cap_mask, d->C * std::max<int64_t>(n + m, 1));
  if (st != LP_OK) return st;
  uint8_t* cx = d->mx;
  uint8_t* cy = d->mx + (size_t)len * (size_t)n;
  for (double* p : {d->lx, d->lx0, d->gc, d->glv, d->guv, d->sx}) {
    st = zero(p, n, s);
    if (st != LP_OK) return st;
  }
  for (double* p : {d->ly, d->ly0, d->glc, d->guc, d->sy}) {
    st = zero(p, m, s);
    if (st != LP_OK) return st;
  }
  std::vector<cudaEvent_t> ev(6 * (size_t)reps, nullptr);
  struct Events {
    std::vector<cudaEvent_t>& v;
    ~Events() {
      for (auto& e : v)
        if (e) cudaEventDestroy(e);
    }
  } guard{ev};
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int kind = 0; kind < 3; ++kind) {
    for (int32_t r = 0; r < reps; ++r) {
      cudaEvent_t e0 = ev[2 * ((size_t)kind * reps + r)], e1 = ev[2 * ((size_t)kind * reps + r) + 1];
      if (kind < 2) st = load_ck(h, 0, s);
      if (st != LP_OK) return st;
      CK(cudaEventRecord(e0, s));
      if (kind == 0) st = forward_run(h, 0, len, nullptr, nullptr, s);
      else if (kind == 1) st = forward_run(h, 0, len, cx, cy, s);
      else st = backward_run(h, 0, d->K, len, cx, cy, s);
      if (st != LP_OK) return st;
      CK(cudaEventRecord(e1, s));
    }
  }
  CK(cudaStreamSynchronize(s));
  for (int kind = 0; kind < 3; ++kind) {
    double tot = 0.0;
    for (int32_t r = 0; r < reps; ++r) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[2 * ((size_t)kind * reps + r)], ev[2 * ((size_t)kind * reps + r) + 1]));
      tot += ms;
    }
    ms_out[kind] = tot / reps;
  }
  ms_out[3] = (double)len;
  h->last_stream = s;
  return LP_OK;
}

}  // extern "C"
