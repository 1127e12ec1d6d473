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
#include <type_traits>

#include "batch.cuh"

namespace pdhg {

namespace {

struct Sched {
  double tau, sigma, al, be, ep;
  int rho;
};

// Iteration of a kernel = clk->t0 + its offset in the segment; clk->K = the map's length (the
// seeds enter at its last iteration).  One captured segment serves every segment this way.
__global__ void kd_set_clock(DiffClock* clk, int64_t t0, int64_t K) {
  clk->t0 = t0;
  clk->K = K;
}

// Frozen schedule of instance k at iteration t from its trace row (r, omega, restart, k_t).
__device__ __forceinline__ Sched sched_at(const double* __restrict__ trace, int64_t cap, int k, int64_t t,
                                          const double* __restrict__ eta, double gamma) {
  const double* r = trace + ((size_t)k * (size_t)cap + (size_t)t) * 4;
  const double om = r[1], e = eta[k];
  Sched s;
  s.tau = e / om;
  s.sigma = e * om;
  s.rho = r[2] != 0.0 ? 1 : 0;
  const double kk = r[3];
  const double aw = (kk + 1.0) / (kk + 2.0);
  s.al = aw * (1.0 + gamma);
  s.be = -aw * gamma;
  s.ep = 1.0 / (kk + 2.0);
  return s;
}

__device__ __forceinline__ uint8_t clamp_code(double v, double lo, double hi) {
  return v < lo ? 1 : (v > hi ? 2 : 0);
}

#define GRID_STRIDE(i, len) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (len); i += (int64_t)gridDim.x * blockDim.x)

// Forward, column side of iteration t: xhat, xbar (and the codes of a).
__global__ void kd_col_fwd(int64_t n, const int32_t* __restrict__ icol, const double* __restrict__ trace,
                           int64_t cap, const double* __restrict__ eta, double gamma, const DiffClock* __restrict__ clk, int32_t off,
                           const double* __restrict__ c, const double* __restrict__ lv,
                           const double* __restrict__ uv, const double* __restrict__ x,
                           const double* __restrict__ aty, double* __restrict__ xh, double* __restrict__ xbar,
                           uint8_t* __restrict__ code) {
  const int64_t t = clk->t0 + off;
  GRID_STRIDE(j, n) {
    const Sched s = sched_at(trace, cap, icol[j], t, eta, gamma);
    const double xj = x[j];
    const double a = fma(-s.tau, c[j] - aty[j], xj);
    const double lo = lv[j], hi = uv[j];
    const double h = clampd(a, lo, hi);
    xh[j] = h;
    xbar[j] = 2.0 * h - xj;
    if (code) code[j] = clamp_code(a, lo, hi);
  }
}

// Forward, row side of iteration t: yhat, the y update (Halpern or restart) and the codes of s.
__global__ void kd_row_fwd(int64_t m, const int32_t* __restrict__ irow, const double* __restrict__ trace,
                           int64_t cap, const double* __restrict__ eta, double gamma, const DiffClock* __restrict__ clk, int32_t off,
                           const double* __restrict__ lc, const double* __restrict__ uc,
                           const double* __restrict__ v, double* __restrict__ y, double* __restrict__ y0,
                           double* __restrict__ yh, uint8_t* __restrict__ code) {
  const int64_t t = clk->t0 + off;
  GRID_STRIDE(i, m) {
    const Sched s = sched_at(trace, cap, irow[i], t, eta, gamma);
    const double yi = y[i];
    const double sv = v[i] - yi / s.sigma;
    const double lo = lc[i], hi = uc[i];
    const double h = s.sigma * (clampd(sv, lo, hi) - sv);
    yh[i] = h;
    if (code) code[i] = clamp_code(sv, lo, hi);
    if (s.rho) {
      y[i] = h;
      y0[i] = h;
    } else {
      y[i] = s.al * h + s.be * yi + s.ep * y0[i];
    }
  }
}

// Forward: the x update of iteration t (after A xbar has been taken).
__global__ void kd_col_upd(int64_t n, const int32_t* __restrict__ icol, const double* __restrict__ trace,
                           int64_t cap, const double* __restrict__ eta, double gamma, const DiffClock* __restrict__ clk, int32_t off,
                           const double* __restrict__ xh, double* __restrict__ x, double* __restrict__ x0) {
  const int64_t t = clk->t0 + off;
  GRID_STRIDE(j, n) {
    const Sched s = sched_at(trace, cap, icol[j], t, eta, gamma);
    const double h = xh[j];
    if (s.rho) {
      x[j] = h;
      x0[j] = h;
    } else {
      x[j] = s.al * h + s.be * x[j] + s.ep * x0[j];
    }
  }
}

// Adjoint, row side of iteration t (first half): from (ly, ly0) of (y', y0') to lv = ls and the
// partial adjoints of (y, y0); accumulates the row-bound gradients.
__global__ void kd_row_bwd(int64_t m, const int32_t* __restrict__ irow, const double* __restrict__ trace,
                           int64_t cap, const double* __restrict__ eta, double gamma, const DiffClock* __restrict__ clk, int32_t off,
                           const uint8_t* __restrict__ code, const double* __restrict__ seed,
                           double* __restrict__ ly, double* __restrict__ ly0, double* __restrict__ lv,
                           double* __restrict__ glc, double* __restrict__ guc) {
  const int64_t t = clk->t0 + off;
  GRID_STRIDE(i, m) {
    const Sched s = sched_at(trace, cap, irow[i], t, eta, gamma);
    const double a_y = ly[i], a_y0 = ly0[i];
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
    if (seed && t == clk->K - 1) lyh += seed[i];
    const uint8_t cd = code[i];
    const double ls = cd == 0 ? 0.0 : -s.sigma * lyh;
    if (cd == 1) glc[i] += s.sigma * lyh;
    if (cd == 2) guc[i] += s.sigma * lyh;
    lv[i] = ls;
    ly[i] = lyp - ls / s.sigma;
    ly0[i] = ly0p;
  }
}

// Adjoint, column side of iteration t: from (lx, lx0) and lxbar = A^T lv to the adjoints of
// (x, x0) and laty = tau la; accumulates the gradients of c and the variable bounds.
__global__ void kd_col_bwd(int64_t n, const int32_t* __restrict__ icol, const double* __restrict__ trace,
                           int64_t cap, const double* __restrict__ eta, double gamma, const DiffClock* __restrict__ clk, int32_t off,
                           const uint8_t* __restrict__ code, const double* __restrict__ seed,
                           const double* __restrict__ lxbar, double* __restrict__ lx, double* __restrict__ lx0,
                           double* __restrict__ laty, double* __restrict__ gc, double* __restrict__ glv,
                           double* __restrict__ guv) {
  const int64_t t = clk->t0 + off;
  GRID_STRIDE(j, n) {
    const Sched s = sched_at(trace, cap, icol[j], t, eta, gamma);
    const double a_x = lx[j], a_x0 = lx0[j];
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
    if (seed && t == clk->K - 1) lxh += seed[j];
    const double lb = lxbar[j];
    lxh += 2.0 * lb;
    lxp -= lb;
    const uint8_t cd = code[j];
    const double la = cd == 0 ? lxh : 0.0;
    if (cd == 1) glv[j] += lxh;
    if (cd == 2) guv[j] += lxh;
    lxp += la;
    gc[j] -= s.tau * la;
    laty[j] = s.tau * la;
    lx[j] = lxp;
    lx0[j] = lx0p;
  }
}

__global__ void kd_add(int64_t len, double* __restrict__ dst, const double* __restrict__ src) {
  GRID_STRIDE(i, len) dst[i] += src[i];
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
  CK(get(&d->irow, m)); CK(get(&d->icol, n)); CK(get(&d->clk, 1));
  CK(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
  for (double** p : {&d->x, &d->x0, &d->xh, &d->xbar, &d->aty, &d->lx, &d->lx0, &d->lxbar, &d->laty, &d->sx,
                     &d->gc, &d->glv, &d->guv})
    CK(get(p, n));
  for (double** p : {&d->y, &d->y0, &d->yh, &d->v, &d->ly, &d->ly0, &d->lv, &d->ltmp, &d->sy, &d->glc, &d->guc})
    CK(get(p, m));
  kd_owner<<<h->gridS, kThreads, 0, h->setup_stream>>>(h->d_inst, h->count, d->irow, d->icol);
  CK(cudaGetLastError());
  if (!h->d_eta) {
    CK(h->alloc(&h->d_eta, h->count));
    CK(cudaMemcpy(h->d_eta, h->eta.data(), sizeof(double) * h->count, cudaMemcpyHostToDevice));
  }
  CK(cudaStreamSynchronize(h->setup_stream));
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

// One forward iteration (clock t0 + off) of every instance on the diff state.  code_x / code_y:
// where to store the clamp codes (NULL: not stored).
lp_status forward_step(lp_batch* h, int32_t off, uint8_t* code_x, uint8_t* code_y, cudaStream_t s) {
  Diff* d = h->diff;
  const int64_t n = h->sum_n, m = h->sum_m;
  const double g = h->prm.gamma;
  const int gA = grid_for(h->ntA, kWarps, 8 * h->num_sms), gT = grid_for(h->ntT, kWarps, 8 * h->num_sms);
  if (h->ntT > 0) kb_spmv<double><<<gT, kThreads, 0, s>>>(h->tasksT, h->ntT, h->rpT, h->ciT, h->valT, d->y, d->aty);
  if (n > 0)
    kd_col_fwd<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->trace, h->trace_cap, h->d_eta, g, d->clk, off, h->c, h->lv, h->uv,
                                           d->x, d->aty, d->xh, d->xbar, code_x);
  if (h->ntA > 0) kb_spmv<double><<<gA, kThreads, 0, s>>>(h->tasksA, h->ntA, h->rpA, h->ciA, h->valA, d->xbar, d->v);
  if (m > 0)
    kd_row_fwd<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->trace, h->trace_cap, h->d_eta, g, d->clk, off, h->lc, h->uc, d->v,
                                           d->y, d->y0, d->yh, code_y);
  if (n > 0)
    kd_col_upd<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->trace, h->trace_cap, h->d_eta, g, d->clk, off, d->xh, d->x, d->x0);
  CK(cudaGetLastError());
  return LP_OK;
}

// One adjoint iteration (clock t0 + off; codes of that iteration in code_x / code_y; the seeds
// enter at the map's last iteration).
lp_status backward_step(lp_batch* h, int32_t off, const uint8_t* code_x, const uint8_t* code_y, cudaStream_t s) {
  Diff* d = h->diff;
  const int64_t n = h->sum_n, m = h->sum_m;
  const double g = h->prm.gamma;
  const int gA = grid_for(h->ntA, kWarps, 8 * h->num_sms), gT = grid_for(h->ntT, kWarps, 8 * h->num_sms);
  if (m > 0)
    kd_row_bwd<<<vgrid(h, m), 256, 0, s>>>(m, d->irow, h->trace, h->trace_cap, h->d_eta, g, d->clk, off, code_y,
                                           d->sy, d->ly, d->ly0, d->lv, d->glc, d->guc);
  if (n > 0) {
    if (h->ntT > 0) kb_spmv<double><<<gT, kThreads, 0, s>>>(h->tasksT, h->ntT, h->rpT, h->ciT, h->valT, d->lv, d->lxbar);
    else CK(cudaMemsetAsync(d->lxbar, 0, sizeof(double) * n, s));
    kd_col_bwd<<<vgrid(h, n), 256, 0, s>>>(n, d->icol, h->trace, h->trace_cap, h->d_eta, g, d->clk, off, code_x,
                                           d->sx, d->lxbar, d->lx, d->lx0, d->laty, d->gc, d->glv,
                                           d->guv);
  }
  if (m > 0 && h->ntA > 0) {
    kb_spmv<double><<<gA, kThreads, 0, s>>>(h->tasksA, h->ntA, h->rpA, h->ciA, h->valA, d->laty, d->ltmp);
    kd_add<<<vgrid(h, m), 256, 0, s>>>(m, d->ly, d->ltmp);
  }
  CK(cudaGetLastError());
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

// The graph of one segment of len iterations (offsets 0..len-1 of the clock): kind 0 forward,
// 1 forward storing the clamp codes of offset o at codes + o (n + m), 2 the adjoint from offset
// len-1 down to 0.  Captured once per (kind, len, codes buffer) and replayed for every segment.
lp_status segment_graph(lp_batch* h, int kind, int64_t len, cudaGraphExec_t* out) {
  Diff* d = h->diff;
  const uint8_t* codes = kind == 0 ? nullptr : d->mx;
  if (d->seg[kind] && d->seg_len[kind] == len && d->seg_codes[kind] == codes) {
    *out = d->seg[kind];
    return LP_OK;
  }
  if (d->seg[kind]) {
    cudaGraphExecDestroy(d->seg[kind]);
    d->seg[kind] = nullptr;
  }
  const size_t n = (size_t)h->sum_n, m = (size_t)h->sum_m;
  uint8_t* cx = d->mx;
  uint8_t* cy = d->mx + (size_t)len * n;
  CK(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
  lp_status st = LP_OK;
  for (int64_t o = 0; o < len && st == LP_OK; ++o) {
    if (kind == 0) st = forward_step(h, (int32_t)o, nullptr, nullptr, d->cap);
    else if (kind == 1) st = forward_step(h, (int32_t)o, cx + o * n, cy + o * m, d->cap);
    else {
      const int64_t q = len - 1 - o;
      st = backward_step(h, (int32_t)q, cx + q * n, cy + q * m, d->cap);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(d->cap, &g);
  if (st != LP_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("segment capture: ") + cudaGetErrorString(e));
  const cudaError_t ei = cudaGraphInstantiate(&d->seg[kind], g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(LP_ERR_CUDA, std::string("segment instantiate: ") + cudaGetErrorString(ei));
  d->seg_len[kind] = len;
  d->seg_codes[kind] = codes;
  *out = d->seg[kind];
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
  // 1. the frozen schedule
  st = batch_schedule_solve(h, K, s);
  if (st != LP_OK) return st;
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
  cudaGraphExec_t gf = nullptr;
  if (K >= C) {
    st = segment_graph(h, 0, C, &gf);
    if (st != LP_OK) return st;
  }
  for (int64_t q = 0; q < nck; ++q) {
    const int64_t t0 = q * C, len = std::min(C, K - t0);
    st = save_ck(h, q, s);
    if (st != LP_OK) return st;
    kd_set_clock<<<1, 1, 0, s>>>(d->clk, t0, K);
    if (len == C) {
      CK(cudaGraphLaunch(gf, s));
    } else {
      for (int64_t o = 0; o < len && st == LP_OK; ++o) st = forward_step(h, (int32_t)o, nullptr, nullptr, s);
      if (st != LP_OK) return st;
    }
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
  cudaGraphExec_t grec = nullptr, gbwd = nullptr;
  if (K >= C) {
    st = segment_graph(h, 1, C, &grec);
    if (st == LP_OK) st = segment_graph(h, 2, C, &gbwd);
    if (st != LP_OK) return st;
  }
  for (int64_t q = (K + C - 1) / C - 1; q >= 0; --q) {
    const int64_t t0 = q * C, len = std::min(C, K - t0);
    st = load_ck(h, q, s);
    if (st != LP_OK) return st;
    kd_set_clock<<<1, 1, 0, s>>>(d->clk, t0, K);
    if (len == C) {
      CK(cudaGraphLaunch(grec, s));
      CK(cudaGraphLaunch(gbwd, s));
      continue;
    }
    // a shorter last segment: its codes are laid out for its own length
    uint8_t* lx_codes = d->mx;
    uint8_t* ly_codes = d->mx + (size_t)len * n;
    for (int64_t o = 0; o < len && st == LP_OK; ++o)
      st = forward_step(h, (int32_t)o, lx_codes + (size_t)o * n, ly_codes + (size_t)o * m, s);
    for (int64_t o = len - 1; o >= 0 && st == LP_OK; --o)
      st = backward_step(h, (int32_t)o, lx_codes + (size_t)o * n, ly_codes + (size_t)o * m, s);
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

}  // extern "C"
