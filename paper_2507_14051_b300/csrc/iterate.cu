// Iteration kernels of restarted reflected-Halpern PDHG (cuPDLPx, arXiv 2507.14051).
//
// One iteration t is two streaming kernels, each fused with its epilogue and closed by the
// block that finishes last (a deterministic fixed-order reduction plus the scalar control):
//
//   K1 (rows of A, gathers xhat_t):
//     deferred Halpern update of the y side decided at t-1 (Section 3, reflected Halpern):
//       y  <- ha*yhat + hb*y + he*y0,  Ax <- ha*Axhat + hb*Ax + he*Ax0   (or <- yhat, Axhat
//       at a restart, which also resets the anchors);
//     v = A xhat_t; A xbar = 2v - Ax (xbar = 2xhat - x);
//     dual step of eq. (pdhg), Section 2.2, in the form yhat = sigma (proj_S(s) - s),
//       s = A xbar - y/sigma;
//     sums |y - yhat|^2, (y - yhat)^T (Ax - Axhat), |yhat - y0|^2 and, on check iterations,
//       the primal residual and the y part of the dual objective (Section 4);
//     last block: fixed-point residual r_t = ||z - T z||_P (Section 2.2 P, Section 3),
//       restart test (Section 3, three conditions), PID update of omega (Section 3).
//   K2 (rows of A^T, gathers yhat_t):
//     u = A^T yhat_t; x side of the Halpern update (decided by K1 of this iteration), the
//       maintained A^T y likewise; next primal step (eq. pdhg first line)
//       xhat_{t+1} = proj_X(x - tau (c - A^T y));
//     sums |x - xhat_{t+1}|^2, |xhat_{t+1} - x0|^2 and, on check iterations, c^T xhat_t, the
//       dual residual and the r part of the dual objective (Section 4);
//     last block: relative KKT test (Section 4) -> done / status.
//
// A x and A^T y of the current iterate are maintained by the same affine updates as x and y
// (exact in exact arithmetic; refreshed from true products at every restart), so one SpMV
// per side per iteration suffices.
#include "kernels.cuh"

namespace pdhg {

__device__ __forceinline__ bool is_check(const Ctl* ctl, int64_t t) {
  return ((t + 1) % ctl->check_every) == 0 || (t + 1 == ctl->max_iter);
}

// Restart test, Section 3: (1) r <= b_s r0; (2) r <= b_n r0 and r > r_prev; (3) k >= b_a T.
__device__ __forceinline__ int restart_test(const Ctl* ctl, int64_t k, int64_t t, double r) {
  if (k < 1) return 0;
  if (r <= ctl->beta_s * ctl->r0) return 1;
  if (r <= ctl->beta_n * ctl->r0 && r > ctl->r_prev) return 1;
  if ((double)k >= ctl->beta_a * (double)(t + 1)) return 1;
  return 0;
}

// PID primal weight update, Section 3: e = log(sqrt(w)|dx| / (|dy|/sqrt(w))),
// log w <- log w - (K_P e + K_I sum e + K_D (e - e_prev)); skipped when a norm is 0 or not
// finite; log w kept in [-23, 23].
__device__ __forceinline__ double pid_update(Ctl* ctl, double omega, double dxn, double dyn) {
  if (!(dxn > 0.0) || !(dyn > 0.0) || !isfinite(dxn) || !isfinite(dyn)) return omega;
  const double sw = sqrt(omega);
  const double e = log((sw * dxn) / (dyn / sw));
  ctl->pid_integral += e;
  const double de = ctl->pid_has_prev ? e - ctl->pid_eprev : 0.0;
  double lw = log(omega) - (ctl->kp * e + ctl->ki * ctl->pid_integral + ctl->kd * de);
  lw = fmin(fmax(lw, -23.0), 23.0);
  ctl->pid_eprev = e;
  ctl->pid_has_prev = 1;
  return exp(lw);
}

__global__ void __launch_bounds__(kThreads, 3) k1_rows(RowArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->done) return;
  const int64_t t = ctl->t;
  const bool check = is_check(ctl, t);
  const double* __restrict__ xh = (t & 1) ? a.xh1 : a.xh0;
  const int mode = (t == 0) ? 2 : ctl->restart;  // 0 combine, 1 restart, 2 first iteration
  const double ha = ctl->ha, hb = ctl->hb, he = ctl->he;
  const double sigma = ctl->sigma, inv_sigma = ctl->inv_sigma;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row(a.bins, a.rp, a.ci, a.val, xh, pol, s, [&](int i, double v, double (&acc)[kNumSums]) {
    double yi, axi, y0i;
    if (mode == 0) {
      y0i = a.y0[i];
      yi = fma(ha, a.yh[i], fma(hb, a.y[i], he * y0i));
      axi = fma(ha, a.axh[i], fma(hb, a.ax[i], he * a.ax0[i]));
    } else if (mode == 1) {
      yi = a.yh[i];
      axi = a.axh[i];
      y0i = yi;
      a.y0[i] = yi;
      a.ax0[i] = axi;
    } else {
      yi = 0.0;
      axi = 0.0;
      y0i = 0.0;
    }
    const double lo = a.lc[i], hi = a.uc[i];
    const double w = fma(2.0, v, -axi);  // A(2 xhat - x)
    const double sv = fma(-yi, inv_sigma, w);
    const double yn = sigma * (clampd(sv, lo, hi) - sv);
    const double dy = yi - yn;
    acc[0] = fma(dy, dy, acc[0]);
    acc[1] = fma(dy, axi - v, acc[1]);
    const double d0 = yn - y0i;
    acc[2] = fma(d0, d0, acc[2]);
    if (check) {
      const double pr = (v - clampd(v, lo, hi)) * a.inv_dr[i];
      acc[3] = fma(pr, pr, acc[3]);
      acc[4] += (yn > 0.0 ? lo * yn : 0.0) + (yn < 0.0 ? hi * yn : 0.0);
    }
    if (mode != 2) {
      a.y[i] = yi;
      a.ax[i] = axi;
    }
    a.yh[i] = yn;
    a.axh[i] = v;
  });
  const int nsums = check ? 5 : 3;
  if (!block_sums_last(s, nsums, a.partials, &ctl->count1)) return;
  double tot[kNumSums];
  block_totals(a.partials, gridDim.x, nsums, &a.bins, tot);
  if (threadIdx.x != 0) return;

  // ---- scalar control (one thread) ----
  const double eta = ctl->eta, om = ctl->omega;
  const double r2 = fma(ctl->w_over_eta, ctl->sxx, fma(ctl->inv_eta_w, tot[0], 2.0 * tot[1]));
  const double r = sqrt(r2 > 0.0 ? r2 : 0.0);
  const int64_t k = ctl->k;
  if (k == 0) ctl->r0 = r;
  if (check) {
    ctl->pres2 = tot[3];
    ctl->dobj_y = tot[4];
  }
  ctl->omega_used = om;
  ctl->restarts_used = ctl->restarts;
  const bool tr = a.trace != nullptr && t < ctl->trace_cap;
  if (tr) {
    a.trace[4 * t + 0] = r;
    a.trace[4 * t + 1] = om;
    a.trace[4 * t + 2] = 0.0;
    a.trace[4 * t + 3] = (double)k;
  }
  ctl->count1 = 0;
  if (!isfinite(r2)) {
    ctl->status = kNumerical;
    ctl->iters = t + 1;
    ctl->done = 1;
    return;
  }
  const int rs = ctl->restart_enabled && (t + 1 < ctl->max_iter) ? restart_test(ctl, k, t, r) : 0;
  if (rs) {
    double omn = om;
    if (ctl->pid_enabled) omn = pid_update(ctl, om, sqrt(ctl->sx0), sqrt(tot[2]));
    ctl->omega = omn;
    ctl->tau = eta / omn;
    ctl->sigma = eta * omn;
    ctl->inv_sigma = 1.0 / (eta * omn);
    ctl->w_over_eta = omn / eta;
    ctl->inv_eta_w = 1.0 / (eta * omn);
    ctl->k = 0;
    ctl->restarts += 1;
    if (tr) a.trace[4 * t + 2] = 1.0;
  } else {
    const double kk = (double)k;
    const double aw = (kk + 1.0) / (kk + 2.0);
    ctl->ha = aw * (1.0 + ctl->gamma);
    ctl->hb = -aw * ctl->gamma;
    ctl->he = 1.0 / (kk + 2.0);
    ctl->r_prev = r;
    ctl->k = k + 1;
  }
  ctl->restart = rs;
}

__global__ void __launch_bounds__(kThreads, 3) k2_cols(ColArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->done) return;
  const int64_t t = ctl->t;
  const bool check = is_check(ctl, t);
  const double* __restrict__ xc_buf = (t & 1) ? a.xh1 : a.xh0;
  double* __restrict__ xn_buf = (t & 1) ? a.xh0 : a.xh1;
  const int restart = ctl->restart;
  const double ha = ctl->ha, hb = ctl->hb, he = ctl->he, tau = ctl->tau;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row(a.bins, a.rp, a.ci, a.val, a.yh, pol, s, [&](int j, double u, double (&acc)[kNumSums]) {
    const double xc = xc_buf[j];
    double xj, atyj, x0j;
    if (restart) {
      xj = xc;
      atyj = u;
      x0j = xc;
      a.x0[j] = xc;
      a.aty0[j] = u;
    } else {
      x0j = a.x0[j];
      xj = fma(ha, xc, fma(hb, a.x[j], he * x0j));
      atyj = fma(ha, u, fma(hb, a.aty[j], he * a.aty0[j]));
    }
    const double cj = a.c[j], lo = a.lv[j], hi = a.uv[j];
    const double xn = clampd(fma(-tau, cj - atyj, xj), lo, hi);
    const double dx = xj - xn;
    acc[0] = fma(dx, dx, acc[0]);
    const double d0 = xn - x0j;
    acc[1] = fma(d0, d0, acc[1]);
    if (check) {
      acc[2] = fma(cj, xc, acc[2]);
      const double rc = cj - u;
      const bool fl = isfinite(lo), fu = isfinite(hi);
      const double rr = (fl && fu) ? rc : (fl ? fmax(rc, 0.0) : (fu ? fmin(rc, 0.0) : 0.0));
      const double dd = (rc - rr) * a.inv_dc[j];
      acc[3] = fma(dd, dd, acc[3]);
      acc[4] += (rr > 0.0 ? lo * rr : 0.0) + (rr < 0.0 ? hi * rr : 0.0);
    }
    a.x[j] = xj;
    a.aty[j] = atyj;
    xn_buf[j] = xn;
  });
  const int nsums = check ? 5 : 2;
  if (!block_sums_last(s, nsums, a.partials, &ctl->count2)) return;
  double tot[kNumSums];
  block_totals(a.partials, gridDim.x, nsums, &a.bins, tot);
  if (threadIdx.x != 0) return;

  ctl->sxx = tot[0];
  ctl->sx0 = tot[1];
  ctl->count2 = 0;
  if (check) {
    const double pobj = tot[2], dobj = ctl->dobj_y + tot[4];
    const double pres = sqrt(ctl->pres2), dres = sqrt(tot[3]);
    const double rg = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    const double rp = pres / (1.0 + ctl->lu_norm);
    const double rd = dres / (1.0 + ctl->c_norm);
    double mx = rg;
    if (!(rp <= mx)) mx = rp;
    if (!(rd <= mx)) mx = rd;
    ctl->kkt[0] = rg;
    ctl->kkt[1] = rp;
    ctl->kkt[2] = rd;
    ctl->kkt[3] = mx;
    ctl->kkt[4] = pobj;
    ctl->kkt[5] = dobj;
    ctl->kkt[6] = pres;
    ctl->kkt[7] = dres;
    if (rg <= ctl->tol && rp <= ctl->tol && rd <= ctl->tol) {
      ctl->status = kOptimal;
      ctl->iters = t + 1;
      ctl->done = 1;
      return;
    }
  }
  if (t + 1 >= ctl->max_iter) {
    ctl->status = kIterLimit;
    ctl->iters = t + 1;
    ctl->done = 1;
    return;
  }
  ctl->t = t + 1;
}

// Installs the scalar state of a new solve (built on the host, passed by value so that
// back-to-back solves on one stream cannot race on a host staging buffer).
__global__ void k_init_ctl(Ctl* dst, Ctl src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = src;
}

// First primal step from z = 0: xhat_0 = proj_X(-tau c); zeroes the iterate, the anchors and
// the maintained products; sums |0 - xhat_0|^2 and |xhat_0 - 0|^2 for r_0.
__global__ void __launch_bounds__(kThreads) k_init_cols(int32_t n, const double* __restrict__ c,
                                                        const double* __restrict__ lv,
                                                        const double* __restrict__ uv,
                                                        double* xh0, double* x, double* x0,
                                                        double* aty, double* aty0, Ctl* ctl,
                                                        double* partials) {
  const double tau = ctl->tau;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double xn = clampd(-tau * c[j], lv[j], uv[j]);
    xh0[j] = xn;
    x[j] = 0.0;
    x0[j] = 0.0;
    aty[j] = 0.0;
    aty0[j] = 0.0;
    s[0] = fma(xn, xn, s[0]);
  }
  if (!block_sums_last(s, 1, partials, &ctl->count0)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, nullptr, tot);
  if (threadIdx.x != 0) return;
  ctl->sxx = tot[0];
  ctl->sx0 = tot[0];
  ctl->count0 = 0;
}

__global__ void k_init_rows(int32_t m, double* y, double* y0, double* yh, double* ax, double* ax0,
                            double* axh) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    y[i] = 0.0;
    y0[i] = 0.0;
    yh[i] = 0.0;
    ax[i] = 0.0;
    ax0[i] = 0.0;
    axh[i] = 0.0;
  }
}

// Sets the device-side loop condition: keep iterating while the solve is not done.  Guard:
// each body performs at most `unroll` iterations, so more than max_iter/unroll + 2 bodies
// means the control logic failed to finish the solve; stop with an internal-error status
// instead of looping.
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

}  // namespace pdhg
