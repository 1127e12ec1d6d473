// Device functions of one PDHG iteration, shared by the single-instance kernels (iterate.cu)
// and the batched loop (batch.cu): the row-phase and column-phase epilogues, the scalar
// control after each phase (restart test and PID, Section 3; relative KKT test, Section 4) and
// the mixed-precision hand-over of the scalar state.
#pragma once
#include "kernels.cuh"

namespace pdhg {

__device__ __forceinline__ bool is_check(const Ctl& c, int64_t t) {
  return ((t + 1) % c.check_every) == 0 || (t + 1 == c.max_iter);
}

// Restart test, Section 3: (1) r <= b_s r0; (2) r <= b_n r0 and r > r_prev; (3) k >= b_a T.
// Taken on squared residuals (r, r0, r_prev >= 0, so r <= b r0 <=> r^2 <= b^2 r0^2): r2 = r^2,
// and c.r0, c.r_prev hold r0^2 and r_prev^2.  An FP64 square root is a ~900-cycle dependent
// chain on this GPU, on the serial control path of every iteration; the squares need none.
__device__ __forceinline__ int restart_test(const Ctl& c, int64_t k, int64_t t, double r2) {
  if (k < 1) return 0;
  const double bs2 = c.beta_s * c.beta_s, bn2 = c.beta_n * c.beta_n;  // independent of r2
  if (r2 <= bs2 * c.r0) return 1;
  if (r2 <= bn2 * c.r0 && r2 > c.r_prev) return 1;
  if ((double)k >= c.beta_a * (double)(t + 1)) return 1;
  return 0;
}

// What the restart test takes from the state before the totals are known, computed off the
// control's serial path (by a warp that waits for the totals anyway): the thresholds
// beta_s^2 r0^2 and beta_n^2 r0^2 (c.r0 holds r0^2), r_{t-1}^2, the artificial condition
// k >= beta_a (t + 1), and whether restarts are allowed at t.  restart_test_pre with them
// decides as restart_test does, bit for bit.
struct RestartPre {
  double thr_s, thr_n, r_prev;
  int art, allow;
};
__device__ __forceinline__ RestartPre restart_pre(const Ctl& c) {
  RestartPre p;
  p.thr_s = (c.beta_s * c.beta_s) * c.r0;
  p.thr_n = (c.beta_n * c.beta_n) * c.r0;
  p.r_prev = c.r_prev;
  p.art = (double)c.k >= c.beta_a * (double)(c.t + 1) ? 1 : 0;
  p.allow = (c.restart_enabled && c.t + 1 < c.max_iter) ? 1 : 0;
  return p;
}
__device__ __forceinline__ int restart_test_pre(const RestartPre& p, int64_t k, double r2) {
  if (k < 1) return 0;
  if (r2 <= p.thr_s) return 1;
  if (r2 <= p.thr_n && r2 > p.r_prev) return 1;
  return p.art;
}

// PID primal weight update, Section 3: e = log(sqrt(w)|dx| / (|dy|/sqrt(w))),
// log w <- log w - (K_P e + K_I sum e + K_D (e - e_prev)); skipped when a norm is 0 or not
// finite; log w kept in [-23, 23].
__device__ __forceinline__ double pid_update(Ctl& c, double omega, double dxn, double dyn) {
  if (!(dxn > 0.0) || !(dyn > 0.0) || !isfinite(dxn) || !isfinite(dyn)) return omega;
  const double sw = sqrt(omega);
  const double e = log((sw * dxn) / (dyn / sw));
  c.pid_integral += e;
  const double de = c.pid_has_prev ? e - c.pid_eprev : 0.0;
  double lw = log(omega) - (c.kp * e + c.ki * c.pid_integral + c.kd * de);
  lw = fmin(fmax(lw, -23.0), 23.0);
  c.pid_eprev = e;
  c.pid_has_prev = 1;
  return exp(lw);
}

// FP64 accumulation of a product / value computed in the phase's value type: for FP64 the
// product is fused into the accumulator, for FP32 the product is rounded to FP32 and added in
// FP64 (the reductions stay FP64 in both precisions).
__device__ __forceinline__ void acc_fma(double& a, double p, double q) { a = fma(p, q, a); }
__device__ __forceinline__ void acc_fma(double& a, float p, float q) { a += (double)(p * q); }
__device__ __forceinline__ double fmav(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double maxv(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float maxv(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double minv(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float minv(float a, float b) { return fminf(a, b); }

// ------------------------------------------------------------------ row phase

struct RowStep {
  int mode;  // 0 Halpern combine, 1 restart, 2 first iteration (state is zero)
  int check;
  int cand;  // stall-guard slot written at this check iteration
  double ha, hb, he, sigma, inv_sigma;
};

__device__ __forceinline__ RowStep row_step(const Ctl& c) {
  RowStep st;
  st.mode = (c.t == 0) ? 2 : c.restart;
  st.check = is_check(c, c.t) ? 1 : 0;
  st.cand = c.cand_slot;
  st.ha = c.ha;
  st.hb = c.hb;
  st.he = c.he;
  st.sigma = c.sigma;
  st.inv_sigma = c.inv_sigma;
  return st;
}

// Operands of the row epilogue that depend only on the row: loaded before the row's SpMV so
// that their latency overlaps it.
template <class V>
struct RowIn {
  V y0, yh, y, axh, ax, ax0, lo, hi;
};

template <class V>
__device__ __forceinline__ RowIn<V> row_load(const RowArgsT<V>& a, const RowStep& st, int i) {
  RowIn<V> in;
  if (st.mode == 0) {
    in.y0 = a.y0[i];
    in.yh = a.yh[i];
    in.y = a.y[i];
    in.axh = a.axh[i];
    in.ax = a.ax[i];
    in.ax0 = a.ax0[i];
  } else if (st.mode == 1) {
    in.yh = a.yh[i];
    in.axh = a.axh[i];
    in.y0 = in.y = in.ax = in.ax0 = V(0);
  } else {
    in.y0 = in.yh = in.y = in.axh = in.ax = in.ax0 = V(0);
  }
  in.lo = a.lc[i];
  in.hi = a.uc[i];
  return in;
}

// kPidSums: also accumulate |yhat - y0|^2 (slot 2), which only the PID update at a restart
// reads; a driver that evaluates it only when a restart happens passes false (slot 2 stays 0).
template <class V, bool kPidSums = true>
__device__ __forceinline__ void row_finish(const RowArgsT<V>& a, const RowStep& st, int i, V v,
                                           const RowIn<V>& in, double (&acc)[kNumSums]) {
  const V ha = (V)st.ha, hb = (V)st.hb, he = (V)st.he;
  const V sigma = (V)st.sigma, inv_sigma = (V)st.inv_sigma;
  V yi, axi, y0i;
  if (st.mode == 0) {
    y0i = in.y0;
    yi = fmav(ha, in.yh, fmav(hb, in.y, he * y0i));
    axi = fmav(ha, in.axh, fmav(hb, in.ax, he * in.ax0));
  } else if (st.mode == 1) {
    yi = in.yh;
    axi = in.axh;
    y0i = yi;
    a.y0[i] = yi;
    a.ax0[i] = axi;
  } else {
    yi = V(0);
    axi = V(0);
    y0i = V(0);
  }
  const V lo = in.lo, hi = in.hi;
  const V w = fmav(V(2), v, -axi);  // A(2 xhat - x)
  const V sv = fmav(-yi, inv_sigma, w);
  const V yn = sigma * (clampd(sv, lo, hi) - sv);
  const V dy = yi - yn;
  acc_fma(acc[0], dy, dy);
  acc_fma(acc[1], dy, axi - v);
  if (kPidSums) {
    const V d0 = yn - y0i;
    acc_fma(acc[2], d0, d0);
  }
  if (st.check) {
    const V pr = (v - clampd(v, lo, hi)) * a.inv_dr[i];
    acc_fma(acc[3], pr, pr);
    acc[4] += (double)((yn > V(0) ? lo * yn : V(0)) + (yn < V(0) ? hi * yn : V(0)));
    if (a.yb0) (st.cand ? a.yb1 : a.yb0)[i] = yn;
  }
  if (st.mode != 2) {
    a.y[i] = yi;
    a.ax[i] = axi;
  }
  a.yh[i] = yn;
  a.axh[i] = v;
}

template <class V, bool kPidSums = true>
__device__ __forceinline__ void row_epilogue(const RowArgsT<V>& a, const RowStep& st, int i, V v,
                                             double (&acc)[kNumSums]) {
  row_finish<V, kPidSums>(a, st, i, v, row_load(a, st, i), acc);
}

// Issued before the row's SpMV: brings the row epilogue's operands to L1 while the SpMV runs,
// without holding registers across it.
template <class V>
__device__ __forceinline__ void row_prefetch(const RowArgsT<V>& a, const RowStep& st, int i) {
  if (st.mode == 0) {
    prefetch_l1(a.y0 + i);
    prefetch_l1(a.y + i);
    prefetch_l1(a.ax + i);
    prefetch_l1(a.ax0 + i);
  }
  if (st.mode != 2) {
    prefetch_l1(a.yh + i);
    prefetch_l1(a.axh + i);
  }
  prefetch_l1(a.lc + i);
  prefetch_l1(a.uc + i);
}

// Reflected Halpern weights of epoch step k + 1 (Section 3): x' = ha xhat + hb x + he x0 with
// ha = (k+1)/(k+2) (1 + gamma), hb = -(k+1)/(k+2) gamma, he = 1/(k+2).
struct Halpern {
  double ha, hb, he;
};
__device__ __forceinline__ Halpern halpern_weights(int64_t k, double gamma) {
  const double kk = (double)k;
  const double aw = (kk + 1.0) / (kk + 2.0);
  Halpern h;
  h.ha = aw * (1.0 + gamma);
  h.hb = -aw * gamma;
  h.he = 1.0 / (kk + 2.0);
  return h;
}

// Scalar control after the row phase of iteration c.t, on totals tot[0..2] (and tot[3..4] on
// check iterations).  Writes the trace row if `trace` is given.  `next` (or NULL): the weights
// halpern_weights(c.k, c.gamma), computed beforehand off this serial path.
// row_decide does all of it but the new primal weight of a restart, and returns the restart flag
// (1), 0, or -1 once the solve has ended (NUMERICAL); row_restart_weight then applies the PID
// update (Section 3) from the squared norms |xhat - x0|^2 and |yhat - y0|^2 of the epoch.
// `cross` scales the summed cross term tot[1]: 2 when it sums (y - yhat)(A x - A xhat) (the
// plain epilogues), 1 when it sums (y - yhat)(A x - A xbar), which is twice that (the reflected
// form, xbar = 2 xhat - x).
// pre (or NULL): restart_pre(c) taken before this call, off the serial path.
__device__ __forceinline__ int row_decide(Ctl& c, const double (&tot)[kNumSums], bool check, double* trace,
                                          const Halpern* next = nullptr, double cross = 2.0,
                                          const RestartPre* pre = nullptr) {
  const int64_t t = c.t;
  const double om = c.omega;
  const double r2raw = fma(c.w_over_eta, c.sxx, fma(c.inv_eta_w, tot[0], cross * tot[1]));
  const double r2 = r2raw > 0.0 ? r2raw : 0.0;  // r_t^2 (the test and the state use squares)
  const int64_t k = c.k;
  if (k == 0) c.r0 = r2;
  if (check) {
    c.pres2 = tot[3];
    c.dobj_y = tot[4];
  }
  c.omega_used = om;
  c.restarts_used = c.restarts;
  const bool tr = trace != nullptr && t < c.trace_cap;
  if (tr) {
    trace[4 * t + 0] = sqrt(r2);
    trace[4 * t + 1] = om;
    trace[4 * t + 2] = 0.0;
    trace[4 * t + 3] = (double)k;
  }
  if (!isfinite(r2raw)) {
    c.status = kNumerical;
    c.iters = t + 1;
    c.done = 1;
    return -1;
  }
  const int rs = pre ? (pre->allow ? restart_test_pre(*pre, k, r2) : 0)
                     : (c.restart_enabled && (t + 1 < c.max_iter) ? restart_test(c, k, t, r2) : 0);
  if (rs) {
    c.k = 0;
    c.restarts += 1;
    if (tr) trace[4 * t + 2] = 1.0;
  } else {
    const Halpern h = next ? *next : halpern_weights(k, c.gamma);
    c.ha = h.ha;
    c.hb = h.hb;
    c.he = h.he;
    c.r_prev = r2;
    c.k = k + 1;
  }
  c.restart = rs;
  return rs;
}

__device__ __forceinline__ void row_restart_weight(Ctl& c, double dx2, double dy2) {
  const double eta = c.eta, om = c.omega;
  double omn = om;
  if (c.pid_enabled) omn = pid_update(c, om, sqrt(dx2), sqrt(dy2));
  c.omega = omn;
  c.tau = eta / omn;
  c.sigma = eta * omn;
  c.inv_sigma = 1.0 / (eta * omn);
  c.w_over_eta = omn / eta;
  c.inv_eta_w = 1.0 / (eta * omn);
}

// Scalar control after the row phase with the PID norms accumulated in the phase (c.sx0 from the
// last column phase, tot[2] from this row phase).
__device__ __forceinline__ void row_control(Ctl& c, const double (&tot)[kNumSums], bool check,
                                            double* trace, const Halpern* next = nullptr) {
  if (row_decide(c, tot, check, trace, next) == 1) row_restart_weight(c, c.sx0, tot[2]);
}

// --------------------------------------------------------------- column phase

template <class V>
struct ColStepT {
  int restart;
  int check;
  int cand;
  double ha, hb, he, tau;
  const V* xc;  // xhat_t
  V* xn;        // xhat_{t+1}
};

template <class V>
__device__ __forceinline__ ColStepT<V> col_step(const Ctl& c, const ColArgsT<V>& a) {
  ColStepT<V> st;
  st.restart = c.restart;
  st.check = is_check(c, c.t) ? 1 : 0;
  st.cand = c.cand_slot;
  st.ha = c.ha;
  st.hb = c.hb;
  st.he = c.he;
  st.tau = c.tau;
  st.xc = (c.t & 1) ? a.xh1 : a.xh0;
  st.xn = (c.t & 1) ? a.xh0 : a.xh1;
  return st;
}

template <class V>
struct ColIn {
  V xc, x0, x, aty, aty0, c, lo, hi;
};

template <class V>
__device__ __forceinline__ ColIn<V> col_load(const ColArgsT<V>& a, const ColStepT<V>& st, int j) {
  ColIn<V> in;
  in.xc = st.xc[j];
  if (st.restart) {
    in.x0 = in.x = in.aty = in.aty0 = V(0);
  } else {
    in.x0 = a.x0[j];
    in.x = a.x[j];
    in.aty = a.aty[j];
    in.aty0 = a.aty0[j];
  }
  in.c = a.c[j];
  in.lo = a.lv[j];
  in.hi = a.uv[j];
  return in;
}

// kPidSums: also accumulate |xhat' - x0|^2 (slot 1), which only the PID update at a restart reads
// (as c.sx0); with false slot 1 stays 0.
template <class V, bool kPidSums = true>
__device__ __forceinline__ void col_finish(const ColArgsT<V>& a, const ColStepT<V>& st, int j, V u,
                                           const ColIn<V>& in, double (&acc)[kNumSums]) {
  const V ha = (V)st.ha, hb = (V)st.hb, he = (V)st.he, tau = (V)st.tau;
  const V xc = in.xc;
  V xj, atyj, x0j;
  if (st.restart) {
    xj = xc;
    atyj = u;
    x0j = xc;
    a.x0[j] = xc;
    a.aty0[j] = u;
  } else {
    x0j = in.x0;
    xj = fmav(ha, xc, fmav(hb, in.x, he * x0j));
    atyj = fmav(ha, u, fmav(hb, in.aty, he * in.aty0));
  }
  const V cj = in.c, lo = in.lo, hi = in.hi;
  const V xn = clampd(fmav(-tau, cj - atyj, xj), lo, hi);
  const V dx = xj - xn;
  acc_fma(acc[0], dx, dx);
  if (kPidSums) {
    const V d0 = xn - x0j;
    acc_fma(acc[1], d0, d0);
  }
  if (st.check) {
    acc_fma(acc[2], cj, xc);
    const V rc = cj - u;
    const bool fl = isfinite(lo), fu = isfinite(hi);
    const V rr = (fl && fu) ? rc : (fl ? maxv(rc, V(0)) : (fu ? minv(rc, V(0)) : V(0)));
    const V dd = (rc - rr) * a.inv_dc[j];
    acc_fma(acc[3], dd, dd);
    acc[4] += (double)((rr > V(0) ? lo * rr : V(0)) + (rr < V(0) ? hi * rr : V(0)));
    if (a.xb0) (st.cand ? a.xb1 : a.xb0)[j] = xc;
  }
  a.x[j] = xj;
  a.aty[j] = atyj;
  st.xn[j] = xn;
}

template <class V, bool kPidSums = true>
__device__ __forceinline__ void col_epilogue(const ColArgsT<V>& a, const ColStepT<V>& st, int j, V u,
                                             double (&acc)[kNumSums]) {
  col_finish<V, kPidSums>(a, st, j, u, col_load(a, st, j), acc);
}

template <class V>
__device__ __forceinline__ void col_prefetch(const ColArgsT<V>& a, const ColStepT<V>& st, int j) {
  prefetch_l1(st.xc + j);
  if (!st.restart) {
    prefetch_l1(a.x0 + j);
    prefetch_l1(a.x + j);
    prefetch_l1(a.aty + j);
    prefetch_l1(a.aty0 + j);
  }
  prefetch_l1(a.c + j);
  prefetch_l1(a.lv + j);
  prefetch_l1(a.uv + j);
}

// ------------------------------------------------ reflected form (gamma = 1)
//
// With gamma = 1 the reflected Halpern step of Section 3 is z' = lam (2 zhat - z) + mu z0,
// lam = (k+1)/(k+2), mu = 1/(k+2): the reflected point 2 zhat - z is the same xbar = 2 xhat - x
// that the dual step of eq. (pdhg) evaluates A at.  The loop kernel's reflected form keeps the
// reflected points instead of the iterates:
//   row phase t:    gathers xbar_t, so its SpMV gives w_t = A xbar_t directly; the iterate
//                   y_t = lam qy_{t-1} + mu y0 and A x_t = lam w_{t-1} + mu A x0 (after a
//                   restart: yhat_{t-1} and A xhat_{t-1}); stores yhat_t, qy_t = 2 yhat_t - y_t
//                   and w_t;
//   column phase t: gathers qy_t (after a restart decision: yhat_t), so its SpMV gives
//                   A^T qy_t and A^T y_{t+1} = lam A^T qy_t + mu A^T y0 directly; the iterate
//                   x_{t+1} = lam xbar_t + mu x0 (after a restart: xhat_t); stores xhat_{t+1}
//                   and xbar_{t+1} = 2 xhat_{t+1} - x_{t+1}.
// Nothing else is carried between iterations, so each side reads and writes three vectors
// fewer than the plain form and spends fewer FP64 operations per entry (12 per row, 9 per
// column).  The products the plain form has at hand are computed where they are needed, by an
// SpMV of their own (the exact products, as in the plain form):
//   A xhat_t before the row phase of a check iteration (the primal residual; stored in ax);
//   A^T yhat_t before the column phase of a check iteration that does not restart (the dual
//     residual; stored in aty; after a restart decision the phase's own SpMV gives it);
//   A xhat_t at a restart (the next row phase's A x and anchor product; stored in axh).
// The maintained A x and A^T y of the reflected form carry the Halpern recursion's rounding
// through an epoch, so averages such as (w_t + A x_t) / 2 would move the KKT test's residuals,
// which near the tolerance are differences of nearly equal products, by up to 1e-3 relative.
// The fixed-point residual's cross term is summed as (y - yhat)(A x - w) = 2 (y - yhat) A (x - xhat).

// The scalars in the iterates' type (rounded once per block and iteration, not per row).
template <class V>
struct RowStepR {
  int mode;  // 0 Halpern combine, 1 restart, 2 first iteration (state is zero)
  int check;
  int cand;
  V lam, mu, sigma, inv_sigma;
};

// check: whether iteration c.t is a check iteration, if the caller has it (-1: computed here;
// the test takes a 64-bit remainder, a long chain on the serial control path).
template <class V>
__device__ __forceinline__ RowStepR<V> row_step_r(const Ctl& c, int check = -1) {
  RowStepR<V> st;
  st.mode = (c.t == 0) ? 2 : c.restart;
  st.check = check >= 0 ? check : (is_check(c, c.t) ? 1 : 0);
  st.cand = c.cand_slot;
  st.lam = (V)(-c.hb);  // gamma = 1: hb = -lam
  st.mu = (V)c.he;
  st.sigma = (V)c.sigma;
  st.inv_sigma = (V)c.inv_sigma;
  return st;
}

template <class V>
__device__ __forceinline__ void row_prefetch_r(const RowArgsT<V>& a, const RowStepR<V>& st, int i) {
  if (st.mode == 0) {
    prefetch_l1(a.qy + i);
    prefetch_l1(a.y0 + i);
    prefetch_l1(a.w + i);
    prefetch_l1(a.ax0 + i);
  } else if (st.mode == 1) {
    prefetch_l1(a.yh + i);
    prefetch_l1(a.axh + i);
  }
  prefetch_l1(a.lc + i);
  prefetch_l1(a.uc + i);
}

// Row epilogue of the reflected form: wv = A xbar_t of row i.
template <class V>
__device__ __forceinline__ void row_epilogue_r(const RowArgsT<V>& a, const RowStepR<V>& st, int i, V wv,
                                               double (&acc)[kNumSums]) {
  const V sigma = st.sigma, inv_sigma = st.inv_sigma;
  V yi, axi;
  if (st.mode == 0) {
    const V lam = st.lam, mu = st.mu;
    yi = fmav(lam, a.qy[i], mu * a.y0[i]);
    axi = fmav(lam, a.w[i], mu * a.ax0[i]);
  } else if (st.mode == 1) {
    yi = a.yh[i];
    axi = a.axh[i];
    a.y0[i] = yi;
    a.ax0[i] = axi;
  } else {
    yi = V(0);
    axi = V(0);
  }
  const V lo = a.lc[i], hi = a.uc[i];
  const V sv = fmav(-yi, inv_sigma, wv);
  const V yn = sigma * (clampd(sv, lo, hi) - sv);
  const V dy = yi - yn;
  acc_fma(acc[0], dy, dy);
  acc_fma(acc[1], dy, axi - wv);
  if (st.check) {
    const V v = a.ax[i];  // A xhat_t, by the check iteration's own SpMV
    const V pr = (v - clampd(v, lo, hi)) * a.inv_dr[i];
    acc_fma(acc[3], pr, pr);
    acc[4] += (double)((yn > V(0) ? lo * yn : V(0)) + (yn < V(0) ? hi * yn : V(0)));
    if (a.yb0) (st.cand ? a.yb1 : a.yb0)[i] = yn;
  }
  a.qy[i] = fmav(V(2), yn, -yi);
  a.yh[i] = yn;
  a.w[i] = wv;
}

template <class V>
struct ColStepR {
  int restart;
  int check;  // iteration t is a check iteration
  int cand;
  V lam, mu, tau;  // in the iterates' type
  const V* xc;  // xhat_t
  V* xn;        // xhat_{t+1}
};

template <class V>
__device__ __forceinline__ ColStepR<V> col_step_r(const Ctl& c, const ColArgsT<V>& a, int check = -1) {
  ColStepR<V> st;
  st.restart = c.restart;
  st.check = check >= 0 ? check : (is_check(c, c.t) ? 1 : 0);
  st.cand = c.cand_slot;
  st.lam = (V)(-c.hb);
  st.mu = (V)c.he;
  st.tau = (V)c.tau;
  st.xc = (c.t & 1) ? a.xh1 : a.xh0;
  st.xn = (c.t & 1) ? a.xh0 : a.xh1;
  return st;
}

template <class V>
__device__ __forceinline__ void col_prefetch_r(const ColArgsT<V>& a, const ColStepR<V>& st, int j) {
  if (st.restart || st.check) prefetch_l1(st.xc + j);
  if (!st.restart) {
    prefetch_l1(a.xbar + j);
    prefetch_l1(a.x0 + j);
    prefetch_l1(a.aty0 + j);
  }
  prefetch_l1(a.c + j);
  prefetch_l1(a.lv + j);
  prefetch_l1(a.uv + j);
}

// Column epilogue of the reflected form: u = A^T qy_t of column j (A^T yhat_t after a restart
// decision).
template <class V>
__device__ __forceinline__ void col_epilogue_r(const ColArgsT<V>& a, const ColStepR<V>& st, int j, V u,
                                               double (&acc)[kNumSums]) {
  const V tau = st.tau;
  V xj, atyj;
  if (st.restart) {
    xj = st.xc[j];
    atyj = u;
    a.x0[j] = xj;
    a.aty0[j] = u;
  } else {
    const V lam = st.lam, mu = st.mu;
    xj = fmav(lam, a.xbar[j], mu * a.x0[j]);
    atyj = fmav(lam, u, mu * a.aty0[j]);
  }
  const V cj = a.c[j], lo = a.lv[j], hi = a.uv[j];
  const V xn = clampd(fmav(-tau, cj - atyj, xj), lo, hi);
  const V dx = xj - xn;
  acc_fma(acc[0], dx, dx);
  if (st.check) {
    const V xc = st.xc[j];
    const V atyh = st.restart ? u : a.aty[j];  // A^T yhat_t (the check iteration's own SpMV)
    acc_fma(acc[2], cj, xc);
    const V rc = cj - atyh;
    const bool fl = isfinite(lo), fu = isfinite(hi);
    const V rr = (fl && fu) ? rc : (fl ? maxv(rc, V(0)) : (fu ? minv(rc, V(0)) : V(0)));
    const V dd = (rc - rr) * a.inv_dc[j];
    acc_fma(acc[3], dd, dd);
    acc[4] += (double)((rr > V(0) ? lo * rr : V(0)) + (rr < V(0) ? hi * rr : V(0)));
    if (a.xb0) (st.cand ? a.xb1 : a.xb0)[j] = xc;
  }
  a.xbar[j] = fmav(V(2), xn, -xj);
  st.xn[j] = xn;
}

// Scalar control after the column phase: carries the x-side sums to the next residual, runs
// the relative KKT test on check iterations (Section 4), and advances t.
__device__ __forceinline__ void col_control(Ctl& c, const double (&tot)[kNumSums], bool check) {
  const int64_t t = c.t;
  c.sxx = tot[0];
  c.sx0 = tot[1];
  if (check) {
    const double pobj = tot[2], dobj = c.dobj_y + tot[4];
    const double pres = sqrt(c.pres2), dres = sqrt(tot[3]);
    const double rg = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    const double rp = pres / (1.0 + c.lu_norm);
    const double rd = dres / (1.0 + c.c_norm);
    double mx = rg;
    if (!(rp <= mx)) mx = rp;
    if (!(rd <= mx)) mx = rd;
    c.kkt[0] = rg;
    c.kkt[1] = rp;
    c.kkt[2] = rd;
    c.kkt[3] = mx;
    c.kkt[4] = pobj;
    c.kkt[5] = dobj;
    c.kkt[6] = pres;
    c.kkt[7] = dres;
    if (rg <= c.tol && rp <= c.tol && rd <= c.tol) {
      c.status = kOptimal;
      c.iters = t + 1;
      c.done = 1;
      return;
    }
    if (c.patience > 0) {  // FP32 phase: stop once its rounding floor stalls or reverses progress
      if (mx < c.best_kkt) {
        c.best_kkt = mx;
        c.since_best = 0;
        c.omega_best = c.omega;
        c.integral_best = c.pid_integral;
        c.eprev_best = c.pid_eprev;
        for (int q = 0; q < 8; ++q) c.kkt_best[q] = c.kkt[q];
        c.best_slot = c.cand_slot;  // zhat_t of this check is in that slot; write the other next
        c.cand_slot ^= 1;
      } else if (++c.since_best >= c.patience || !(mx <= 100.0 * c.best_kkt)) {
        c.status = kStalled;
        c.iters = t + 1;
        c.done = 1;
        return;
      }
    }
  }
  if (t + 1 >= c.max_iter) {
    c.status = kIterLimit;
    c.iters = t + 1;
    c.done = 1;
    return;
  }
  c.t = t + 1;
}

// Hand-over from the FP32 phase to the FP64 refinement phase (a new epoch anchored at the FP32
// point): the FP64 phase continues the iteration count, omega and the PID state, starts with
// k = 0 and the restart flag set (so its first row step takes y = yhat, Ax = A xhat as iterate
// and anchor), gets the final tolerance and max_iter_fp64 further iterations.  After a stall
// of the FP32 phase, omega and the PID state go back to their values at its best check (past
// that point the FP32 rounding, not the iterate, drove the PID).  A NUMERICAL end of the FP32
// phase is kept and ends the solve.
__device__ __forceinline__ void switch_ctl(Ctl& c, double tol, int64_t max_iter_fp64) {
  const int64_t it32 = c.iters;
  c.iters32 = it32;
  if (c.status == kNumerical) return;
  if (c.status == kStalled && c.best_kkt < INFINITY) {
    const double om = c.omega_best, eta = c.eta;
    c.omega = om;
    c.tau = eta / om;
    c.sigma = eta * om;
    c.inv_sigma = 1.0 / (eta * om);
    c.w_over_eta = om / eta;
    c.inv_eta_w = 1.0 / (eta * om);
    c.pid_integral = c.integral_best;
    c.pid_eprev = c.eprev_best;
  }
  c.patience = 0;
  c.t = it32;
  c.k = 0;
  c.restart = 1;
  c.done = 0;
  c.status = 0;
  c.tol = tol;
  c.max_iter = it32 + max_iter_fp64;
  c.bodies = 0;
}

}  // namespace pdhg
