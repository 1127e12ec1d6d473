/*
 * FP64 oracle for restarted reflected-Halpern PDHG on LP (cuPDLPx, arXiv 2507.14051).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain sequential C, double precision, natural
 * row/column order, no blocking, fusion or reordering.  It shares no code, no
 * header and no constant generator with the CUDA library; only tests, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Problem (Section 2.1, eq. lp):
 *   min c^T x  s.t.  l_c <= A x <= u_c,  l_v <= x <= u_v     (bounds may be +-inf)
 * Dual (same equation): max -p(-y; l_c, u_c) - p(-r; l_v, u_v)  s.t.  c - A^T y = r,
 *   y in Y, r in R, p(y; l, u) = u^T y+ - l^T y-  (Section 1.2, notation).
 *
 * Reading of the saddle form (Section 2.1, eq. lp-pd).  The printed Lagrangian
 * carries +y^T A x, but the PDHG step (Section 2.2, eq. pdhg) moves x along
 * -(c - A^T y) and the metric P has +A off the diagonal; both belong to
 * L(x, y) = c^T x - y^T A x + p(-y; l_c, u_c)-type terms, i.e. the bilinear
 * term enters with a minus sign.  Everything below follows eq. pdhg and P.
 *
 * Functions (each cites the passage it follows):
 *   orc_spmv / orc_spmv_t      y = A x, x = A^T y                 (products in eq. pdhg)
 *   orc_pdhg_step              one PDHG step T(z)                  (Section 2.2, eq. pdhg)
 *   orc_p_norm_sq              ||(dx, dy)||_P^2                    (Section 2.2, matrix P)
 *   orc_kkt                    relative KKT error                  (Section 4, termination criteria)
 *   orc_restart_decide         the three restart conditions         (Section 3, adaptive restart)
 *   orc_pid_update             PID update of log(omega)            (Section 3, primal weight update)
 *   orc_power_norm             ||A||_2 by power iteration          (Section 3, stepsize)
 *   orc_solve                  the whole iteration                 (Sections 2.2, 3, 4)
 *
 * Parity pins for every function live in tests/ (closed forms, invariants,
 * brute force, a library LP solver, the Halpern rate bound).  The PID gains
 * are not printed in the paper; their default values are therefore a reading,
 * but the PID arithmetic is pinned by its P-only special case.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double gamma;            /* reflection coefficient, Section 3 "Reflection", in [0, 1] */
  double beta_sufficient;  /* Section 3, restart condition 1 */
  double beta_necessary;   /* Section 3, restart condition 2 */
  double beta_artificial;  /* Section 3, restart condition 3 */
  double k_p, k_i, k_d;    /* Section 3, PID gains */
  double eta;              /* > 0: step size used as given; <= 0: 0.998 / ||A||_2 by power iteration */
  double omega0;           /* initial primal weight, Section 3 ("set to 1.0") */
  int64_t check_every;     /* termination test every this many iterations (and at the last one) */
  int32_t restart_enabled; /* 0: plain reflected Halpern without restarts */
  int32_t pid_enabled;     /* 0: primal weight fixed at omega0 */
  double power_tol;        /* relative change that stops the power iteration */
  int64_t power_max_iter;
  uint64_t power_seed;
  int32_t ruiz_iters;      /* diagonal preconditioning: Ruiz passes (0: none) */
  int32_t pc_enabled;      /* then one Pock-Chambolle pass with exponent pc_alpha */
  double pc_alpha;
  int32_t rescale;         /* then divide the objective by ||c~||_2 and all bounds by the 2-norm
                              of the finite constraint bounds (1 where a norm is 0) */
} orc_params;

enum { ORC_OPTIMAL = 1, ORC_ITER_LIMIT = 2, ORC_NUMERICAL = 3 };

/* ---------------------------------------------------------------- products */

/* out = A x (row i: sum over its stored entries in storage order). */
void orc_spmv(int32_t m, const int64_t* rp, const int32_t* ci, const double* val,
              const double* x, double* out) {
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += val[p] * x[ci[p]];
    out[i] = s;
  }
}

/* out = A^T y, accumulated row by row in natural order. */
void orc_spmv_t(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val,
                const double* y, double* out) {
  for (int32_t j = 0; j < n; ++j) out[j] = 0.0;
  for (int32_t i = 0; i < m; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) out[ci[p]] += val[p] * y[i];
}

static double clampd(double v, double lo, double hi) {
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}

/* ------------------------------------------------------------- PDHG step */

/*
 * One PDHG step (Section 2.2, eq. pdhg) with tau = eta/omega, sigma = eta*omega:
 *   x+ = proj_X(x - tau (c - A^T y))
 *   y+ = y - sigma A(2x+ - x) - sigma proj_{-S}(y/sigma - A(2x+ - x)),  -S = [-u_c, -l_c].
 * The dual line is evaluated in the equivalent form
 *   y+ = sigma (proj_S(s) - s),  s = A(2x+ - x) - y/sigma,
 * which follows from proj_{-S}(w) = -proj_S(-w).  Both forms are the same map;
 * this one keeps y+ in Y exactly in floating point (a row with l_c = -inf gets
 * y+ <= 0 because proj_S(s) <= s), whereas rounding in the printed form can
 * leave multipliers of the wrong sign of order 1e-17 on such rows, which make
 * the dual objective of Section 4 minus infinity.
 * work: n + m doubles.
 */
void orc_pdhg_step(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val,
                   const double* c, const double* lc, const double* uc, const double* lv,
                   const double* uv, double eta, double omega, const double* x, const double* y,
                   double* xp, double* yp, double* work) {
  const double tau = eta / omega, sigma = eta * omega;
  double* aty = work;       /* n */
  double* axbar = work + n; /* m */
  orc_spmv_t(m, n, rp, ci, val, y, aty);
  for (int32_t j = 0; j < n; ++j) xp[j] = clampd(x[j] - tau * (c[j] - aty[j]), lv[j], uv[j]);
  double* xbar = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t j = 0; j < n; ++j) xbar[j] = 2.0 * xp[j] - x[j];
  orc_spmv(m, rp, ci, val, xbar, axbar);
  free(xbar);
  for (int32_t i = 0; i < m; ++i) {
    double s = axbar[i] - y[i] / sigma;
    yp[i] = sigma * (clampd(s, lc[i], uc[i]) - s);
  }
}

/* ||(dx, dy)||_P^2 = (omega/eta)|dx|^2 + 2 dy^T A dx + |dy|^2/(eta omega)   (Section 2.2, P). */
double orc_p_norm_sq(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val,
                     double eta, double omega, const double* dx, const double* dy) {
  double* adx = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  orc_spmv(m, rp, ci, val, dx, adx);
  double sx = 0.0, sy = 0.0, cross = 0.0;
  for (int32_t j = 0; j < n; ++j) sx += dx[j] * dx[j];
  for (int32_t i = 0; i < m; ++i) {
    sy += dy[i] * dy[i];
    cross += dy[i] * adx[i];
  }
  free(adx);
  return (omega / eta) * sx + 2.0 * cross + sy / (eta * omega);
}

/* ------------------------------------------------------------------- KKT */

/*
 * Relative KKT error of (x, y) (Section 4, optimality termination criteria).
 *   r      = proj_R(c - A^T y), R_j from the finiteness of (l_v, u_v) (Section 2.1);
 *   pobj   = c^T x;
 *   dobj   = -p(-y; l_c, u_c) - p(-r; l_v, u_v) = sum l_c y+ - u_c y-  +  sum l_v r+ - u_v r-,
 *            a zero multiplier contributing 0 even against an infinite bound;
 *   gap    = |pobj - dobj|                   vs eps (1 + |pobj| + |dobj|)
 *   pres   = ||A x - proj_[l_c,u_c](A x)||_2 vs eps (1 + ||(L, U)||_2), the norm over the
 *            finite entries of l_c and u_c;
 *   dres   = ||c - A^T y - r||_2             vs eps (1 + ||c||_2);
 *   the fourth criterion ||r - proj_R(r)|| is zero for this choice of r.
 * out[0..7] = rel_gap, rel_pres, rel_dres, rel_kkt (max of the three), pobj, dobj, pres, dres.
 */
void orc_kkt(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val,
             const double* c, const double* lc, const double* uc, const double* lv,
             const double* uv, const double* x, const double* y, double* out) {
  double* ax = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* aty = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  orc_spmv(m, rp, ci, val, x, ax);
  orc_spmv_t(m, n, rp, ci, val, y, aty);
  double pobj = 0.0, dobj = 0.0, pres2 = 0.0, dres2 = 0.0, lu2 = 0.0, c2 = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    pobj += c[j] * x[j];
    c2 += c[j] * c[j];
    double rc = c[j] - aty[j];
    int fl = isfinite(lv[j]), fu = isfinite(uv[j]);
    double r;
    if (fl && fu) r = rc;                    /* R_j = R   */
    else if (fl) r = rc > 0.0 ? rc : 0.0;    /* R_j = R+  */
    else if (fu) r = rc < 0.0 ? rc : 0.0;    /* R_j = R-  */
    else r = 0.0;                            /* R_j = {0} */
    if (r > 0.0) dobj += lv[j] * r;
    if (r < 0.0) dobj += uv[j] * r;          /* -u_v r-  with r- = -r */
    double d = rc - r;
    dres2 += d * d;
  }
  for (int32_t i = 0; i < m; ++i) {
    if (y[i] > 0.0) dobj += lc[i] * y[i];
    if (y[i] < 0.0) dobj += uc[i] * y[i];
    double p = ax[i] - clampd(ax[i], lc[i], uc[i]);
    pres2 += p * p;
    if (isfinite(lc[i])) lu2 += lc[i] * lc[i];
    if (isfinite(uc[i])) lu2 += uc[i] * uc[i];
  }
  free(ax);
  free(aty);
  double gap = fabs(pobj - dobj);
  double pres = sqrt(pres2), dres = sqrt(dres2);
  out[0] = gap / (1.0 + fabs(pobj) + fabs(dobj));
  out[1] = pres / (1.0 + sqrt(lu2));
  out[2] = dres / (1.0 + sqrt(c2));
  double mx = out[0];
  if (!(out[1] <= mx)) mx = out[1];
  if (!(out[2] <= mx)) mx = out[2];
  out[3] = mx;
  out[4] = pobj;
  out[5] = dobj;
  out[6] = pres;
  out[7] = dres;
}

/* --------------------------------------------------------------- restart */

/*
 * Restart test at step k >= 1 of the current epoch (Section 3, adaptive restart):
 *   (1) r_k <= beta_sufficient r_0
 *   (2) r_k <= beta_necessary  r_0  and  r_k > r_{k-1}
 *   (3) k >= beta_artificial T,  T = total iterations so far (t + 1 for 0-based t).
 * Returns 1 to restart.
 */
int32_t orc_restart_decide(int64_t k, int64_t t, double r, double r0, double r_prev,
                           double beta_s, double beta_n, double beta_a) {
  if (k < 1) return 0;
  if (r <= beta_s * r0) return 1;
  if (r <= beta_n * r0 && r > r_prev) return 1;
  if ((double)k >= beta_a * (double)(t + 1)) return 1;
  return 0;
}

/* ------------------------------------------------------------------- PID */

/*
 * PID update at a restart (Section 3, primal weight update):
 *   e_n = log( sqrt(w) |dx| / (|dy| / sqrt(w)) )
 *   log w_{n+1} = log w_n - [K_P e_n + K_I sum_{i<=n} e_i + K_D (e_n - e_{n-1})]
 * The derivative term is 0 at the first update.  If |dx| or |dy| is zero or
 * not finite, nothing changes.  log w is kept in [-23, 23].
 * state[0] = integral, state[1] = e_prev, state[2] = 1 once e_prev is set.
 * Returns the new omega.
 */
double orc_pid_update(double omega, double dx_norm, double dy_norm, double kp, double ki, double kd,
                      double* state) {
  if (!(dx_norm > 0.0) || !(dy_norm > 0.0) || !isfinite(dx_norm) || !isfinite(dy_norm)) return omega;
  double sw = sqrt(omega);
  double e = log((sw * dx_norm) / (dy_norm / sw));
  state[0] += e;
  double de = state[2] != 0.0 ? e - state[1] : 0.0;
  double lw = log(omega) - (kp * e + ki * state[0] + kd * de);
  if (lw > 23.0) lw = 23.0;
  if (lw < -23.0) lw = -23.0;
  state[1] = e;
  state[2] = 1.0;
  return exp(lw);
}

/* -------------------------------------------------------- power iteration */

/* splitmix64 (Steele, Lea, Flood 2014; the public-domain reference by S. Vigna). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* start vector entry: uniform on [-1, 1) from the top 53 bits */
double orc_start_entry(uint64_t seed, uint64_t i) {
  return (double)(splitmix64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/*
 * ||A||_2 by power iteration on A^T A (Section 3, stepsize: "approximated by
 * power iteration").  v_0 from splitmix64; each step w = A v, lambda = |w|^2
 * (the Rayleigh quotient of A^T A at unit v), v = A^T w / |A^T w|.  Stops when
 * |lambda - lambda_prev| <= tol * lambda or after max_iter steps.  Returns
 * sqrt(lambda); 0 for A = 0.  *iters_out receives the step count.
 */
double orc_power_norm(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val,
                      double tol, int64_t max_iter, uint64_t seed, int64_t* iters_out) {
  if (m == 0 || n == 0) { if (iters_out) *iters_out = 0; return 0.0; }
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)m);
  double nv = 0.0;
  for (int32_t j = 0; j < n; ++j) { v[j] = orc_start_entry(seed, (uint64_t)j); nv += v[j] * v[j]; }
  nv = sqrt(nv);
  for (int32_t j = 0; j < n; ++j) v[j] /= nv;
  double lam = 0.0, lam_prev = 0.0;
  int64_t it = 0;
  for (it = 1; it <= max_iter; ++it) {
    orc_spmv(m, rp, ci, val, v, w);
    lam = 0.0;
    for (int32_t i = 0; i < m; ++i) lam += w[i] * w[i];
    if (lam == 0.0) break;
    orc_spmv_t(m, n, rp, ci, val, w, v);
    double s = 0.0;
    for (int32_t j = 0; j < n; ++j) s += v[j] * v[j];
    s = sqrt(s);
    for (int32_t j = 0; j < n; ++j) v[j] /= s;
    if (it > 1 && fabs(lam - lam_prev) <= tol * lam) break;
    lam_prev = lam;
  }
  if (it > max_iter) it = max_iter;
  free(v);
  free(w);
  if (iters_out) *iters_out = it;
  return sqrt(lam);
}

/* ------------------------------------------------------- preconditioning */

/*
 * Diagonal preconditioning.  The paper evaluates termination "on the original
 * LP instance, not the preconditioned ones" (Section 4) without defining the
 * preconditioner; this oracle uses the two published diagonal scalings of the
 * PDLP family, applied as  A~ = D_r A D_c:
 *   Ruiz equilibration (D. Ruiz, 2001): each pass divides every row by the
 *     square root of its largest |entry| and every column by the square root of
 *     its largest |entry|, both measured on the matrix at the start of the pass;
 *   Pock-Chambolle (T. Pock and A. Chambolle, 2011) with exponent alpha: row i
 *     divided by sqrt(sum_j |a_ij|^(2-alpha)), column j by sqrt(sum_i |a_ij|^alpha).
 * A row or column without entries keeps the factor 1.  Entries are updated
 * in place as val <- (val * fr[i]) * fc[j] for each pass's factors fr, fc.
 * dr, dc receive the accumulated factors.
 */
void orc_scale(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, double* val,
               int32_t ruiz_iters, int32_t pc_enabled, double pc_alpha, double* dr, double* dc) {
  double* fr = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* fc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < m; ++i) dr[i] = 1.0;
  for (int32_t j = 0; j < n; ++j) dc[j] = 1.0;
  int32_t passes = ruiz_iters + (pc_enabled ? 1 : 0);
  for (int32_t pass = 0; pass < passes; ++pass) {
    int pc = (pass == ruiz_iters);
    for (int32_t i = 0; i < m; ++i) fr[i] = 0.0;
    for (int32_t j = 0; j < n; ++j) fc[j] = 0.0;
    for (int32_t i = 0; i < m; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        double a = fabs(val[p]);
        if (pc) {
          fr[i] += pow(a, 2.0 - pc_alpha);
          fc[ci[p]] += pow(a, pc_alpha);
        } else {
          if (a > fr[i]) fr[i] = a;
          if (a > fc[ci[p]]) fc[ci[p]] = a;
        }
      }
    for (int32_t i = 0; i < m; ++i) fr[i] = fr[i] > 0.0 ? 1.0 / sqrt(fr[i]) : 1.0;
    for (int32_t j = 0; j < n; ++j) fc[j] = fc[j] > 0.0 ? 1.0 / sqrt(fc[j]) : 1.0;
    for (int32_t i = 0; i < m; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) val[p] = (val[p] * fr[i]) * fc[ci[p]];
    for (int32_t i = 0; i < m; ++i) dr[i] *= fr[i];
    for (int32_t j = 0; j < n; ++j) dc[j] *= fc[j];
  }
  free(fr);
  free(fc);
}

/* ------------------------------------------------------------------ solve */

/*
 * Restarted reflected Halpern PDHG (Sections 2.2 and 3), from the all-zero
 * start (Section 4, initialization), terminated by the relative KKT test of
 * Section 4.  If preconditioning is on, the iteration runs on the scaled LP
 * (A~ = D_r A D_c, c~ = D_c c, [l_c, u_c]~ = D_r [l_c, u_c], [l_v, u_v]~ = [l_v, u_v] / D_c)
 * and every KKT test, like the returned point, uses the original LP with
 * x = D_c x~, y = D_r y~.  Iteration t (0-based) with epoch step k:
 *   zhat = T(z)                                  eq. pdhg with tau = eta/w, sigma = eta w
 *   r_t  = ||z - zhat||_P                        fixed-point residual, Section 3
 *   if r_t^2 is not finite                       -> NUMERICAL, return zhat
 *   if t is a check iteration and KKT(zhat)<=tol -> OPTIMAL,   return zhat
 *   if t + 1 == max_iter                          -> ITER_LIMIT, return zhat
 *   restart test (three conditions, Section 3), with r_0 the epoch's first
 *   residual and r_{k-1} the previous one;
 *   on restart: PID update of w from |xhat - x0| and |yhat - y0| (Section 3),
 *               anchor and iterate <- zhat ("reset to the current solution"), k <- 0
 *   otherwise:  z <- (k+1)/(k+2) ((1+gamma) zhat - gamma z) + z0/(k+2), k <- k+1
 *               (reflected Halpern update, Section 3)
 * A check iteration is one with (t + 1) % check_every == 0, or the last one.
 * The restart point is zhat = T(z), a point of X x Y.  The step size is
 * 0.998 / ||A~||_2 unless params->eta > 0 gives it.
 *
 * trace (optional, trace_cap rows of 4): r_t, omega used at t, restart flag, k.
 * kkt_out[0..7] as orc_kkt for the returned point.
 */
int32_t orc_solve(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* val_in,
                  const double* c_in, const double* lc_in, const double* uc_in, const double* lv_in,
                  const double* uv_in, const orc_params* prm, double tol, int64_t max_iter,
                  double* x_out, double* y_out, double* kkt_out, int64_t* iters_out,
                  double* eta_out, double* omega_out, int64_t trace_cap, double* trace) {
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  int64_t nnz = rp[m];
  /* scaled copy of the LP (identity factors when preconditioning is off) */
  double* val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double* dr = (double*)malloc(sizeof(double) * mm);
  double* dc = (double*)malloc(sizeof(double) * nn);
  double *c = (double*)malloc(sizeof(double) * nn), *lv = (double*)malloc(sizeof(double) * nn),
         *uv = (double*)malloc(sizeof(double) * nn);
  double *lc = (double*)malloc(sizeof(double) * mm), *uc = (double*)malloc(sizeof(double) * mm);
  if (nnz > 0) memcpy(val, val_in, sizeof(double) * (size_t)nnz);
  orc_scale(m, n, rp, ci, val, prm->ruiz_iters, prm->pc_enabled, prm->pc_alpha, dr, dc);
  for (int32_t j = 0; j < n; ++j) {
    c[j] = c_in[j] * dc[j];
    lv[j] = lv_in[j] / dc[j];
    uv[j] = uv_in[j] / dc[j];
  }
  for (int32_t i = 0; i < m; ++i) {
    lc[i] = lc_in[i] * dr[i];
    uc[i] = uc_in[i] * dr[i];
  }
  /* bound/objective rescaling: x' = x~ / beta, y' = y~ / gamma_c with beta = ||finite (l_c~,
     u_c~)||_2, gamma_c = ||c~||_2; the LP in (x', y') has objective c~ / gamma_c and bounds / beta */
  double beta = 1.0, gamma_c = 1.0;
  if (prm->rescale) {
    double b2 = 0.0, c2 = 0.0;
    for (int32_t i = 0; i < m; ++i) {
      if (isfinite(lc[i])) b2 += lc[i] * lc[i];
      if (isfinite(uc[i])) b2 += uc[i] * uc[i];
    }
    for (int32_t j = 0; j < n; ++j) c2 += c[j] * c[j];
    if (b2 > 0.0) beta = sqrt(b2);
    if (c2 > 0.0) gamma_c = sqrt(c2);
    for (int32_t j = 0; j < n; ++j) {
      c[j] /= gamma_c;
      lv[j] /= beta;
      uv[j] /= beta;
    }
    for (int32_t i = 0; i < m; ++i) {
      lc[i] /= beta;
      uc[i] /= beta;
    }
  }

  double eta = prm->eta;
  if (!(eta > 0.0)) {
    double na = orc_power_norm(m, n, rp, ci, val, prm->power_tol, prm->power_max_iter,
                               prm->power_seed, NULL);
    eta = na > 0.0 ? 0.998 / na : 1.0;
  }
  double* x = (double*)calloc(nn, sizeof(double));
  double* y = (double*)calloc(mm, sizeof(double));
  double* x0 = (double*)calloc(nn, sizeof(double));
  double* y0 = (double*)calloc(mm, sizeof(double));
  double* xh = (double*)calloc(nn, sizeof(double));
  double* yh = (double*)calloc(mm, sizeof(double));
  double* dx = (double*)calloc(nn, sizeof(double));
  double* dy = (double*)calloc(mm, sizeof(double));
  double* xo = (double*)calloc(nn, sizeof(double)); /* x in the original space */
  double* yo = (double*)calloc(mm, sizeof(double));
  double* work = (double*)calloc(nn + mm, sizeof(double));
  double omega = prm->omega0;
  double pid_state[3] = {0.0, 0.0, 0.0};
  int64_t k = 0, t = 0;
  double r0 = 0.0, r_prev = 0.0;
  int32_t status = ORC_ITER_LIMIT;
  double kkt[8] = {NAN, NAN, NAN, NAN, NAN, NAN, NAN, NAN};
  const double g = prm->gamma;

  for (t = 0; t < max_iter; ++t) {
    orc_pdhg_step(m, n, rp, ci, val, c, lc, uc, lv, uv, eta, omega, x, y, xh, yh, work);
    for (int32_t j = 0; j < n; ++j) dx[j] = x[j] - xh[j];
    for (int32_t i = 0; i < m; ++i) dy[i] = y[i] - yh[i];
    double r2 = orc_p_norm_sq(m, n, rp, ci, val, eta, omega, dx, dy);
    double r = sqrt(r2 > 0.0 ? r2 : 0.0);
    if (k == 0) r0 = r;
    if (trace && t < trace_cap) {
      trace[4 * t + 0] = r;
      trace[4 * t + 1] = omega;
      trace[4 * t + 2] = 0.0;
      trace[4 * t + 3] = (double)k;
    }
    if (!isfinite(r2)) { status = ORC_NUMERICAL; break; }
    int last = (t + 1 == max_iter);
    if (((t + 1) % prm->check_every) == 0 || last) {
      for (int32_t j = 0; j < n; ++j) xo[j] = xh[j] * dc[j] * beta;
      for (int32_t i = 0; i < m; ++i) yo[i] = yh[i] * dr[i] * gamma_c;
      orc_kkt(m, n, rp, ci, val_in, c_in, lc_in, uc_in, lv_in, uv_in, xo, yo, kkt);
      if (kkt[0] <= tol && kkt[1] <= tol && kkt[2] <= tol) { status = ORC_OPTIMAL; break; }
    }
    if (last) { status = ORC_ITER_LIMIT; break; }
    int restart = prm->restart_enabled &&
                  orc_restart_decide(k, t, r, r0, r_prev, prm->beta_sufficient,
                                     prm->beta_necessary, prm->beta_artificial);
    if (restart) {
      if (prm->pid_enabled) {
        double sx = 0.0, sy = 0.0;
        for (int32_t j = 0; j < n; ++j) sx += (xh[j] - x0[j]) * (xh[j] - x0[j]);
        for (int32_t i = 0; i < m; ++i) sy += (yh[i] - y0[i]) * (yh[i] - y0[i]);
        omega = orc_pid_update(omega, sqrt(sx), sqrt(sy), prm->k_p, prm->k_i, prm->k_d, pid_state);
      }
      for (int32_t j = 0; j < n; ++j) x[j] = x0[j] = xh[j];
      for (int32_t i = 0; i < m; ++i) y[i] = y0[i] = yh[i];
      k = 0;
      if (trace && t < trace_cap) trace[4 * t + 2] = 1.0;
    } else {
      double a = (double)(k + 1) / (double)(k + 2), b = 1.0 / (double)(k + 2);
      for (int32_t j = 0; j < n; ++j) x[j] = a * ((1.0 + g) * xh[j] - g * x[j]) + b * x0[j];
      for (int32_t i = 0; i < m; ++i) y[i] = a * ((1.0 + g) * yh[i] - g * y[i]) + b * y0[i];
      r_prev = r;
      k += 1;
    }
  }
  for (int32_t j = 0; j < n; ++j) xo[j] = xh[j] * dc[j] * beta;
  for (int32_t i = 0; i < m; ++i) yo[i] = yh[i] * dr[i] * gamma_c;
  if (status == ORC_NUMERICAL || max_iter <= 0)
    orc_kkt(m, n, rp, ci, val_in, c_in, lc_in, uc_in, lv_in, uv_in, xo, yo, kkt);
  if (n > 0) memcpy(x_out, xo, sizeof(double) * (size_t)n);
  if (m > 0) memcpy(y_out, yo, sizeof(double) * (size_t)m);
  if (kkt_out) memcpy(kkt_out, kkt, sizeof(kkt));
  if (iters_out) *iters_out = (max_iter <= 0) ? 0 : ((t < max_iter) ? t + 1 : max_iter);
  if (eta_out) *eta_out = eta;
  if (omega_out) *omega_out = omega;
  free(x); free(y); free(x0); free(y0); free(xh); free(yh); free(dx); free(dy);
  free(xo); free(yo); free(work);
  free(val); free(dr); free(dc); free(c); free(lv); free(uv); free(lc); free(uc);
  return status;
}
