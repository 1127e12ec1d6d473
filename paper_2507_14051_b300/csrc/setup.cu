// Setup kernels: diagonal preconditioning and the power iteration for ||A||_2.
//
// Preconditioning.  The paper checks termination "on the original LP, not the preconditioned
// one" (Section 4) without defining the preconditioner; the library applies the two diagonal
// scalings of the PDLP family, A~ = D_r A D_c:
//   Ruiz equilibration (D. Ruiz, 2001): per pass, rows divided by sqrt(max |a_ij|) and
//     columns by sqrt(max |a_ij|), both measured on the matrix at the start of the pass;
//   Pock-Chambolle (T. Pock, A. Chambolle, 2011), exponent alpha: rows divided by
//     sqrt(sum_j |a_ij|^(2-alpha)), columns by sqrt(sum_i |a_ij|^alpha).
// An empty row or column keeps factor 1.  Each pass updates both stored copies (A and A^T)
// entry by entry as (a * f_row) * f_col, so the two copies stay bit-identical.
//
// Power iteration (Section 3, "Stepsize": ||A||_2 approximated by power iteration): with
// u the unnormalised iterate and s = 1/|u|, each step forms w = s * A u, lambda = |w|^2 (the
// Rayleigh quotient of A^T A at u/|u|), then u = A^T w and s = 1/|u|.  ||A||_2 = sqrt(lambda).
#include "kernels.cuh"

namespace pdhg {

// Per-row statistic of a CSR matrix, then the factor 1/sqrt(stat) (1 when stat == 0).  kind 0:
// max |a|; kind 1: sum |a|^expo.  Rows [0, split) (the long ones: the storage orders rows by
// decreasing length) take one warp each, the others one thread each: an FP64 warp instruction
// costs the FP64 pipe the same whatever its active lanes, so a warp per short row (and its
// lane-0 division and square root) would cost 32 times the arithmetic.
__device__ __forceinline__ double row_stat_term(double a, int32_t kind, double expo) {
  return kind == 0 ? a : (expo == 1.0 ? a : pow(a, expo));
}
__global__ void k_row_factor(int32_t rows, int32_t split, const int32_t* __restrict__ rp,
                             const double* __restrict__ val, int32_t kind, double expo,
                             double* __restrict__ f) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < split; r += nw) {
    const int b = rp[r], e = rp[r + 1];
    double acc = 0.0;
    for (int p = b + lane; p < e; p += 32) {
      const double a = row_stat_term(fabs(val[p]), kind, expo);
      acc = kind == 0 ? fmax(acc, a) : acc + a;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(kFull, acc, off);
      acc = kind == 0 ? fmax(acc, o) : acc + o;
    }
    if (lane == 0) f[r] = acc > 0.0 ? 1.0 / sqrt(acc) : 1.0;
  }
  for (int r = split + blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int b = rp[r], e = rp[r + 1];
    double acc = 0.0;
    for (int p = b; p < e; ++p) {
      const double a = row_stat_term(fabs(val[p]), kind, expo);
      acc = kind == 0 ? fmax(acc, a) : acc + a;
    }
    f[r] = acc > 0.0 ? 1.0 / sqrt(acc) : 1.0;
  }
}

// val <- (val * f_row) * f_col on one stored copy.  For the copy of A, row r of the storage
// is a row of A (f_row = fr[r], f_col = fc[ci]); for the copy of A^T, row r of the storage is
// a column of A (f_row = fr[ci], f_col = fc[r]).  Rows [0, split) one warp each, the others
// one thread each (as k_row_factor).
__global__ void k_apply_factors(int32_t rows, int32_t split, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ ci, double* __restrict__ val,
                                const double* __restrict__ fr, const double* __restrict__ fc,
                                int32_t transposed) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < split; r += nw) {
    const int b = rp[r], e = rp[r + 1];
    for (int p = b + lane; p < e; p += 32) {
      const int o = ci[p];
      const double frow = transposed ? fr[o] : fr[r];
      const double fcol = transposed ? fc[r] : fc[o];
      val[p] = (val[p] * frow) * fcol;
    }
  }
  for (int r = split + blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int b = rp[r], e = rp[r + 1];
    for (int p = b; p < e; ++p) {
      const int o = ci[p];
      const double frow = transposed ? fr[o] : fr[r];
      const double fcol = transposed ? fc[r] : fc[o];
      val[p] = (val[p] * frow) * fcol;
    }
  }
}

__global__ void k_mul_inplace(int32_t len, double* __restrict__ d, const double* __restrict__ f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    d[i] *= f[i];
}

// Sliced tile copies (BinTable::sell_*): slot k takes CSR entry src[k], or column -1 and value 0
// for padding.
__global__ void k_sell_gather(int64_t len, const int32_t* __restrict__ src, const int32_t* __restrict__ ci,
                              const double* __restrict__ val, int32_t* __restrict__ sell_ci,
                              double* __restrict__ sell_val) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = src[k];
    sell_ci[k] = q >= 0 ? ci[q] : -1;
    sell_val[k] = q >= 0 ? val[q] : 0.0;
  }
}

// Scaled column data: c~ = c d_c, l_v~ = l_v / d_c, u_v~ = u_v / d_c, inv_dc = 1 / d_c.
__global__ void k_scale_cols(int32_t n, const double* __restrict__ dc, double* c, double* lv,
                             double* uv, double* inv_dc) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double d = dc[j];
    c[j] = c[j] * d;
    lv[j] = lv[j] / d;
    uv[j] = uv[j] / d;
    inv_dc[j] = 1.0 / d;
  }
}

// Scaled row data: l_c~ = l_c d_r, u_c~ = u_c d_r, inv_dr = 1 / d_r.
__global__ void k_scale_rows(int32_t m, const double* __restrict__ dr, double* lc, double* uc,
                             double* inv_dr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double d = dr[i];
    lc[i] = lc[i] * d;
    uc[i] = uc[i] * d;
    inv_dr[i] = 1.0 / d;
  }
}

__global__ void __launch_bounds__(kThreads) k_pw_start(int32_t n, const int32_t* __restrict__ col_perm,
                                                       uint64_t seed, double* __restrict__ u,
                                                       PwCtl* pw, double* partials) {
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double v = start_entry(seed, (uint64_t)col_perm[j]);
    u[j] = v;
    s[0] = fma(v, v, s[0]);
  }
  if (!block_sums_last(s, 1, partials, &pw->count_b)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, nullptr, tot);
  if (threadIdx.x != 0) return;
  pw->s = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
  pw->count_b = 0;
}

// w = s * (A u); lambda = |w|^2, also recorded as hist[step] so that the host can apply the
// stopping rule to a batch of steps after one synchronisation.
__global__ void __launch_bounds__(kThreads) k_pw_rows(const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ u,
                                                      double* __restrict__ w, BinTable bins,
                                                      PwCtl* pw, double* partials, double* hist,
                                                      int32_t step) {
  const double sc = pw->s;
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row(bins, rp, ci, val, u, pol, s, [&](int i, double v, double (&acc)[kNumSums]) {
    v *= sc;
    w[i] = v;
    acc[0] = fma(v, v, acc[0]);
  });
  if (!block_sums_last(s, 1, partials, &pw->count_a)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, &bins, tot);
  if (threadIdx.x != 0) return;
  pw->lambda = tot[0];
  hist[step] = tot[0];
  pw->count_a = 0;
}

// u = A^T w; s = 1/|u|.
__global__ void __launch_bounds__(kThreads) k_pw_cols(const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ w,
                                                      double* __restrict__ u, BinTable bins,
                                                      PwCtl* pw, double* partials) {
  double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const LoadPolicy pol = make_policy();
  for_each_row(bins, rp, ci, val, w, pol, s, [&](int j, double v, double (&acc)[kNumSums]) {
    u[j] = v;
    acc[0] = fma(v, v, acc[0]);
  });
  if (!block_sums_last(s, 1, partials, &pw->count_b)) return;
  double tot[kNumSums];
  block_totals(partials, gridDim.x, 1, &bins, tot);
  if (threadIdx.x != 0) return;
  pw->s = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
  pw->count_b = 0;
}

}  // namespace pdhg
