// Kernel argument blocks and launch declarations of the solver (definitions in iterate.cu
// and setup.cu).
#pragma once

#include "device.cuh"

namespace pdhg {

struct RowArgs {
  const int32_t* rp;
  const int32_t* ci;
  const double* val;
  const double* xh0;  // xhat ping-pong: xhat_t is xh[t & 1]
  const double* xh1;
  double *y, *y0, *yh, *ax, *ax0, *axh;
  const double *lc, *uc, *inv_dr;
  Ctl* ctl;
  double* partials;
  double* trace;
  BinTable bins;
};

struct ColArgs {
  const int32_t* rp;
  const int32_t* ci;
  const double* val;
  const double* yh;
  double *xh0, *xh1;
  double *x, *x0, *aty, *aty0;
  const double *c, *lv, *uv, *inv_dc;
  Ctl* ctl;
  double* partials;
  BinTable bins;
};

struct PwCtl {
  double lambda, s;
  unsigned int count_a, count_b;
  int32_t step;  // index of the current step inside a batch (lambda is also stored in hist[step])
};

// iterate.cu
__global__ void k1_rows(RowArgs a);
__global__ void k2_cols(ColArgs a);
__global__ void k_loop(RowArgs ra, ColArgs ca, double* part_rows, double* part_cols, int32_t iters,
                       cudaGraphConditionalHandle cond, int32_t use_cond);
__global__ void k_init_ctl(Ctl* dst, Ctl src);
__global__ void k_init_cols(int32_t n, const double* c, const double* lv, const double* uv,
                            double* xh0, double* x, double* x0, double* aty, double* aty0,
                            Ctl* ctl, double* partials);
__global__ void k_init_rows(int32_t m, double* y, double* y0, double* yh, double* ax,
                            double* ax0, double* axh);
__global__ void k_set_cond(cudaGraphConditionalHandle h, Ctl* ctl, int32_t unroll);
__global__ void k_unpermute_scale(int32_t len, const int32_t* perm, const double* v,
                                  const double* d, double* out);
__global__ void k_spmv(const int32_t* rp, const int32_t* ci, const double* val, const double* x,
                       double* y, BinTable bins);

// setup.cu
__global__ void k_row_factor(int32_t rows, const int32_t* rp, const double* val, int32_t kind,
                             double expo, double* f);
__global__ void k_apply_factors(int32_t rows, const int32_t* rp, const int32_t* ci, double* val,
                                const double* fr, const double* fc, int32_t transposed);
__global__ void k_mul_inplace(int32_t len, double* d, const double* f);
__global__ void k_scale_cols(int32_t n, const double* dc, double* c, double* lv, double* uv,
                             double* inv_dc);
__global__ void k_scale_rows(int32_t m, const double* dr, double* lc, double* uc, double* inv_dr);
__global__ void k_pw_start(int32_t n, const int32_t* col_perm, uint64_t seed, double* u, PwCtl* pw,
                           double* partials);
__global__ void k_pw_rows(const int32_t* rp, const int32_t* ci, const double* val, const double* u,
                          double* w, BinTable bins, PwCtl* pw, double* partials, double* hist,
                          int32_t step);
__global__ void k_pw_cols(const int32_t* rp, const int32_t* ci, const double* val, const double* w,
                          double* u, BinTable bins, PwCtl* pw, double* partials);

}  // namespace pdhg
