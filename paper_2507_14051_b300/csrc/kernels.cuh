// Kernel argument blocks and launch declarations of the solver (definitions in iterate.cu
// and setup.cu).
#pragma once

#include "device.cuh"

namespace pdhg {

// Argument blocks of the two phases, for value type V (double: FP64 path; float: the FP32
// phase of the mixed-precision solve).  The scalar state, the reductions and the control are
// FP64 in both.
template <class V>
struct RowArgsT {
  const int32_t* rp;
  const int32_t* ci;
  const V* val;
  const V* xh0;  // xhat ping-pong: xhat_t is xh[t & 1]
  const V* xh1;
  V *y, *y0, *yh, *ax, *ax0, *axh;
  const V *lc, *uc, *inv_dr;
  V *yb0, *yb1;  // FP32 stall guard: yhat at check iterations, two slots (null: guard off)
  // reflected form of the loop kernel (gamma = 1): qy = 2 yhat - y (the reflected dual point,
  // gathered by the column phase), w = A xbar of the last row phase, xbar = 2 xhat - x (the
  // gathered primal point)
  V *qy, *w;
  const V* xbar;
  Ctl* ctl;
  double* partials;
  double* trace;
  BinTable bins;
  int32_t m;  // rows
};

template <class V>
struct ColArgsT {
  const int32_t* rp;
  const int32_t* ci;
  const V* val;
  const V* yh;
  V *xh0, *xh1;
  V *x, *x0, *aty, *aty0;
  const V *c, *lv, *uv, *inv_dc;
  V *xb0, *xb1;  // FP32 stall guard: xhat at check iterations, two slots (null: guard off)
  // reflected form of the loop kernel: xbar = 2 xhat - x (written here, gathered by the row
  // phase), qy = 2 yhat - y (gathered here)
  V* xbar;
  const V* qy;
  Ctl* ctl;
  double* partials;
  BinTable bins;
  int32_t n;  // columns
};

using RowArgs = RowArgsT<double>;
using ColArgs = ColArgsT<double>;

struct PwCtl {
  double lambda, s;
  unsigned int count_a, count_b;
  int32_t step;  // index of the current step inside a batch (lambda is also stored in hist[step])
};

// iterate.cu.  The phase kernels are templates over the value type V of the matrix and the
// iterates (double; float for the first phase of a mixed-precision solve).  A __global__
// template is launched only from the file that instantiates it (elsewhere its launch stub has no
// registered device code), so other files launch them through these pointers.
template <class V>
struct IterKernels {
  void (*rows)(RowArgsT<V>);
  void (*cols)(ColArgsT<V>);
  void (*loop)(RowArgsT<V>, ColArgsT<V>, double*, double*, double*, int32_t, cudaGraphConditionalHandle, int32_t);
  // the loop kernel in the reflected form (gamma = 1 only), and both forms as one-cluster launches
  void (*loop_refl)(RowArgsT<V>, ColArgsT<V>, double*, double*, double*, int32_t, cudaGraphConditionalHandle,
                    int32_t);
  void (*loop_one)(RowArgsT<V>, ColArgsT<V>, double*, double*, double*, int32_t, cudaGraphConditionalHandle,
                   int32_t);
  void (*loop_refl_one)(RowArgsT<V>, ColArgsT<V>, double*, double*, double*, int32_t,
                        cudaGraphConditionalHandle, int32_t);
  void (*init_cols)(int32_t, const V*, const V*, const V*, V*, V*, V*, V*, V*, V*, Ctl*, double*);
  void (*init_rows)(int32_t, V*, V*, V*, V*, V*, V*);
};
template <class V>
IterKernels<V> iter_kernels();  // instantiated for double and float in iterate.cu

// smem_loop.cu: the loop kernel as one thread-block cluster that holds the whole LP in its CTAs'
// shared memory.  CTA q owns rows [rs[q], rs[q + 1]) and columns [cs[q], cs[q + 1]) of the
// solver's (permuted) index space.
constexpr int kSmMaxCtas = 16;
struct SmSplit {
  int32_t rs[kSmMaxCtas + 1];
  int32_t cs[kSmMaxCtas + 1];
  int32_t smem_bytes;  // dynamic shared memory per CTA of the launch
};

// Byte offsets of one CTA's arrays in its dynamic shared memory (each start 16-byte aligned):
// the table of partial sums (two buffers of kSmMaxCtas x kNumSums doubles), the replicas of
// the gathered vectors (xbar, xhat in two buffers, n each; qy, yhat, m each), the CTA's rows of
// A (mr + 1 local offsets, nzr indices and values) with its row-slice vectors, and its rows of
// A^T (nc + 1 offsets, nzc entries) with its column-slice vectors.  vb: bytes per value.
struct SmLayout {
  uint32_t part, xbar, xh0, xh1, qy, yh;
  uint32_t rp, ci, val, y0, w, ax0, axh, ax, lc, uc, inv_dr;
  uint32_t rpT, ciT, valT, x0, aty0, aty, c, lv, uv, inv_dc;
  uint64_t total;  // bytes (the offsets are meaningful only when total fits the launch)
};
__host__ __device__ inline uint32_t sm_take(uint64_t& o, uint64_t bytes) {
  const uint64_t at = o;
  o += (bytes + 15u) & ~uint64_t(15);
  return (uint32_t)at;
}
__host__ __device__ inline SmLayout sm_layout(int64_t m, int64_t n, int64_t mr, int64_t nc, int64_t nzr,
                                              int64_t nzc, int vb) {
  SmLayout L;
  uint64_t o = 0;
  L.part = sm_take(o, (uint64_t)2 * kSmMaxCtas * kNumSums * 8);
  L.xbar = sm_take(o, n * vb);
  L.xh0 = sm_take(o, n * vb);
  L.xh1 = sm_take(o, n * vb);
  L.qy = sm_take(o, m * vb);
  L.yh = sm_take(o, m * vb);
  L.rp = sm_take(o, (mr + 1) * 4);
  L.ci = sm_take(o, nzr * 4);
  L.val = sm_take(o, nzr * vb);
  uint32_t* rowv[8] = {&L.y0, &L.w, &L.ax0, &L.axh, &L.ax, &L.lc, &L.uc, &L.inv_dr};
  for (uint32_t* f : rowv) *f = sm_take(o, mr * vb);
  L.rpT = sm_take(o, (nc + 1) * 4);
  L.ciT = sm_take(o, nzc * 4);
  L.valT = sm_take(o, nzc * vb);
  uint32_t* colv[7] = {&L.x0, &L.aty0, &L.aty, &L.c, &L.lv, &L.uv, &L.inv_dc};
  for (uint32_t* f : colv) *f = sm_take(o, nc * vb);
  L.total = o;
  return L;
}
template <class V>
using SmLoopFn = void (*)(RowArgsT<V>, ColArgsT<V>, SmSplit, int32_t, cudaGraphConditionalHandle, int32_t);
template <class V>
SmLoopFn<V> sm_loop_kernel();  // instantiated for double and float in smem_loop.cu
__global__ void k_init_ctl(Ctl* dst, Ctl src);
__global__ void k_set_cond(cudaGraphConditionalHandle h, Ctl* ctl, int32_t unroll);
__global__ void k_unpermute_scale(int32_t len, const int32_t* perm, const double* v,
                                  const double* d, double* out);
__global__ void k_spmv(const int32_t* rp, const int32_t* ci, const double* val, const double* x,
                       double* y, BinTable bins);
// mixed precision: conversions and the hand-over from the FP32 phase to the FP64 phase
__global__ void k_to_float(int64_t len, const double* src, float* dst);
__global__ void k_switch_ctl(Ctl* ctl, double tol, int64_t max_iter_fp64);
__global__ void k_switch_vectors(int32_t n, int32_t m, Ctl* ctl, const float* xh0f,
                                 const float* xh1f, const float* yhf, const float* xb0,
                                 const float* xb1, const float* yb0, const float* yb1, double* x,
                                 double* x0, double* yh, double* xh0, double* xh1,
                                 int32_t fp32_only);
__global__ void k_warm_cols(int32_t n, const double* c, const double* lv, const double* uv,
                            double* xh0, double* xh1, const double* x, const double* aty,
                            double* aty0, double* xbar, Ctl* ctl, double* partials);

// setup.cu
__global__ void k_row_factor(int32_t rows, int32_t split, const int32_t* rp, const double* val, int32_t kind,
                             double expo, double* f);
__global__ void k_apply_factors(int32_t rows, int32_t split, const int32_t* rp, const int32_t* ci, double* val,
                                const double* fr, const double* fc, int32_t transposed);
__global__ void k_mul_inplace(int32_t len, double* d, const double* f);
__global__ void k_scale_cols(int32_t n, const double* dc, double* c, double* lv, double* uv,
                             double* inv_dc);
__global__ void k_scale_rows(int32_t m, const double* dr, double* lc, double* uc, double* inv_dr);
__global__ void k_sell_gather(int64_t len, const int32_t* src, const int32_t* ci, const double* val,
                              int32_t* sell_ci, double* sell_val);
__global__ void k_pw_start(int32_t n, const int32_t* col_perm, uint64_t seed, double* u, PwCtl* pw,
                           double* partials);
__global__ void k_pw_rows(const int32_t* rp, const int32_t* ci, const double* val, const double* u,
                          double* w, BinTable bins, PwCtl* pw, double* partials, double* hist,
                          int32_t step);
__global__ void k_pw_cols(const int32_t* rp, const int32_t* ci, const double* val, const double* w,
                          double* u, BinTable bins, PwCtl* pw, double* partials);

}  // namespace pdhg
