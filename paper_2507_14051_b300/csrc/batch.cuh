// Shared definitions of the batched solver (batch.cu) and the differentiable unrolled solve
// (diff.cu): the concatenated layout, per-instance state records, the batch handle and the
// task-list SpMV.
#pragma once
#include <string>
#include <vector>

#include "host_util.h"
#include "lp_batch.h"
#include "lp_diff.h"
#include "step.cuh"

namespace pdhg {

constexpr int kBatchUnroll = 16;  // iterations per launch of the batch loop kernel
// The batch's tile schedule when lp_params.lane_target / tile_rows are 0 (measured on 512 uneven
// LPs: 4.74 ms per FP64 iteration of the grid loop, against 5.08 ms with (8, 32)).
constexpr int kBatchLaneTarget = 32;
constexpr int kBatchTileRows = 8;
constexpr int kLocalCtas = 8;       // CTAs (SMs) of the cluster that runs one small instance
constexpr int kMaxInst = LP_BATCH_MAX_INSTANCES;

// Place of one instance in the concatenated arrays.
struct BInst {
  int32_t row0, m, col0, n;
  int32_t ta0, nta;  // its tasks in the row-task list (A)
  int32_t tt0, ntt;  // its tasks in the column-task list (A^T)
  int32_t local;     // 1: solved by one cluster (kb_cluster_loop), not by the grid loop
  int32_t pad;
};

// Step of the coming row phase of one instance (written by the previous column control).
struct BRow {
  RowStep st;
  int32_t par;  // t & 1: which xhat buffer holds xhat_t
};

// Step of the coming column phase of one instance (written by the row control).
struct BCol {
  int32_t restart, check, cand, par;
  double ha, hb, he, tau;
};

// Batch-wide state of a stage.
struct BatchCtl {
  unsigned int n_done;   // instances finished in this stage
  int32_t overrun;       // the loop outran max_iter (internal error)
  int64_t bodies, max_bodies;
  unsigned int pw_left;  // power iteration: instances not converged yet
};

// Power iteration state of one instance.
struct BPw {
  double lam, prev, s;
  int32_t done, iters;
};

template <class V>
struct BatchArgs {
  RowArgsT<V> ra;  // concatenated row-side vectors and A (bins unused)
  ColArgsT<V> ca;  // concatenated column-side vectors and A^T (bins unused)
  const int4* tasksA;
  const int4* tasksT;
  const BInst* inst;
  int32_t count;
  Ctl* ctl;
  BRow* rstep;
  BCol* cstep;
  int32_t* done;
  double* tpartA;
  double* tpartT;
  BatchCtl* bc;
  double* trace;      // NULL, or per instance trace_cap rows of (r, omega, restart, k)
  int64_t trace_cap;
};

// Trace rows of instance ii (NULL when not tracing).
template <class V>
__device__ __forceinline__ double* trace_of(const BatchArgs<V>& a, int ii) {
  return a.trace ? a.trace + (size_t)ii * (size_t)a.trace_cap * 4 : nullptr;
}

// Task descriptor: x = first (global) row, y = rows in the tile, z = (G << 24) | entries per
// lane, w = instance.
__device__ __forceinline__ int task_lanes(const int4& t) { return t.z >> 24; }
__device__ __forceinline__ int task_per_lane(const int4& t) { return t.z & 0xFFFFFF; }

// y = A x over a task list (no epilogue): hand-over products and the power iteration.
template <class V>
__global__ void __launch_bounds__(kThreads) kb_spmv(const int4* __restrict__ tasks, int32_t ntasks,
                                                    const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci,
                                                    const V* __restrict__ val, const V* __restrict__ x,
                                                    V* __restrict__ y) {
  const LoadPolicy pol = make_policy();
  const int lane = threadIdx.x & 31;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < ntasks; j += gridDim.x * kWarps) {
    const int4 td = tasks[j];
    const V v = tile_spmv(rp, ci, val, x, td.x, td.y, task_lanes(td), task_per_lane(td), lane, pol);
    if (lane < td.y) y[td.x + lane] = v;
  }
}

}  // namespace pdhg

using namespace pdhg;
using namespace pdhg_host;

// ====================================================================== host side

// Frozen schedule of one instance at one iteration of the differentiable solve (diff.cu).
struct DiffSched {
  double tau, sigma, inv_sigma, al, be, ep;
  int rho;
};

// Buffers of the differentiable unrolled solve (diff.cu), made on first use; a buffer that must
// grow (trace, checkpoints) is freed and made again.
struct Diff {
  int64_t K = 0, C = 0;          // steps and checkpoint spacing of the last forward
  int64_t cap_trace = 0, cap_ck = 0, cap_mask = 0;
  bool forward_done = false;
  int32_t *irow = nullptr, *icol = nullptr;  // instance of each global row / column
  double *x = nullptr, *y = nullptr, *x0 = nullptr, *y0 = nullptr, *xh = nullptr, *yh = nullptr;
  double *xbar = nullptr;
  double *lx = nullptr, *ly = nullptr, *lx0 = nullptr, *ly0 = nullptr, *lv = nullptr;
  double *lxbar = nullptr, *laty = nullptr, *sx = nullptr, *sy = nullptr;
  double *gc = nullptr, *glv = nullptr, *guv = nullptr, *glc = nullptr, *guc = nullptr;
  double* ck = nullptr;                       // checkpoints: (x, y, x0, y0) every C steps
  DiffSched* sched = nullptr;                 // schedule table (instance, iteration)
  int64_t cap_sched = 0;
  uint8_t *mx = nullptr, *my = nullptr;       // clamp codes of one segment
  std::vector<void*> own;                     // fixed-size buffers
  ~Diff() {
    for (void* p : own) cudaFree(p);
    cudaFree(ck);
    cudaFree(sched);
    cudaFree(mx);
    cudaFree(my);
  }
};

struct lp_batch {
  int device = 0, num_sms = 0;
  int32_t count = 0;
  lp_params prm{};
  int64_t sum_m = 0, sum_n = 0, sum_nnz = 0;
  int32_t ntA = 0, ntT = 0;
  std::vector<BInst> inst;
  std::vector<double> eta;
  int32_t n_local = 0, n_wide = 0;  // small instances; the first n_wide of them run on clusters
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int32_t* local_list = nullptr;  // device: the small instances (cluster loop)
  int32_t* local_next = nullptr;  // device: next unclaimed entry of the wide [0] and tiny [1] lists
  std::vector<int32_t> local_host;  // host copy of local_list
  int grid = 1, grid32 = 1, gridS = 1;  // loop grids (FP64, FP32), block-per-instance grid
  bool solved = false;
  cudaStream_t last_stream = nullptr;
  cudaStream_t setup_stream = nullptr;

  // device
  int32_t *rpA = nullptr, *ciA = nullptr, *rpT = nullptr, *ciT = nullptr;
  double *valA = nullptr, *valT = nullptr;
  int32_t *row_perm = nullptr, *col_perm = nullptr;  // per instance, local original index
  double *c = nullptr, *lv = nullptr, *uv = nullptr, *inv_dc = nullptr, *dc = nullptr;
  double *x = nullptr, *x0 = nullptr, *xh0 = nullptr, *xh1 = nullptr, *aty = nullptr, *aty0 = nullptr;
  double *lc = nullptr, *uc = nullptr, *inv_dr = nullptr, *dr = nullptr;
  double *y = nullptr, *y0 = nullptr, *yh = nullptr, *ax = nullptr, *ax0 = nullptr, *axh = nullptr;
  // reflected form of the small instances' shared-memory loop: qy = 2 yhat - y, w = A xbar,
  // xbar = 2 xhat - x
  double *qy = nullptr, *w = nullptr, *xbar = nullptr;
  double* out_buf = nullptr;
  struct F32 {
    float *valA = nullptr, *valT = nullptr;
    float *c = nullptr, *lv = nullptr, *uv = nullptr, *inv_dc = nullptr;
    float *x = nullptr, *x0 = nullptr, *xh0 = nullptr, *xh1 = nullptr, *aty = nullptr, *aty0 = nullptr;
    float *lc = nullptr, *uc = nullptr, *inv_dr = nullptr;
    float *y = nullptr, *y0 = nullptr, *yh = nullptr, *ax = nullptr, *ax0 = nullptr, *axh = nullptr;
    float *xb0 = nullptr, *xb1 = nullptr, *yb0 = nullptr, *yb1 = nullptr;
    float *qy = nullptr, *w = nullptr, *xbar = nullptr;
  } f32;
  // the small instances' shared-memory loop (kb_sm_loop): CTAs per cluster (0: not used),
  // dynamic shared memory per CTA (FP64, FP32), and per entry of local_list its split
  int sm_ctas = 0;
  int32_t sm_bytes[2] = {0, 0};
  SmSplit* d_splits = nullptr;
  int4 *tasksA = nullptr, *tasksT = nullptr;
  BInst* d_inst = nullptr;
  Ctl *ctl = nullptr, *ctl_init = nullptr;
  BRow* rstep = nullptr;
  BCol* cstep = nullptr;
  int32_t* done = nullptr;
  double *tpartA = nullptr, *tpartT = nullptr;
  BatchCtl* bc = nullptr;
  BPw* pw = nullptr;
  double* trace = nullptr;  // differentiation: per-instance trace of the schedule solve
  int64_t trace_cap = 0;
  double* d_eta = nullptr;  // step sizes on the device (differentiation)
  Diff* diff = nullptr;
  cudaGraph_t graph64 = nullptr, graph32 = nullptr;
  cudaGraphExec_t exec64 = nullptr, exec32 = nullptr;

  std::vector<void*> allocations;
  template <class T>
  cudaError_t alloc(T** p, size_t count_) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (count_ > 0 ? count_ : 1) * sizeof(T));
    if (e == cudaSuccess) allocations.push_back(v);
    *p = static_cast<T*>(v);
    return e;
  }
  ~lp_batch() {
    if (last_stream) cudaStreamSynchronize(last_stream);
    delete diff;
    cudaFree(trace);
    if (exec64) cudaGraphExecDestroy(exec64);
    if (graph64) cudaGraphDestroy(graph64);
    if (exec32) cudaGraphExecDestroy(exec32);
    if (graph32) cudaGraphDestroy(graph32);
    for (void* p : allocations) cudaFree(p);
    if (setup_stream) cudaStreamDestroy(setup_stream);
    if (side_stream) cudaStreamDestroy(side_stream);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }
};

template <class V>
void fill_batch_args(const lp_batch* h, BatchArgs<V>& a);

template <>
inline void fill_batch_args<double>(const lp_batch* h, BatchArgs<double>& a) {
  a = BatchArgs<double>{};
  a.ra.rp = h->rpA; a.ra.ci = h->ciA; a.ra.val = h->valA;
  a.ra.xh0 = h->xh0; a.ra.xh1 = h->xh1;
  a.ra.y = h->y; a.ra.y0 = h->y0; a.ra.yh = h->yh; a.ra.ax = h->ax; a.ra.ax0 = h->ax0; a.ra.axh = h->axh;
  a.ra.lc = h->lc; a.ra.uc = h->uc; a.ra.inv_dr = h->inv_dr;
  a.ca.rp = h->rpT; a.ca.ci = h->ciT; a.ca.val = h->valT; a.ca.yh = h->yh;
  a.ca.xh0 = h->xh0; a.ca.xh1 = h->xh1;
  a.ca.x = h->x; a.ca.x0 = h->x0; a.ca.aty = h->aty; a.ca.aty0 = h->aty0;
  a.ca.c = h->c; a.ca.lv = h->lv; a.ca.uv = h->uv; a.ca.inv_dc = h->inv_dc;
  a.ra.qy = h->qy; a.ra.w = h->w; a.ra.xbar = h->xbar; a.ca.xbar = h->xbar; a.ca.qy = h->qy;
  a.tasksA = h->tasksA; a.tasksT = h->tasksT; a.inst = h->d_inst; a.count = h->count;
  a.ctl = h->ctl; a.rstep = h->rstep; a.cstep = h->cstep; a.done = h->done;
  a.tpartA = h->tpartA; a.tpartT = h->tpartT; a.bc = h->bc;
  a.trace = nullptr; a.trace_cap = 0;
}

template <>
inline void fill_batch_args<float>(const lp_batch* h, BatchArgs<float>& a) {
  const auto& f = h->f32;
  a = BatchArgs<float>{};
  a.ra.rp = h->rpA; a.ra.ci = h->ciA; a.ra.val = f.valA;
  a.ra.xh0 = f.xh0; a.ra.xh1 = f.xh1;
  a.ra.y = f.y; a.ra.y0 = f.y0; a.ra.yh = f.yh; a.ra.ax = f.ax; a.ra.ax0 = f.ax0; a.ra.axh = f.axh;
  a.ra.lc = f.lc; a.ra.uc = f.uc; a.ra.inv_dr = f.inv_dr;
  a.ra.yb0 = f.yb0; a.ra.yb1 = f.yb1;
  a.ca.rp = h->rpT; a.ca.ci = h->ciT; a.ca.val = f.valT; a.ca.yh = f.yh;
  a.ca.xh0 = f.xh0; a.ca.xh1 = f.xh1;
  a.ca.x = f.x; a.ca.x0 = f.x0; a.ca.aty = f.aty; a.ca.aty0 = f.aty0;
  a.ca.c = f.c; a.ca.lv = f.lv; a.ca.uv = f.uv; a.ca.inv_dc = f.inv_dc;
  a.ca.xb0 = f.xb0; a.ca.xb1 = f.xb1;
  a.ra.qy = f.qy; a.ra.w = f.w; a.ra.xbar = f.xbar; a.ca.xbar = f.xbar; a.ca.qy = f.qy;
  a.tasksA = h->tasksA; a.tasksT = h->tasksT; a.inst = h->d_inst; a.count = h->count;
  a.ctl = h->ctl; a.rstep = h->rstep; a.cstep = h->cstep; a.done = h->done;
  a.tpartA = h->tpartA; a.tpartT = h->tpartT; a.bc = h->bc;
  a.trace = nullptr; a.trace_cap = 0;
}


// A solve of exactly K FP64 iterations of every instance recording its trace (batch.cu).
lp_status batch_schedule_solve(lp_batch* h, int64_t K, cudaStream_t s);
