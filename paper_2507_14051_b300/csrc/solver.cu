// Host runtime of the solver and its C ABI (include/lp.h).
//
// lp_create: validation -> row/column length binning and one permutation of rows and columns
// (rows of similar length contiguous, longest first) -> CSR of A and of A^T with 32-bit offsets
// -> upload -> diagonal preconditioning on the device -> power iteration on the device ->
// capture of the iteration loop as one CUDA graph (a conditional while node whose body is
// `unroll` pairs of the two iteration kernels plus the kernel that sets the loop condition).
// lp_solve: resets the scalar state, runs the first primal step, launches the graph.
// lp_get: waits, un-permutes and un-scales the last PDHG output.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "lp.h"
#include "kernels.cuh"
#include "host_util.h"
#include <nvtx3/nvToolsExt.h>

using namespace pdhg;
using namespace pdhg_host;

namespace {
thread_local std::string g_err;

// NVTX range around an entry point (visible in a profiler's timeline; the header-only NVTX API
// does nothing unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

// Sets the calling thread's lp_last_error message (used by entry points in other files).
void pdhg_set_last_error(const std::string& msg) { g_err = msg; }

struct lp_solver {
  int device = 0;
  int num_sms = 148;
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  lp_params prm{};
  std::vector<int32_t> row_perm, col_perm;  // permuted index -> original index
  BinTable binsA{}, binsT{};
  int gridA = 1, gridT = 1, gridV = 1, gridL = 1, gridL32 = 1, max_grid = 1;
  bool loop_active = false;  // the graph body is the cooperative loop kernel
  bool refl = false;         // the loop kernel runs in the reflected form (gamma = 1)
  int cluster = 0;           // > 0: the loop kernel runs as one cluster of this many CTAs
  int cluster_max = 0;       // the largest cluster the loop kernels can be launched as (16 or 8)
  bool small = false;        // each phase has at most kClusterTasks tasks
  bool loop_fits = false;    // both phases' grids fit on the device at once
  // the shared-memory cluster loop (smem_loop.cu): CTAs (0: the LP does not fit, driver not
  // offered), row / column slices, dynamic shared memory per CTA for FP64 [0] and FP32 [1]
  int sm_ctas = 0;
  SmSplit sm_split{};
  int32_t sm_bytes[2] = {0, 0};
  bool sm_active = false;  // the graph body is the shared-memory cluster loop
  int tile_rows_used = 1;    // rows per tile of the bins (lp_params.tile_rows, or the automatic choice)
  // device storage
  int32_t *rpA = nullptr, *ciA = nullptr, *rpT = nullptr, *ciT = nullptr;
  double *valA = nullptr, *valT = nullptr;
  int32_t *d_row_perm = nullptr, *d_col_perm = nullptr;
  double *c = nullptr, *lv = nullptr, *uv = nullptr, *inv_dc = nullptr, *dc = nullptr;
  double *lc = nullptr, *uc = nullptr, *inv_dr = nullptr, *dr = nullptr;
  double *x = nullptr, *x0 = nullptr, *xh0 = nullptr, *xh1 = nullptr, *aty = nullptr, *aty0 = nullptr;
  double *y = nullptr, *y0 = nullptr, *yh = nullptr, *ax = nullptr, *ax0 = nullptr, *axh = nullptr;
  // reflected form of the loop kernel (gamma = 1): xbar = 2 xhat - x, qy = 2 yhat - y, w = A xbar
  double *xbar = nullptr, *qy = nullptr, *w = nullptr;
  // sliced copies of the one-lane-per-row tiles (BinTable::sell_*) of A and A^T
  double *sell_valA = nullptr, *sell_valT = nullptr;
  int32_t *sell_ciA = nullptr, *sell_ciT = nullptr, *sell_offA = nullptr, *sell_offT = nullptr;
  int32_t *sell_srcA = nullptr, *sell_srcT = nullptr;  // source entry of each slot (-1: padding)
  int64_t sell_lenA = 0, sell_lenT = 0;
  // FP32 phase of the mixed-precision solve (allocated when precision != 0)
  struct F32 {
    float *valA = nullptr, *valT = nullptr;
    float *c = nullptr, *lv = nullptr, *uv = nullptr, *inv_dc = nullptr;
    float *x = nullptr, *x0 = nullptr, *xh0 = nullptr, *xh1 = nullptr, *aty = nullptr, *aty0 = nullptr;
    float *lc = nullptr, *uc = nullptr, *inv_dr = nullptr;
    float *y = nullptr, *y0 = nullptr, *yh = nullptr, *ax = nullptr, *ax0 = nullptr, *axh = nullptr;
    float *xb0 = nullptr, *xb1 = nullptr, *yb0 = nullptr, *yb1 = nullptr;  // stall guard's slots
    float *xbar = nullptr, *qy = nullptr, *w = nullptr;  // reflected form of the loop kernel
    float *sell_valA = nullptr, *sell_valT = nullptr;      // sliced tiles' values
  } f32;
  cudaGraph_t graph32 = nullptr;
  cudaGraphExec_t exec32 = nullptr;
  bool loop_active32 = false;
  double* out_buf = nullptr;
  double* partials = nullptr;
  double* partials2 = nullptr;  // column-phase partials of the loop kernel
  double* partials3 = nullptr;  // the loop kernel's restart-time PID norms
  double* trace = nullptr;
  int64_t trace_cap = 0;
  Ctl* ctl = nullptr;
  PwCtl* pw = nullptr;
  double* pinned = nullptr;  // 8 doubles of pinned host memory for scalar read-back
  double lu_norm = 0.0, c_norm = 0.0;
  double eta = 0.0, norm_A = 0.0;
  int64_t pw_iters = 0;
  bool power_valid = false;
  double rescale_ratio = 1.0;  // ||c~|| / ||b~|| of the preconditioned data  // norm_A holds the power-iteration estimate for the current settings
  bool solved = false;
  cudaStream_t last_stream = nullptr;
  cudaStream_t setup_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_unroll = 0;
  std::vector<void*> allocations;

  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (count > 0 ? count : 1) * sizeof(T));
    if (e == cudaSuccess) allocations.push_back(v);
    *p = static_cast<T*>(v);
    return e;
  }
  ~lp_solver() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (exec32) cudaGraphExecDestroy(exec32);
    if (graph32) cudaGraphDestroy(graph32);
    for (void* p : allocations) cudaFree(p);
    if (pinned) cudaFreeHost(pinned);
    if (setup_stream) cudaStreamDestroy(setup_stream);
  }
};

namespace {

// Tasks per phase up to which the automatic choice runs the loop kernel as one cluster (at most
// one task per warp of a 16-CTA cluster).
constexpr int64_t kClusterTasks = 16 * kWarps;

// Schedule over rows already sorted by decreasing length class.  The leading rows longer than
// kLongRowMin become chunk tasks of kChunkNnz entries.  Each remaining length class becomes a
// bin of tiles shaped by tile_shape: G lanes per row (at most lane_target entries per lane and
// pass) and R rows per tile.
BinTable make_bins(const std::vector<int32_t>& rp, int lane_target, int tile_rows, std::vector<int4>& chunks) {
  BinTable bt{};
  const int32_t rows = (int32_t)rp.size() - 1;
  int32_t r = 0;
  chunks.clear();
  while (r < rows && rp[r + 1] - rp[r] > kLongRowMin) {
    const int32_t nch = (rp[r + 1] - rp[r] + kChunkNnz - 1) / kChunkNnz;
    const int32_t first = (int32_t)chunks.size();
    for (int32_t q = 0; q < nch; ++q) chunks.push_back(make_int4(r, first, nch, 0));
    ++r;
  }
  bt.long_rows = r;
  bt.nchunks = (int32_t)chunks.size();
  int32_t task = 0;
  while (r < rows) {
    const int cls = length_class(rp[r + 1] - rp[r]);
    int32_t e = r + 1;
    while (e < rows && length_class(rp[e + 1] - rp[e]) == cls) ++e;
    const TileShape ts = tile_shape(int64_t(1) << cls, lane_target, tile_rows);
    Bin& b = bt.bin[bt.nbins++];
    b.row0 = r;
    b.row1 = e;
    b.lanes = ts.lanes;
    b.rows_per_tile = ts.rows;
    b.task0 = task;
    b.per_lane = ts.per_lane;
    task += (e - r + ts.rows - 1) / ts.rows;
    r = e;
  }
  bt.ntasks = task;
  return bt;
}

// Sliced layout of a bin table's one-lane-per-row bins (32-row tiles; BinTable::sell_*): marks
// those bins, and returns per tile task (counted from the first tile task) its first slot
// (off, ntasks + 1 entries) and per slot the CSR entry it holds (src, -1 for padding).  Returns
// false (and marks nothing) if the slots would not fit 32-bit offsets.
bool build_sell(const std::vector<int32_t>& rp, BinTable& bt, std::vector<int32_t>& off, std::vector<int32_t>& src) {
  off.assign((size_t)bt.ntasks + 1, 0);
  int64_t total = 0;
  for (int b = 0; b < bt.nbins; ++b) {
    const Bin& B = bt.bin[b];
    const bool sl = B.lanes == 1 && B.rows_per_tile == 32;
    const int32_t ntiles = (B.row1 - B.row0 + B.rows_per_tile - 1) / B.rows_per_tile;
    for (int32_t t = 0; t < ntiles; ++t) {
      off[B.task0 + t] = (int32_t)total;
      if (!sl) continue;
      const int32_t r0 = B.row0 + t * 32, r1 = r0 + 32 < B.row1 ? r0 + 32 : B.row1;
      int32_t slots = 0;
      for (int32_t r = r0; r < r1; ++r) slots = rp[r + 1] - rp[r] > slots ? rp[r + 1] - rp[r] : slots;
      total += (int64_t)32 * slots;
      if (total >= (int64_t(1) << 31)) return false;
    }
  }
  off[bt.ntasks] = (int32_t)total;
  src.assign((size_t)total, -1);
  for (int b = 0; b < bt.nbins; ++b) {
    Bin& B = bt.bin[b];
    if (!(B.lanes == 1 && B.rows_per_tile == 32)) continue;
    B.sliced = 1;
    for (int32_t r = B.row0; r < B.row1; ++r) {
      const int32_t t = B.task0 + (r - B.row0) / 32, L = (r - B.row0) % 32;
      for (int32_t k = rp[r]; k < rp[r + 1]; ++k) src[(size_t)off[t] + (size_t)32 * (k - rp[r]) + L] = k;
    }
  }
  return true;
}

void fill_args(const lp_solver* h, RowArgs& ra, ColArgs& ca) {
  ra = RowArgs{};
  ra.rp = h->rpA; ra.ci = h->ciA; ra.val = h->valA;
  ra.xh0 = h->xh0; ra.xh1 = h->xh1;
  ra.y = h->y; ra.y0 = h->y0; ra.yh = h->yh; ra.ax = h->ax; ra.ax0 = h->ax0; ra.axh = h->axh;
  ra.lc = h->lc; ra.uc = h->uc; ra.inv_dr = h->inv_dr;
  ra.qy = h->qy; ra.w = h->w; ra.xbar = h->xbar;
  ra.ctl = h->ctl; ra.partials = h->partials; ra.trace = h->trace_cap > 0 ? h->trace : nullptr;
  ra.bins = h->binsA;
  ra.m = h->m;
  ca = ColArgs{};
  ca.rp = h->rpT; ca.ci = h->ciT; ca.val = h->valT; ca.yh = h->yh;
  ca.xh0 = h->xh0; ca.xh1 = h->xh1;
  ca.x = h->x; ca.x0 = h->x0; ca.aty = h->aty; ca.aty0 = h->aty0;
  ca.c = h->c; ca.lv = h->lv; ca.uv = h->uv; ca.inv_dc = h->inv_dc;
  ca.xbar = h->xbar; ca.qy = h->qy;
  ca.ctl = h->ctl; ca.partials = h->partials; ca.bins = h->binsT;
  ca.n = h->n;
}

void fill_args(const lp_solver* h, RowArgsT<float>& ra, ColArgsT<float>& ca) {
  const auto& f = h->f32;
  ra = RowArgsT<float>{};
  ra.rp = h->rpA; ra.ci = h->ciA; ra.val = f.valA;
  ra.xh0 = f.xh0; ra.xh1 = f.xh1;
  ra.y = f.y; ra.y0 = f.y0; ra.yh = f.yh; ra.ax = f.ax; ra.ax0 = f.ax0; ra.axh = f.axh;
  ra.lc = f.lc; ra.uc = f.uc; ra.inv_dr = f.inv_dr;
  ra.yb0 = f.yb0; ra.yb1 = f.yb1;
  ra.qy = f.qy; ra.w = f.w; ra.xbar = f.xbar;
  ra.ctl = h->ctl; ra.partials = h->partials; ra.trace = h->trace_cap > 0 ? h->trace : nullptr;
  ra.bins = h->binsA;
  ra.bins.sell_val = f.sell_valA;
  ra.m = h->m;
  ca = ColArgsT<float>{};
  ca.rp = h->rpT; ca.ci = h->ciT; ca.val = f.valT; ca.yh = f.yh;
  ca.xh0 = f.xh0; ca.xh1 = f.xh1;
  ca.x = f.x; ca.x0 = f.x0; ca.aty = f.aty; ca.aty0 = f.aty0;
  ca.c = f.c; ca.lv = f.lv; ca.uv = f.uv; ca.inv_dc = f.inv_dc;
  ca.xb0 = f.xb0; ca.xb1 = f.xb1;
  ca.xbar = f.xbar; ca.qy = f.qy;
  ca.ctl = h->ctl; ca.partials = h->partials; ca.bins = h->binsT;
  ca.bins.sell_val = f.sell_valT;
  ca.n = h->n;
}

// Launch configuration of the loop kernel: cooperative over its whole grid, or (h->cluster > 0)
// one cluster of h->cluster CTAs spread over as many SMs.
template <class V>
cudaError_t launch_loop(const lp_solver* h, const RowArgsT<V>& ra, const ColArgsT<V>& ca, int32_t iters,
                        cudaGraphConditionalHandle cond, int32_t use_cond, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3((unsigned)kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  if (h->sm_active) {
    SmSplit sp = h->sm_split;
    sp.smem_bytes = h->sm_bytes[sizeof(V) == sizeof(float) ? 1 : 0];
    cfg.gridDim = dim3((unsigned)h->sm_ctas);
    cfg.dynamicSmemBytes = (size_t)sp.smem_bytes;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)h->sm_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicySpread;
    cfg.numAttrs = 2;
    cfg.attrs = attr;
    return cudaLaunchKernelEx(&cfg, sm_loop_kernel<V>(), ra, ca, sp, iters, cond, use_cond);
  }
  if (h->cluster > 0) {
    cfg.gridDim = dim3((unsigned)h->cluster);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)h->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicySpread;
    cfg.numAttrs = 2;
  } else {
    cfg.gridDim = dim3((unsigned)(sizeof(V) == sizeof(float) ? h->gridL32 : h->gridL));
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.numAttrs = 1;
  }
  cfg.attrs = attr;
  const IterKernels<V> k = iter_kernels<V>();
  auto kern = h->cluster > 0 ? (h->refl ? k.loop_refl_one : k.loop_one) : (h->refl ? k.loop_refl : k.loop);
  return cudaLaunchKernelEx(&cfg, kern, ra, ca, h->partials, h->partials2, h->partials3, iters, cond, use_cond);
}

// Sets up the shared-memory cluster loop if the LP fits: the largest cluster (16, else 8) that
// the kernel can be launched as with the shared memory its slices need, in both precisions the
// solve uses.  Leaves h->sm_ctas = 0 otherwise.
void setup_sm_loop(lp_solver* h, const std::vector<int32_t>& rpA, const std::vector<int32_t>& rpT) {
  h->sm_ctas = 0;
  if (h->m < 1 || h->n < 1) return;
  for (size_t i = 0; i + 1 < rpA.size(); ++i)
    if (rpA[i + 1] - rpA[i] > kSmMaxLen) return;
  for (size_t j = 0; j + 1 < rpT.size(); ++j)
    if (rpT[j + 1] - rpT[j] > kSmMaxLen) return;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int nprec = h->prm.precision != 0 ? 2 : 1;
  for (int c : {16, 8}) {
    SmSplit sp{};
    sm_slices(rpA, c, sp.rs);
    sm_slices(rpT, c, sp.cs);
    int32_t bytes[2] = {0, 0};
    bool ok = true;
    for (int pr = 0; pr < nprec && ok; ++pr) {
      const int vb = pr == 0 ? 8 : 4;
      uint64_t mx = 0;
      for (int q = 0; q < c; ++q) {
        const int32_t a0 = sp.rs[q], a1 = sp.rs[q + 1], b0 = sp.cs[q], b1 = sp.cs[q + 1];
        const uint64_t t = sm_layout(h->m, h->n, a1 - a0, b1 - b0, rpA[a1] - rpA[a0], rpT[b1] - rpT[b0], vb).total;
        mx = t > mx ? t : mx;
      }
      const void* kern = pr == 0 ? (const void*)sm_loop_kernel<double>() : (const void*)sm_loop_kernel<float>();
      cudaFuncAttributes fa{};
      ok = cudaFuncGetAttributes(&fa, kern) == cudaSuccess && mx + fa.sharedSizeBytes <= (uint64_t)optin &&
           cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx) == cudaSuccess &&
           (c <= 8 || cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess);
      if (ok) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3((unsigned)kThreads);
        cfg.dynamicSmemBytes = (size_t)mx;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0;
      }
      bytes[pr] = (int32_t)mx;
    }
    cudaGetLastError();
    if (ok) {
      h->sm_ctas = c;
      h->sm_split = sp;
      h->sm_bytes[0] = bytes[0];
      h->sm_bytes[1] = bytes[1];
      return;
    }
  }
}

// The largest cluster (16, else 8) that every cluster form of the loop kernel can be launched as
// on this device (0 if none: the cluster driver is then not offered).
template <class V>
int max_loop_cluster(int& best) {
  const IterKernels<V> k = iter_kernels<V>();
  decltype(k.loop_one) kerns[2] = {k.loop_one, k.loop_refl_one};
  for (int q = 0; q < 2; ++q) {
    const auto kern = kerns[q];
    int found = 0;
    for (int c : {16, 8}) {
      if (c > best) continue;
      if (c > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)c);
      cfg.blockDim = dim3((unsigned)kThreads);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0) {
        found = c;
        break;
      }
      cudaGetLastError();
    }
    best = found < best ? found : best;
  }
  return best;
}

// Captures the solve loop of one precision: a graph whose conditional while node runs the body
// until the solve is done.  Body: one cooperative launch of the loop kernel (`unroll`
// iterations; it sets the loop condition itself) or, for persistent = 0 or if the driver
// refuses a cooperative kernel in the body, `unroll` pairs of the phase kernels plus the kernel
// that sets the condition.
template <class V>
lp_status build_graph_for(lp_solver* h, cudaGraph_t* graph, cudaGraphExec_t* exec, bool* loop_active) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (*exec) {
      cudaGraphExecDestroy(*exec);
      *exec = nullptr;
    }
    if (*graph) {
      cudaGraphDestroy(*graph);
      *graph = nullptr;
    }
    const int pers = h->prm.persistent;
    const bool want = pers == 1 || pers == 2 || h->sm_active ||
                      ((pers == -1 || pers == 3) && (h->loop_fits || h->cluster > 0));
    const bool loop = want && attempt == 0;
    RowArgsT<V> ra{};
    ColArgsT<V> ca{};
    fill_args(h, ra, ca);
    CK(cudaGraphCreate(graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, *graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, *graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t s = h->setup_stream;
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    if (loop) {
      le = launch_loop<V>(h, ra, ca, h->prm.unroll, cond, 1, s);
    } else {
      for (int u = 0; u < h->prm.unroll; ++u) {
        iter_kernels<V>().rows<<<h->gridA, kThreads, 0, s>>>(ra);
        iter_kernels<V>().cols<<<h->gridT, kThreads, 0, s>>>(ca);
      }
      k_set_cond<<<1, 1, 0, s>>>(cond, h->ctl, h->prm.unroll);
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &captured);
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphInstantiate(exec, *graph, 0);
    else if (e == cudaSuccess) e = le;
    if (e == cudaSuccess) {
      *loop_active = loop;
      return LP_OK;
    }
    cudaGetLastError();  // clear the launch error before retrying without the loop kernel
    if (!loop) return fail(LP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  return fail(LP_ERR_CUDA, "graph capture failed");
}

lp_status build_graph(lp_solver* h) {
  // the reflected form of the loop kernel needs gamma = 1 (2 zhat - z is then both the Halpern
  // step's reflected point and the extrapolated point of the dual step)
  h->refl = h->prm.gamma == 1.0;
  // the shared-memory cluster loop (reflected form only) whenever the LP fits it, for
  // persistent 3 or -1; persistent 3 on an LP that does not fit takes the choice of -1
  h->sm_active = h->refl && h->sm_ctas > 0 && (h->prm.persistent == 3 || h->prm.persistent == -1);
  const bool want_cluster =
      !h->sm_active && (h->prm.persistent == 2 || ((h->prm.persistent == -1 || h->prm.persistent == 3) && h->small));
  h->cluster = want_cluster ? h->cluster_max : 0;
  lp_status st = build_graph_for<double>(h, &h->graph, &h->exec, &h->loop_active);
  if (st != LP_OK) return st;
  if (h->prm.precision != 0) {
    st = build_graph_for<float>(h, &h->graph32, &h->exec32, &h->loop_active32);
    if (st != LP_OK) return st;
  }
  h->graph_unroll = h->prm.unroll;
  return LP_OK;
}

// Power iteration (Section 3, "Stepsize") on the device.  Steps run in batches of kPwBatch
// without host synchronisation; each step records its lambda, and the host then applies the
// stopping rule step by step, so the estimate is the one of the first step that meets it (the
// extra steps of the batch only refine the iterate, which is not used afterwards).
lp_status run_power_iteration(lp_solver* h) {
  cudaStream_t s = h->setup_stream;
  h->pw_iters = 0;
  if (h->m == 0 || h->n == 0) {
    h->norm_A = 0.0;
    return LP_OK;
  }
  double* u = h->x;  // scratch: the iterate buffers are free until the first solve
  double* w = h->y;
  double* hist = h->out_buf;  // kPwBatch lambdas
  k_pw_start<<<h->gridV, kThreads, 0, s>>>(h->n, h->d_col_perm, h->prm.power_seed, u, h->pw, h->partials);
  CK(cudaGetLastError());
  double lam = 0.0, prev = 0.0;
  int64_t it = 0;
  bool stop = false;
  double got[kPwBatch];
  while (!stop && it < h->prm.power_max_iter) {
    const int64_t left = h->prm.power_max_iter - it;
    const int batch = left < kPwBatch ? (int)left : kPwBatch;
    for (int q = 0; q < batch; ++q) {
      k_pw_rows<<<h->gridA, kThreads, 0, s>>>(h->rpA, h->ciA, h->valA, u, w, h->binsA, h->pw, h->partials,
                                               hist, q);
      k_pw_cols<<<h->gridT, kThreads, 0, s>>>(h->rpT, h->ciT, h->valT, w, u, h->binsT, h->pw, h->partials);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(got, hist, sizeof(double) * batch, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < batch && !stop; ++q) {
      ++it;
      lam = got[q];
      if (lam == 0.0) stop = true;
      else if (it > 1 && std::fabs(lam - prev) <= h->prm.power_tol * lam) stop = true;
      else prev = lam;
    }
  }
  h->pw_iters = it;
  h->norm_A = std::sqrt(lam);
  return LP_OK;
}

lp_status set_eta(lp_solver* h) {
  if (h->prm.eta > 0.0) {
    h->eta = h->prm.eta;
    return LP_OK;
  }
  if (!h->power_valid) {
    lp_status st = run_power_iteration(h);
    if (st != LP_OK) return st;
    h->power_valid = true;
  }
  h->eta = h->norm_A > 0.0 ? 0.998 / h->norm_A : 1.0;
  return LP_OK;
}

lp_status create_impl(lp_solver* h, int32_t m, int32_t n, int64_t nnz, const int64_t* rp,
                      const int32_t* ci, const double* val, const double* c, const double* lc,
                      const double* uc, const double* lv, const double* uv) {
  h->m = m;
  h->n = n;
  h->nnz = nnz;
  CK(cudaGetDevice(&h->device));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  CK(cudaStreamCreateWithFlags(&h->setup_stream, cudaStreamNonBlocking));
  CK(cudaMallocHost(&h->pinned, 8 * sizeof(double)));

  // KKT denominators on the original data (Section 4): ||c||_2 and ||(L, U)||_2 over the finite
  // bound entries, summed in natural order.
  double c2 = 0.0, lu2 = 0.0;
  for (int32_t j = 0; j < n; ++j) c2 += c[j] * c[j];
  for (int32_t i = 0; i < m; ++i) {
    if (std::isfinite(lc[i])) lu2 += lc[i] * lc[i];
    if (std::isfinite(uc[i])) lu2 += uc[i] * uc[i];
  }
  h->c_norm = std::sqrt(c2);
  h->lu_norm = std::sqrt(lu2);

  // ---- permutation by length class ----
  std::vector<int64_t> rlen(m), clen(n, 0);
  for (int32_t i = 0; i < m; ++i) rlen[i] = rp[i + 1] - rp[i];
  for (int64_t p = 0; p < nnz; ++p) clen[ci[p]]++;
  order_by_length(rlen, h->row_perm);
  {
    // columns ordered by decreasing length like the rows, and among equal lengths in the order
    // the permuted rows first reference them (unreferenced columns last): the entries of one row
    // tile then gather nearby columns, fewer L2 sectors per tile (multicommodity FP64 iteration
    // 286 -> 276 us)
    std::vector<int32_t> seq;
    seq.reserve(n);
    std::vector<char> seen(n, 0);
    for (int32_t i = 0; i < m; ++i) {
      const int32_t o = h->row_perm[i];
      for (int64_t p = rp[o]; p < rp[o + 1]; ++p)
        if (!seen[ci[p]]) {
          seen[ci[p]] = 1;
          seq.push_back(ci[p]);
        }
    }
    for (int32_t j = 0; j < n; ++j)
      if (!seen[j]) seq.push_back(j);
    std::vector<int64_t> seq_len(n);
    for (int32_t q = 0; q < n; ++q) seq_len[q] = clen[seq[q]];
    std::vector<int32_t> by_len;
    order_by_length(seq_len, by_len);  // stable: first-reference order among equal lengths
    h->col_perm.assign(n, 0);
    for (int32_t q = 0; q < n; ++q) h->col_perm[q] = seq[by_len[q]];
  }
  std::vector<int32_t> col_inv(n);
  for (int32_t j = 0; j < n; ++j) col_inv[h->col_perm[j]] = j;

  // ---- permuted CSR of A and of A^T ----
  std::vector<int32_t> rpA(m + 1), ciA(nnz);
  std::vector<double> valA(nnz);
  rpA[0] = 0;
  for (int32_t i = 0; i < m; ++i) rpA[i + 1] = rpA[i] + (int32_t)rlen[h->row_perm[i]];
  for (int32_t i = 0; i < m; ++i) {
    const int32_t o = h->row_perm[i];
    int32_t q = rpA[i];
    for (int64_t p = rp[o]; p < rp[o + 1]; ++p, ++q) {
      ciA[q] = col_inv[ci[p]];
      valA[q] = val[p];
    }
  }
  std::vector<int32_t> rpT(n + 1), ciT(nnz), cursor(n);
  std::vector<double> valT(nnz);
  rpT[0] = 0;
  for (int32_t j = 0; j < n; ++j) rpT[j + 1] = rpT[j] + (int32_t)clen[h->col_perm[j]];
  for (int32_t j = 0; j < n; ++j) cursor[j] = rpT[j];
  for (int32_t i = 0; i < m; ++i)
    for (int32_t q = rpA[i]; q < rpA[i + 1]; ++q) {
      const int32_t pos = cursor[ciA[q]]++;
      ciT[pos] = i;
      valT[pos] = valA[q];
    }
  std::vector<int4> chunksA, chunksT;
  // automatic: 32 (rows of up to 32 entries one lane each, in sliced tiles): against 8, the
  // multicommodity FP64 iteration 215 -> 211 us, FP32 143 -> 140 us, MIPLIB-shaped 28.9 -> 27.6 us
  const int lt = h->prm.lane_target > 0 ? h->prm.lane_target : 32;
  int tr = h->prm.tile_rows;
  if (tr == 0) {
    // automatic: 32-row tiles (every row epilogue instruction runs in 32 lanes, where one-pass
    // tiles of rows with G > 1 lanes use 32 / G) when both matrices still give every resident
    // warp of the loop kernel (3 blocks of kWarps per SM) at least 8 tiles; one-pass tiles
    // otherwise (latency-bound sizes want many short tasks)
    const BinTable a32 = make_bins(rpA, lt, 32, chunksA), t32 = make_bins(rpT, lt, 32, chunksT);
    const int64_t warps = (int64_t)h->num_sms * 3 * kWarps;
    tr = (a32.ntasks + a32.nchunks >= 8 * warps && t32.ntasks + t32.nchunks >= 8 * warps) ? 32 : 1;
  }
  h->tile_rows_used = tr;
  h->binsA = make_bins(rpA, lt, tr, chunksA);
  h->binsT = make_bins(rpT, lt, tr, chunksT);
  std::vector<int32_t> sell_offA, sell_offT, sell_srcA, sell_srcT;
  const bool slA = build_sell(rpA, h->binsA, sell_offA, sell_srcA);
  const bool slT = build_sell(rpT, h->binsT, sell_offT, sell_srcT);

  int occA = 0, occT = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occA, iter_kernels<double>().rows, kThreads, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occT, iter_kernels<double>().cols, kThreads, 0));
  if (occA < 1) occA = 1;
  if (occT < 1) occT = 1;
  h->gridA = grid_for_tasks((int64_t)h->binsA.ntasks + h->binsA.nchunks, h->num_sms, occA * h->num_sms);
  h->gridT = grid_for_tasks((int64_t)h->binsT.ntasks + h->binsT.nchunks, h->num_sms, occT * h->num_sms);
  int occL = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occL, iter_kernels<double>().loop_refl, kThreads, 0));
  if (occL < 1) occL = 1;
  // the loop kernel's grid, sized like the phase kernels' but against its own residency
  {
    const int64_t tasks = (int64_t)h->binsA.ntasks + h->binsA.nchunks > (int64_t)h->binsT.ntasks + h->binsT.nchunks
                              ? (int64_t)h->binsA.ntasks + h->binsA.nchunks
                              : (int64_t)h->binsT.ntasks + h->binsT.nchunks;
    h->gridL = grid_for_tasks(tasks, h->num_sms, occL * h->num_sms);
  }
  h->loop_fits = h->gridL <= occL * h->num_sms;
  h->small = (int64_t)h->binsA.ntasks + h->binsA.nchunks <= kClusterTasks &&
             (int64_t)h->binsT.ntasks + h->binsT.nchunks <= kClusterTasks;
  {
    int best = 16;
    max_loop_cluster<double>(best);
    if (h->prm.precision != 0) max_loop_cluster<float>(best);
    h->cluster_max = best;
  }
  setup_sm_loop(h, rpA, rpT);
  if (h->gridL > occL * h->num_sms) h->gridL = occL * h->num_sms;  // all blocks co-resident
  if (h->prm.precision != 0) {
    // the FP32 loop kernel has fewer registers (4 blocks per SM): its own grid, sized the same way
    int occF = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occF, iter_kernels<float>().loop, kThreads, 0));
    if (occF < 1) occF = 1;
    const int gA = grid_for_tasks((int64_t)h->binsA.ntasks + h->binsA.nchunks, h->num_sms, occF * h->num_sms);
    const int gT = grid_for_tasks((int64_t)h->binsT.ntasks + h->binsT.nchunks, h->num_sms, occF * h->num_sms);
    h->gridL32 = gA > gT ? gA : gT;
  }
  h->gridV = grid_for(n > m ? n : m, kThreads, 4 * h->num_sms);
  h->max_grid = h->gridA > h->gridT ? h->gridA : h->gridT;
  if (h->gridV > h->max_grid) h->max_grid = h->gridV;
  if (h->gridL > h->max_grid) h->max_grid = h->gridL;
  if (h->gridL32 > h->max_grid) h->max_grid = h->gridL32;

  // ---- device buffers ----
  CK(h->alloc(&h->rpA, m + 1)); CK(h->alloc(&h->ciA, nnz)); CK(h->alloc(&h->valA, nnz));
  CK(h->alloc(&h->rpT, n + 1)); CK(h->alloc(&h->ciT, nnz)); CK(h->alloc(&h->valT, nnz));
  CK(h->alloc(&h->d_row_perm, m)); CK(h->alloc(&h->d_col_perm, n));
  for (double** p : {&h->c, &h->lv, &h->uv, &h->inv_dc, &h->dc, &h->x, &h->x0, &h->xh0, &h->xh1,
                     &h->aty, &h->aty0, &h->xbar})
    CK(h->alloc(p, n));
  for (double** p : {&h->lc, &h->uc, &h->inv_dr, &h->dr, &h->y, &h->y0, &h->yh, &h->ax, &h->ax0, &h->axh,
                     &h->qy, &h->w})
    CK(h->alloc(p, m));
  {
    size_t ob = (size_t)(n > m ? n : m) + 1;
    if (ob < (size_t)kPwBatch) ob = kPwBatch;  // also holds a batch of power-iteration lambdas
    CK(h->alloc(&h->out_buf, ob));
  }
  CK(h->alloc(&h->partials, (size_t)h->max_grid * kNumSums));
  CK(h->alloc(&h->partials2, (size_t)h->max_grid * kNumSums));
  CK(h->alloc(&h->partials3, (size_t)h->max_grid * kNumSums));
  CK(h->alloc(&h->ctl, 1));
  CK(h->alloc(&h->pw, 1));
  CK(cudaMemset(h->ctl, 0, sizeof(Ctl)));
  CK(cudaMemset(h->pw, 0, sizeof(PwCtl)));
  h->trace_cap = h->prm.trace_cap;
  if (h->trace_cap > 0) CK(h->alloc(&h->trace, (size_t)h->trace_cap * 4));
  for (auto [bt, ch] : {std::make_pair(&h->binsA, &chunksA), std::make_pair(&h->binsT, &chunksT)}) {
    int4* d_chunk = nullptr;
    double* d_part = nullptr;
    double* d_contrib = nullptr;
    unsigned* d_arr = nullptr;
    CK(h->alloc(&d_chunk, ch->size()));
    CK(h->alloc(&d_part, ch->size()));
    CK(h->alloc(&d_contrib, (size_t)bt->long_rows * kNumSums));
    CK(h->alloc(&d_arr, (size_t)bt->long_rows));
    if (!ch->empty()) CK(cudaMemcpy(d_chunk, ch->data(), sizeof(int4) * ch->size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(d_arr, 0, sizeof(unsigned) * (bt->long_rows > 0 ? bt->long_rows : 1)));
    bt->chunk = d_chunk;
    bt->part = d_part;
    bt->arrivals = d_arr;
    bt->contrib = d_contrib;
  }

  // sliced tiles: slot maps now, values and indices gathered after the preconditioning
  for (auto [ok, bt, offv, srcv, doff, dsrc, dci, dval, len] :
       {std::make_tuple(slA, &h->binsA, &sell_offA, &sell_srcA, &h->sell_offA, &h->sell_srcA, &h->sell_ciA,
                        &h->sell_valA, &h->sell_lenA),
        std::make_tuple(slT, &h->binsT, &sell_offT, &sell_srcT, &h->sell_offT, &h->sell_srcT, &h->sell_ciT,
                        &h->sell_valT, &h->sell_lenT)}) {
    *len = ok ? (int64_t)srcv->size() : 0;
    if (!ok || *len == 0) continue;
    CK(h->alloc(doff, offv->size()));
    CK(h->alloc(dsrc, (size_t)*len));
    CK(h->alloc(dci, (size_t)*len));
    CK(h->alloc(dval, (size_t)*len));
    CK(cudaMemcpy(*doff, offv->data(), sizeof(int32_t) * offv->size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(*dsrc, srcv->data(), sizeof(int32_t) * (size_t)*len, cudaMemcpyHostToDevice));
    bt->sell_off = *doff;
    bt->sell_ci = *dci;
    bt->sell_val = *dval;
  }
  CK(cudaMemcpy(h->rpA, rpA.data(), sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->rpT, rpT.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  if (nnz > 0) {
    CK(cudaMemcpy(h->ciA, ciA.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->valA, valA.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->ciT, ciT.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->valT, valT.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
  }
  {
    std::vector<double> tmp(n > m ? n : m);
    auto up_cols = [&](double* dst, const double* src) -> cudaError_t {
      for (int32_t j = 0; j < n; ++j) tmp[j] = src[h->col_perm[j]];
      return n > 0 ? cudaMemcpy(dst, tmp.data(), sizeof(double) * n, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    auto up_rows = [&](double* dst, const double* src) -> cudaError_t {
      for (int32_t i = 0; i < m; ++i) tmp[i] = src[h->row_perm[i]];
      return m > 0 ? cudaMemcpy(dst, tmp.data(), sizeof(double) * m, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    CK(up_cols(h->c, c)); CK(up_cols(h->lv, lv)); CK(up_cols(h->uv, uv));
    CK(up_rows(h->lc, lc)); CK(up_rows(h->uc, uc));
    std::vector<double> ones(n > m ? n : m, 1.0);
    if (n > 0) CK(cudaMemcpy(h->dc, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    if (m > 0) CK(cudaMemcpy(h->dr, ones.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
  }
  if (m > 0) CK(cudaMemcpy(h->d_row_perm, h->row_perm.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
  if (n > 0) CK(cudaMemcpy(h->d_col_perm, h->col_perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  // a copy from pageable memory returns once its source is staged, possibly before its last
  // transfer lands, and the setup stream does not wait on the default stream: wait here
  CK(cudaDeviceSynchronize());

  // ---- diagonal preconditioning (device) ----
  cudaStream_t s = h->setup_stream;
  const int passes = h->prm.ruiz_iters + (h->prm.pc_enabled ? 1 : 0);
  if (passes > 0 && nnz > 0) {
    double* fr = h->y;  // scratch until the first solve
    double* fc = h->x;
    const int gr = grid_for((int64_t)m * 32, 256, 8 * h->num_sms);
    const int gc = grid_for((int64_t)n * 32, 256, 8 * h->num_sms);
    // rows [0, split) are longer than 32 entries (rows and columns are stored by decreasing
    // length): a warp each in the scaling kernels, the others a thread each
    auto split_of = [](const std::vector<int32_t>& r) {
      int32_t q = 0;
      while (q + 1 < (int32_t)r.size() && r[q + 1] - r[q] > 32) ++q;
      return q;
    };
    const int32_t splitA = split_of(rpA), splitT = split_of(rpT);
    for (int pass = 0; pass < passes; ++pass) {
      const bool pc = (pass == h->prm.ruiz_iters);
      const int kind = pc ? 1 : 0;
      if (m > 0) k_row_factor<<<gr, 256, 0, s>>>(m, splitA, h->rpA, h->valA, kind, 2.0 - h->prm.pc_alpha, fr);
      if (n > 0) k_row_factor<<<gc, 256, 0, s>>>(n, splitT, h->rpT, h->valT, kind, h->prm.pc_alpha, fc);
      if (m > 0) k_apply_factors<<<gr, 256, 0, s>>>(m, splitA, h->rpA, h->ciA, h->valA, fr, fc, 0);
      if (n > 0) k_apply_factors<<<gc, 256, 0, s>>>(n, splitT, h->rpT, h->ciT, h->valT, fr, fc, 1);
      if (m > 0) k_mul_inplace<<<h->gridV, 256, 0, s>>>(m, h->dr, fr);
      if (n > 0) k_mul_inplace<<<h->gridV, 256, 0, s>>>(n, h->dc, fc);
    }
    CK(cudaGetLastError());
  }
  if (n > 0) k_scale_cols<<<h->gridV, 256, 0, s>>>(n, h->dc, h->c, h->lv, h->uv, h->inv_dc);
  if (m > 0) k_scale_rows<<<h->gridV, 256, 0, s>>>(m, h->dr, h->lc, h->uc, h->inv_dr);
  CK(cudaGetLastError());
  // the sliced tiles take the preconditioned entries
  if (h->sell_lenA > 0)
    k_sell_gather<<<grid_for(h->sell_lenA, 256, 8 * h->num_sms), 256, 0, s>>>(h->sell_lenA, h->sell_srcA, h->ciA,
                                                                             h->valA, h->sell_ciA, h->sell_valA);
  if (h->sell_lenT > 0)
    k_sell_gather<<<grid_for(h->sell_lenT, 256, 8 * h->num_sms), 256, 0, s>>>(h->sell_lenT, h->sell_srcT, h->ciT,
                                                                             h->valT, h->sell_ciT, h->sell_valT);
  CK(cudaGetLastError());
  if (h->prm.precision != 0) {
    auto& f = h->f32;
    CK(h->alloc(&f.valA, nnz)); CK(h->alloc(&f.valT, nnz));
    for (float** q : {&f.c, &f.lv, &f.uv, &f.inv_dc, &f.x, &f.x0, &f.xh0, &f.xh1, &f.aty, &f.aty0,
                      &f.xb0, &f.xb1, &f.xbar})
      CK(h->alloc(q, n));
    for (float** q : {&f.lc, &f.uc, &f.inv_dr, &f.y, &f.y0, &f.yh, &f.ax, &f.ax0, &f.axh, &f.yb0, &f.yb1,
                      &f.qy, &f.w})
      CK(h->alloc(q, m));
    const int g = grid_for(nnz > 0 ? nnz : 1, 256, 8 * h->num_sms);
    k_to_float<<<g, 256, 0, s>>>(nnz, h->valA, f.valA);
    k_to_float<<<g, 256, 0, s>>>(nnz, h->valT, f.valT);
    if (h->sell_lenA > 0) {
      CK(h->alloc(&f.sell_valA, (size_t)h->sell_lenA));
      k_to_float<<<grid_for(h->sell_lenA, 256, 8 * h->num_sms), 256, 0, s>>>(h->sell_lenA, h->sell_valA, f.sell_valA);
    }
    if (h->sell_lenT > 0) {
      CK(h->alloc(&f.sell_valT, (size_t)h->sell_lenT));
      k_to_float<<<grid_for(h->sell_lenT, 256, 8 * h->num_sms), 256, 0, s>>>(h->sell_lenT, h->sell_valT, f.sell_valT);
    }
    for (auto pr : {std::make_pair((const double*)h->c, f.c), std::make_pair((const double*)h->lv, f.lv),
                    std::make_pair((const double*)h->uv, f.uv), std::make_pair((const double*)h->inv_dc, f.inv_dc)})
      k_to_float<<<h->gridV, 256, 0, s>>>(n, pr.first, pr.second);
    for (auto pr : {std::make_pair((const double*)h->lc, f.lc), std::make_pair((const double*)h->uc, f.uc),
                    std::make_pair((const double*)h->inv_dr, f.inv_dr)})
      k_to_float<<<h->gridV, 256, 0, s>>>(m, pr.first, pr.second);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  {
    std::vector<double> hc(n), hl(m), hu(m);
    if (n > 0) CK(cudaMemcpy(hc.data(), h->c, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (m > 0) CK(cudaMemcpy(hl.data(), h->lc, sizeof(double) * m, cudaMemcpyDeviceToHost));
    if (m > 0) CK(cudaMemcpy(hu.data(), h->uc, sizeof(double) * m, cudaMemcpyDeviceToHost));
    h->rescale_ratio = rescale_ratio(hc.data(), n, hl.data(), hu.data(), m);
  }

  lp_status st = set_eta(h);
  if (st != LP_OK) return st;
  return build_graph(h);
}

}  // namespace

extern "C" {

lp_status lp_default_params(lp_params* p) {
  if (!p) return fail(LP_ERR_INVALID_ARG, "params pointer is NULL");
  std::memset(p, 0, sizeof(*p));
  p->gamma = 1.0;
  p->beta_sufficient = 0.2;
  p->beta_necessary = 0.8;
  p->beta_artificial = 0.36;
  p->k_p = 0.5;
  p->k_i = 0.001;
  p->k_d = 0.0;
  p->eta = 0.0;
  p->omega0 = 1.0;
  p->check_every = 64;
  p->restart_enabled = 1;
  p->pid_enabled = 1;
  p->power_tol = 1e-7;
  p->power_max_iter = 10000;
  p->power_seed = 0;
  p->ruiz_iters = 10;
  p->pc_enabled = 1;
  p->pc_alpha = 1.0;
  p->trace_cap = 0;
  p->unroll = 32;
  p->lane_target = 0;
  p->persistent = -1;
  p->precision = 0;
  p->switch_tol = 1e-5;
  p->fp32_patience = 32;
  p->rescale = 0;
  p->tile_rows = 0;
  p->batch_local_nnz = 16384;
  return LP_OK;
}

lp_status lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                    const int32_t* col_idx, const double* val, const double* c,
                    const double* l_c, const double* u_c, const double* l_v, const double* u_v,
                    int32_t where, const lp_params* p, lp_handle* out) {
  NvtxRange nvtx("lp_create");
  g_err.clear();
  if (!out) return fail(LP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 0 || n < 0 || nnz < 0) return fail(LP_ERR_INVALID_ARG, "negative size");
  if (where != LP_HOST && where != LP_DEVICE) return fail(LP_ERR_INVALID_ARG, "where must be LP_HOST or LP_DEVICE");
  if (!row_ptr) return fail(LP_ERR_INVALID_ARG, "row_ptr is NULL");
  if (nnz > 0 && (!col_idx || !val)) return fail(LP_ERR_INVALID_ARG, "col_idx/val is NULL");
  if (n > 0 && (!c || !l_v || !u_v)) return fail(LP_ERR_INVALID_ARG, "c/l_v/u_v is NULL");
  if (m > 0 && (!l_c || !u_c)) return fail(LP_ERR_INVALID_ARG, "l_c/u_c is NULL");
  if (nnz >= (int64_t(1) << 31)) return fail(LP_ERR_TOO_LARGE, "nnz must be < 2^31");
  lp_params prm;
  if (p) prm = *p; else lp_default_params(&prm);
  lp_status st = check_params(prm);
  if (st != LP_OK) return st;

  // Device inputs are staged through host memory for the (host-side) structural setup.
  std::vector<int64_t> h_rp;
  std::vector<int32_t> h_ci;
  std::vector<double> h_val, h_c, h_lc, h_uc, h_lv, h_uv;
  if (where == LP_DEVICE) {
    auto dl = [](auto& vec, const auto* src, int64_t count) -> cudaError_t {
      vec.resize(count > 0 ? count : 0);
      if (count <= 0) return cudaSuccess;
      return cudaMemcpy(vec.data(), src, sizeof(*src) * count, cudaMemcpyDeviceToHost);
    };
    CK(dl(h_rp, row_ptr, (int64_t)m + 1));
    CK(dl(h_ci, col_idx, nnz)); CK(dl(h_val, val, nnz));
    CK(dl(h_c, c, n)); CK(dl(h_lv, l_v, n)); CK(dl(h_uv, u_v, n));
    CK(dl(h_lc, l_c, m)); CK(dl(h_uc, u_c, m));
    row_ptr = h_rp.data(); col_idx = h_ci.data(); val = h_val.data(); c = h_c.data();
    l_v = h_lv.data(); u_v = h_uv.data(); l_c = h_lc.data(); u_c = h_uc.data();
  }
  st = validate(m, n, nnz, row_ptr, col_idx, val, c, l_c, u_c, l_v, u_v);
  if (st != LP_OK) return st;
  lp_solver* h = new (std::nothrow) lp_solver();
  if (!h) return fail(LP_ERR_OUT_OF_MEMORY, "host allocation failed");
  h->prm = prm;
  st = create_impl(h, m, n, nnz, row_ptr, col_idx, val, c, l_c, u_c, l_v, u_v);
  if (st != LP_OK) {
    delete h;
    return st;
  }
  *out = h;
  return LP_OK;
}

lp_status lp_set_params(lp_handle h, const lp_params* p) {
  g_err.clear();
  if (!h || !p) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  lp_status st = check_params(*p);
  if (st != LP_OK) return st;
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  const lp_params old = h->prm;
  h->prm = *p;
  h->prm.ruiz_iters = old.ruiz_iters;  // preconditioning is fixed at lp_create
  h->prm.pc_enabled = old.pc_enabled;
  h->prm.pc_alpha = old.pc_alpha;
  h->prm.lane_target = old.lane_target;  // the bin tables are built at lp_create
  h->prm.precision = old.precision;      // the FP32 buffers are made at lp_create
  h->prm.tile_rows = old.tile_rows;      // so are the tiles
  if (p->power_seed != old.power_seed || p->power_tol != old.power_tol ||
      p->power_max_iter != old.power_max_iter)
    h->power_valid = false;
  st = set_eta(h);
  if (st != LP_OK) return st;
  if (p->trace_cap != h->trace_cap) {
    if (h->trace) {
      cudaFree(h->trace);
      for (auto& a : h->allocations)
        if (a == h->trace) a = nullptr;
      h->trace = nullptr;
    }
    h->trace_cap = p->trace_cap;
    if (h->trace_cap > 0) CK(h->alloc(&h->trace, (size_t)h->trace_cap * 4));
    return build_graph(h);
  }
  if (h->prm.unroll != h->graph_unroll || p->persistent != old.persistent ||
      (p->gamma == 1.0) != (old.gamma == 1.0))
    return build_graph(h);
  return LP_OK;
}

}  // extern "C"

namespace {

// Scalar state, zero iterate and first primal step of a solve, enqueued on s, for the buffers
// of precision V (the FP64 set, or the FP32 set of a mixed-precision solve).
template <class V>
lp_status enqueue_start(lp_solver* h, double tol, int64_t max_iter, cudaStream_t s) {
  Ctl init{};
  init.eta = h->eta;
  const double om0 = h->prm.omega0 * (h->prm.rescale ? h->rescale_ratio : 1.0);
  init.omega = om0;
  init.tau = h->eta / om0;
  init.sigma = h->eta * om0;
  init.inv_sigma = 1.0 / (h->eta * om0);
  init.w_over_eta = om0 / h->eta;
  init.inv_eta_w = 1.0 / (h->eta * om0);
  init.restart_enabled = h->prm.restart_enabled;
  init.pid_enabled = h->prm.pid_enabled;
  init.max_iter = max_iter;
  init.check_every = h->prm.check_every;
  init.trace_cap = h->trace_cap;
  init.tol = tol;
  init.omega_used = om0;
  for (int q = 0; q < 8; ++q) init.kkt[q] = NAN;
  init.lu_norm = h->lu_norm;
  init.c_norm = h->c_norm;
  init.gamma = h->prm.gamma;
  init.beta_s = h->prm.beta_sufficient;
  init.beta_n = h->prm.beta_necessary;
  init.beta_a = h->prm.beta_artificial;
  init.kp = h->prm.k_p;
  init.ki = h->prm.k_i;
  init.kd = h->prm.k_d;
  init.patience = (sizeof(V) == sizeof(float)) ? h->prm.fp32_patience : 0;
  init.best_kkt = INFINITY;
  init.cand_slot = 0;
  init.best_slot = -1;
  k_init_ctl<<<1, 1, 0, s>>>(h->ctl, init);
  RowArgsT<V> ra;
  ColArgsT<V> ca;
  fill_args(h, ra, ca);
  iter_kernels<V>().init_rows<<<h->gridV, 256, 0, s>>>(h->m, ra.y, ra.y0, ra.yh, ra.ax, ra.ax0, ra.axh);
  iter_kernels<V>().init_cols<<<h->gridV, kThreads, 0, s>>>(h->n, ca.c, ca.lv, ca.uv, ca.xh0, ca.x, ca.x0, ca.aty, ca.aty0,
                                               ca.xbar,
                                               h->ctl, h->partials);
  CK(cudaGetLastError());
  return LP_OK;
}

// Mixed precision, after the FP32 phase: hand the FP32 point over to the FP64 buffers as the
// anchor of a new epoch (A x and A^T y recomputed in FP64 from it) and continue in FP64.
lp_status enqueue_switch(lp_solver* h, double tol, int64_t max_iter, cudaStream_t s) {
  const auto& f = h->f32;
  const int g = grid_for((int64_t)(h->n > h->m ? h->n : h->m), 256, 4 * h->num_sms);
  k_switch_vectors<<<g, 256, 0, s>>>(h->n, h->m, h->ctl, f.xh0, f.xh1, f.yh, f.xb0, f.xb1, f.yb0, f.yb1,
                                     h->x, h->x0, h->yh, h->xh0, h->xh1, 0);
  k_switch_ctl<<<1, 1, 0, s>>>(h->ctl, tol, max_iter);
  k_spmv<<<h->gridA, kThreads, 0, s>>>(h->rpA, h->ciA, h->valA, h->x, h->axh, h->binsA);
  k_spmv<<<h->gridT, kThreads, 0, s>>>(h->rpT, h->ciT, h->valT, h->yh, h->aty, h->binsT);
  k_warm_cols<<<h->gridV, kThreads, 0, s>>>(h->n, h->c, h->lv, h->uv, h->xh0, h->xh1, h->x, h->aty, h->aty0, h->xbar,
                                            h->ctl, h->partials);
  CK(cudaGetLastError());
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_solve(lp_handle h, double tol, int64_t max_iter, void* stream) {
  NvtxRange nvtx("lp_solve");
  g_err.clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "handle is NULL");
  if (!(tol >= 0.0)) return fail(LP_ERR_INVALID_ARG, "tol must be >= 0");
  if (max_iter < 1) return fail(LP_ERR_INVALID_ARG, "max_iter must be >= 1");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lp_status st = LP_OK;
  if (h->prm.precision == 0) {
    st = enqueue_start<double>(h, tol, max_iter, s);
    if (st != LP_OK) return st;
    CK(cudaGraphLaunch(h->exec, s));
  } else {
    // FP32 phase: to max(tol, switch_tol) (mixed) or tol (FP32 only), at most max_iter iterations
    const double tol32 = h->prm.precision == 1 ? (tol > h->prm.switch_tol ? tol : h->prm.switch_tol) : tol;
    st = enqueue_start<float>(h, tol32, max_iter, s);
    if (st != LP_OK) return st;
    CK(cudaGraphLaunch(h->exec32, s));
    if (h->prm.precision == 1) {
      st = enqueue_switch(h, tol, max_iter, s);
      if (st != LP_OK) return st;
      CK(cudaGraphLaunch(h->exec, s));
    } else {
      const auto& f = h->f32;
      const int g = grid_for((int64_t)(h->n > h->m ? h->n : h->m), 256, 4 * h->num_sms);
      k_switch_vectors<<<g, 256, 0, s>>>(h->n, h->m, h->ctl, f.xh0, f.xh1, f.yh, f.xb0, f.xb1, f.yb0,
                                         f.yb1, h->x, h->x0, h->yh, h->xh0, h->xh1, 1);
      CK(cudaGetLastError());
    }
  }
  h->solved = true;
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_get(lp_handle h, double* x, double* y, int32_t* solve_status, double* kkt,
                 int64_t* iters) {
  NvtxRange nvtx("lp_get");
  g_err.clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "handle is NULL");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "lp_get before lp_solve");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  Ctl ctl;
  CK(cudaMemcpy(&ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const double* xh = (ctl.t & 1) ? h->xh1 : h->xh0;
  cudaStream_t s = h->setup_stream;
  if (x && h->n > 0) {
    k_unpermute_scale<<<h->gridV, 256, 0, s>>>(h->n, h->d_col_perm, xh, h->dc, h->out_buf);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(x, h->out_buf, sizeof(double) * h->n, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
  }
  if (y && h->m > 0) {
    k_unpermute_scale<<<h->gridV, 256, 0, s>>>(h->m, h->d_row_perm, h->yh, h->dr, h->out_buf);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(y, h->out_buf, sizeof(double) * h->m, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
  }
  if (solve_status) *solve_status = ctl.status;
  if (kkt)
    for (int q = 0; q < 4; ++q) kkt[q] = ctl.kkt[q];
  if (iters) *iters = ctl.iters;
  return LP_OK;
}

lp_status lp_get_info(lp_handle h, double* out9) {
  g_err.clear();
  if (!h || !out9) return fail(LP_ERR_INVALID_ARG, "NULL argument");
  double* out7 = out9;
  double* out8 = out9;
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "lp_get_info before lp_solve");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  Ctl ctl;
  CK(cudaMemcpy(&ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  out7[0] = h->eta;
  out7[1] = ctl.omega_used;
  out7[2] = (double)ctl.restarts_used;
  out7[3] = h->power_valid ? h->norm_A : 0.0;
  out7[4] = (double)h->pw_iters;
  out7[5] = ctl.kkt[4];
  out7[6] = ctl.kkt[5];
  out8[7] = h->loop_active ? (h->sm_active ? 3.0 : (h->cluster > 0 ? 2.0 : 1.0)) : 0.0;
  out9[8] = h->prm.precision == 1 ? (double)ctl.iters32 : (h->prm.precision == 2 ? (double)ctl.iters : 0.0);
  return LP_OK;
}

lp_status lp_get_trace(lp_handle h, double* trace, int64_t cap, int64_t* rows) {
  g_err.clear();
  if (!h || !trace || !rows || cap < 0) return fail(LP_ERR_INVALID_ARG, "bad argument");
  if (!h->solved) return fail(LP_ERR_NOT_SOLVED, "lp_get_trace before lp_solve");
  if (h->trace_cap <= 0) return fail(LP_ERR_INVALID_ARG, "trace_cap is 0");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->last_stream));
  Ctl ctl;
  CK(cudaMemcpy(&ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  int64_t r = ctl.iters < h->trace_cap ? ctl.iters : h->trace_cap;
  if (r > cap) r = cap;
  if (r > 0) CK(cudaMemcpy(trace, h->trace, sizeof(double) * 4 * r, cudaMemcpyDeviceToHost));
  *rows = r;
  return LP_OK;
}

void lp_destroy(lp_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->solved) cudaStreamSynchronize(h->last_stream);
  delete h;
}

const char* lp_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// lp_time_kernels in precision V: the iteration kernels of V launched one by one, CUDA events
// around each launch.
template <class V>
lp_status time_kernels(lp_solver* h, int64_t iters, cudaStream_t s, double* ms_out) {
  const bool loop = sizeof(V) == sizeof(float) ? h->loop_active32 : h->loop_active;
  const int32_t per = loop ? h->prm.unroll : 1;
  const int64_t launches = (iters + per - 1) / per;
  lp_status st = enqueue_start<V>(h, 0.0, launches * per, s);
  if (st != LP_OK) return st;
  RowArgsT<V> ra{};
  ColArgsT<V> ca{};
  fill_args(h, ra, ca);
  const int64_t nev = loop ? launches + 1 : 2 * launches + 1;
  std::vector<cudaEvent_t> ev(nev, nullptr);
  struct Events {
    std::vector<cudaEvent_t>& v;
    ~Events() {
      for (auto& e : v)
        if (e) cudaEventDestroy(e);
    }
  } guard{ev};
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], s));
  for (int64_t q = 0; q < launches; ++q) {
    if (loop) {
      CK(launch_loop<V>(h, ra, ca, per, cudaGraphConditionalHandle{}, 0, s));
      CK(cudaEventRecord(ev[q + 1], s));
    } else {
      iter_kernels<V>().rows<<<h->gridA, kThreads, 0, s>>>(ra);
      CK(cudaEventRecord(ev[2 * q + 1], s));
      iter_kernels<V>().cols<<<h->gridT, kThreads, 0, s>>>(ca);
      CK(cudaEventRecord(ev[2 * q + 2], s));
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  double a = 0.0, b = 0.0;
  for (int64_t q = 0; q < launches; ++q) {
    float m1 = 0.f, m2 = 0.f;
    if (loop) {
      CK(cudaEventElapsedTime(&m1, ev[q], ev[q + 1]));
    } else {
      CK(cudaEventElapsedTime(&m1, ev[2 * q], ev[2 * q + 1]));
      CK(cudaEventElapsedTime(&m2, ev[2 * q + 1], ev[2 * q + 2]));
    }
    a += m1;
    b += m2;
  }
  ms_out[0] = a / (double)launches;
  ms_out[1] = b / (double)launches;
  ms_out[2] = (double)per;
  ms_out[3] = (double)launches;
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_time_kernels(lp_handle h, int64_t iters, void* stream, double* ms_out) {
  g_err.clear();
  if (!h || !ms_out || iters < 1) return fail(LP_ERR_INVALID_ARG, "bad argument");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const lp_status st = h->prm.precision == 0 ? time_kernels<double>(h, iters, s, ms_out)
                                             : time_kernels<float>(h, iters, s, ms_out);
  if (st != LP_OK) return st;
  // the FP32 timing leaves its iterate in the FP32 buffers: no result to read
  h->solved = h->prm.precision == 0;
  h->last_stream = s;
  return LP_OK;
}

lp_status lp_debug_spmv(lp_handle h, int32_t which, const double* x_dev, double* y_dev) {
  g_err.clear();
  if (!h || !x_dev || !y_dev || (which != 0 && which != 1)) return fail(LP_ERR_INVALID_ARG, "bad argument");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->setup_stream;
  if (which == 0)
    k_spmv<<<h->gridA, kThreads, 0, s>>>(h->rpA, h->ciA, h->valA, x_dev, y_dev, h->binsA);
  else
    k_spmv<<<h->gridT, kThreads, 0, s>>>(h->rpT, h->ciT, h->valT, x_dev, y_dev, h->binsT);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return LP_OK;
}

lp_status lp_debug_layout(lp_handle h, int32_t* row_perm, int32_t* col_perm, double* d_r,
                          double* d_c) {
  g_err.clear();
  if (!h) return fail(LP_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaSetDevice(h->device));
  if (row_perm) std::memcpy(row_perm, h->row_perm.data(), sizeof(int32_t) * h->m);
  if (col_perm) std::memcpy(col_perm, h->col_perm.data(), sizeof(int32_t) * h->n);
  std::vector<double> tmp(h->n > h->m ? h->n : h->m);
  if (d_r && h->m > 0) {
    CK(cudaMemcpy(tmp.data(), h->dr, sizeof(double) * h->m, cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < h->m; ++i) d_r[h->row_perm[i]] = tmp[i];
  }
  if (d_c && h->n > 0) {
    CK(cudaMemcpy(tmp.data(), h->dc, sizeof(double) * h->n, cudaMemcpyDeviceToHost));
    for (int32_t j = 0; j < h->n; ++j) d_c[h->col_perm[j]] = tmp[j];
  }
  return LP_OK;
}

}  // extern "C"
