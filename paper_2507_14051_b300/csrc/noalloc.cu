// ||A||_2 by power iteration without any device allocation (lp_power_norm_noalloc in lp.h).
//
// This is the power iteration that lp_create runs, for callers that cannot allocate device
// memory: all of its scratch -- the two iterate vectors, the product A u, the per-block
// partial sums, the scalars and a short history of the estimates -- lives in one file-scope
// static device array that the library reserves on every device that loads it, for the life
// of the process.  The matrix is the caller's CSR of A as given (no transpose, no binning):
// A u is a warp per row, and A^T w is a scatter with atomic adds, so its last bits depend on
// the order of those adds.  The caller's CSR is checked inside the kernels as it is read: an
// entry outside [0, nnz) or a column index outside [0, n) is skipped and raises a flag, which
// the host turns into LP_ERR_INVALID_INPUT.
#include <cmath>
#include <cstring>
#include <string>

#include "lp.h"
#include "device.cuh"

namespace pdhg {
namespace {

constexpr int64_t kNaMaxDim = int64_t(1) << 18;  // m and n at most 262144
constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;
constexpr int kNaBatch = 16;  // power steps per host synchronisation
// layout (doubles): u[kNaMaxDim] | v[kNaMaxDim] | w[kNaMaxDim] | partials[kNaMaxBlocks] |
// ctl[16] | hist[kNaBatch] (the estimate of each step of the current batch)
constexpr int64_t kNaOffU = 0, kNaOffV = kNaMaxDim, kNaOffW = 2 * kNaMaxDim;
constexpr int64_t kNaOffPart = 3 * kNaMaxDim, kNaOffCtl = 3 * kNaMaxDim + kNaMaxBlocks;
constexpr int64_t kNaOffHist = kNaOffCtl + 16;
constexpr int64_t kNaTotal = kNaOffHist + kNaBatch;

static __device__ __align__(256) double g_na_scratch[kNaTotal];

// ctl slots: 0 lambda of the last step, 1 s (= 1/|u|); slot 2 holds an unsigned arrival
// counter, slot 3 an unsigned flag (nonzero: the CSR had an entry out of range)
struct NaPtrs {
  double* base;
  __host__ __device__ double* u() const { return base + kNaOffU; }
  __host__ __device__ double* v() const { return base + kNaOffV; }
  __host__ __device__ double* w() const { return base + kNaOffW; }
  __host__ __device__ double* part() const { return base + kNaOffPart; }
  __host__ __device__ double* ctl() const { return base + kNaOffCtl; }
  __host__ __device__ double* hist() const { return base + kNaOffHist; }
  __host__ __device__ unsigned* counter() const { return reinterpret_cast<unsigned*>(base + kNaOffCtl + 2); }
  __host__ __device__ unsigned* bad() const { return reinterpret_cast<unsigned*>(base + kNaOffCtl + 3); }
};

// Block sum of one value per thread (fixed-order tree); the last block to arrive writes
// f(total) to *dst and rewinds the arrival counter.
template <class F>
__device__ __forceinline__ void na_block_total(double v, NaPtrs p, double* dst, F f) {
  __shared__ double red[kNaThreads];
  __shared__ bool last;
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int k = kNaThreads / 2; k > 0; k >>= 1) {
    if (tid < k) red[tid] += red[tid + k];
    __syncthreads();
  }
  if (tid == 0) {
    p.part()[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(p.counter(), 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  red[tid] = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += kNaThreads) red[tid] += __ldcg(p.part() + b);
  __syncthreads();
  for (int k = kNaThreads / 2; k > 0; k >>= 1) {
    if (tid < k) red[tid] += red[tid + k];
    __syncthreads();
  }
  if (tid == 0) {
    *dst = f(red[0]);
    *p.counter() = 0u;
  }
}

__device__ __forceinline__ double na_start_entry(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;  // splitmix64, as in setup.cu
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Row i's entry range [b, e), clipped to [0, nnz); raises the flag if the offsets are out of
// range or decreasing (the row is then read as clipped, or skipped).
__device__ __forceinline__ void na_row_range(const int64_t* __restrict__ rp, int64_t i, int64_t nnz, NaPtrs p,
                                             int lane, int64_t& b, int64_t& e) {
  b = rp[i];
  e = rp[i + 1];
  if (b < 0 || e > nnz || b > e) {
    if (lane == 0) atomicOr(p.bad(), 1u);
    b = b < 0 ? 0 : (b > nnz ? nnz : b);
    e = e < b ? b : (e > nnz ? nnz : e);
  }
}

// u = start vector (original column order), s = 1/|u|; clears the flag.
__global__ void __launch_bounds__(kNaThreads) na_start(int32_t n, uint64_t seed, NaPtrs p) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.bad() = 0u;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)kNaThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kNaThreads) {
    const double e = na_start_entry(seed, (uint64_t)j);
    p.u()[j] = e;
    acc = fma(e, e, acc);
  }
  na_block_total(acc, p, p.ctl() + 1, [](double t) { return t > 0.0 ? 1.0 / sqrt(t) : 0.0; });
}

// w = s * (A u) (warp per row), lambda = |w|^2 (also stored as hist[q]); v <- 0 for the
// scatter that follows.  Entries with a column index outside [0, n) are skipped.
__global__ void __launch_bounds__(kNaThreads) na_rows(int32_t m, int32_t n, int64_t nnz,
                                                      const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci,
                                                      const double* __restrict__ val, NaPtrs p,
                                                      const double* __restrict__ u, double* __restrict__ v,
                                                      int32_t q) {
  const double sc = p.ctl()[1];
  for (int64_t j = blockIdx.x * (int64_t)kNaThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kNaThreads)
    v[j] = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kNaThreads / 32);
  double acc = 0.0;
  for (int64_t i = (blockIdx.x * (int64_t)kNaThreads + threadIdx.x) >> 5; i < m; i += nw) {
    int64_t b, e;
    na_row_range(rp, i, nnz, p, lane, b, e);
    double d = 0.0;
    for (int64_t k = b + lane; k < e; k += 32) {
      const int32_t j = ci[k];
      if (j >= 0 && j < n) d = fma(val[k], u[j], d);
      else atomicOr(p.bad(), 1u);
    }
    d = warp_sum(d) * sc;
    if (lane == 0) {
      p.w()[i] = d;
      acc = fma(d, d, acc);
    }
  }
  double* hq = p.hist() + q;
  na_block_total(acc, p, p.ctl() + 0, [hq](double t) {
    *hq = t;
    return t;
  });
}

// v += A^T w (scatter, warp per row; out-of-range entries skipped).
__global__ void __launch_bounds__(kNaThreads) na_scatter(int32_t m, int32_t n, int64_t nnz,
                                                         const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci,
                                                         const double* __restrict__ val, NaPtrs p,
                                                         double* __restrict__ v) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kNaThreads / 32);
  for (int64_t i = (blockIdx.x * (int64_t)kNaThreads + threadIdx.x) >> 5; i < m; i += nw) {
    const double wi = p.w()[i];
    int64_t b, e;
    na_row_range(rp, i, nnz, p, lane, b, e);
    for (int64_t k = b + lane; k < e; k += 32) {
      const int32_t j = ci[k];
      if (j >= 0 && j < n) atomicAdd(v + j, val[k] * wi);
    }
  }
}

// s = 1/|v|.
__global__ void __launch_bounds__(kNaThreads) na_norm(int32_t n, NaPtrs p, const double* __restrict__ v) {
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)kNaThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kNaThreads)
    acc = fma(v[j], v[j], acc);
  na_block_total(acc, p, p.ctl() + 1, [](double t) { return t > 0.0 ? 1.0 / sqrt(t) : 0.0; });
}

lp_status na_fail(lp_status code, std::string* err, const std::string& msg) {
  *err = msg;
  return code;
}

}  // namespace
}  // namespace pdhg

// Defined in solver.cu: sets the calling thread's lp_last_error message.
void pdhg_set_last_error(const std::string& msg);

extern "C" lp_status lp_power_norm_noalloc(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                                           const int32_t* col_idx, const double* val, double tol,
                                           int64_t max_iter, uint64_t seed, void* stream,
                                           double* norm_out, int64_t* iters_out) {
  using namespace pdhg;
  std::string err;
  auto done = [&](lp_status code) {
    pdhg_set_last_error(code == LP_OK ? std::string() : err);
    return code;
  };
  if (!norm_out || m < 0 || n < 0 || nnz < 0 || !(tol >= 0.0) || max_iter < 1)
    return done(na_fail(LP_ERR_INVALID_ARG, &err, "lp_power_norm_noalloc: bad argument"));
  if (m > kNaMaxDim || n > kNaMaxDim)
    return done(na_fail(LP_ERR_TOO_LARGE, &err, "lp_power_norm_noalloc: m and n must be at most " +
                                                    std::to_string(kNaMaxDim) + " (size of its static scratch)"));
  if (nnz > 0 && (!row_ptr || !col_idx || !val))
    return done(na_fail(LP_ERR_INVALID_ARG, &err, "lp_power_norm_noalloc: NULL matrix array"));
  if (iters_out) *iters_out = 0;
  if (m == 0 || n == 0 || nnz == 0) {
    *norm_out = 0.0;
    return done(LP_OK);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return done(na_fail(LP_ERR_CUDA, &err, std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
  // The device address of the static scratch in the current device's context, looked up on
  // every call (a host-side lookup once the module is loaded): a cached address would dangle
  // after the context is torn down and re-created (cudaDeviceReset).  The first call on a
  // device may load the module, which is why it must not happen inside a stream capture.
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_na_scratch);
  if (e != cudaSuccess)
    return done(na_fail(LP_ERR_CUDA, &err, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)));
  NaPtrs p{static_cast<double*>(ptr)};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto blocks_for = [&](int64_t work) {
    int64_t b = (work + kNaThreads - 1) / kNaThreads;
    if (b < 1) b = 1;
    if (b > 4 * sms) b = 4 * sms;
    if (b > kNaMaxBlocks) b = kNaMaxBlocks;
    return (int)b;
  };
  const int gv = blocks_for(n);
  const int gr = blocks_for(int64_t(m) * 32 > n ? int64_t(m) * 32 : n);
  // the arrival counter must start at zero; an earlier call always leaves it rewound, but a
  // fresh process starts from the zero-initialised static array as well
  e = cudaMemsetAsync(p.counter(), 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return done(na_fail(LP_ERR_CUDA, &err, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)));
  na_start<<<gv, kNaThreads, 0, s>>>(n, seed, p);
  double* u = p.u();
  double* v = p.v();
  // Steps run kNaBatch at a time; each records its estimate in hist[q], and the host applies
  // the stopping rule to the batch in step order after one synchronisation (steps past the
  // stopping one change only the scratch).
  double got[kNaBatch + 1];
  double lam = 0.0, prev = 0.0;
  int64_t it = 0;
  bool stop = false;
  while (!stop && it < max_iter) {
    const int64_t left = max_iter - it;
    const int batch = left < kNaBatch ? (int)left : kNaBatch;
    for (int q = 0; q < batch; ++q) {
      na_rows<<<gr, kNaThreads, 0, s>>>(m, n, nnz, row_ptr, col_idx, val, p, u, v, q);
      na_scatter<<<gr, kNaThreads, 0, s>>>(m, n, nnz, row_ptr, col_idx, val, p, v);
      na_norm<<<gv, kNaThreads, 0, s>>>(n, p, v);
      double* t = u;
      u = v;
      v = t;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(got, p.hist(), sizeof(double) * batch, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(got + kNaBatch, p.ctl() + 3, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(na_fail(LP_ERR_CUDA, &err, std::string("power iteration: ") + cudaGetErrorString(e)));
    unsigned bad = 0;
    std::memcpy(&bad, got + kNaBatch, sizeof(unsigned));
    if (bad)
      return done(na_fail(LP_ERR_INVALID_INPUT, &err,
                          "lp_power_norm_noalloc: CSR entry out of range (row_ptr outside [0, nnz] or "
                          "decreasing, or a column index outside [0, n))"));
    for (int q = 0; q < batch && !stop; ++q) {
      ++it;
      lam = got[q];
      if (lam == 0.0) stop = true;
      else if (it > 1 && std::fabs(lam - prev) <= tol * lam) stop = true;
      else prev = lam;
    }
  }
  *norm_out = std::sqrt(lam);
  if (iters_out) *iters_out = it;
  return done(LP_OK);
}
