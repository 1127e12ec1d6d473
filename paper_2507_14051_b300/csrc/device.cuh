// Device-side data structures and helpers shared by the solver's kernels (sm_103a).
//
// Storage: A and its transpose are kept as CSR with 32-bit offsets, rows (resp. columns)
// permuted so that rows of similar length are contiguous ("bins").  Each bin is processed in
// tiles of R consecutive rows by one warp, G lanes per row (G a power of two <= 32), so the
// values/indices a pass reads are contiguous and the per-row epilogue that follows the dot
// products runs with lane L owning row L of the tile (coalesced vector traffic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdhg {

constexpr int kWarps = 8;  // warps per block of the streaming kernels
constexpr int kThreads = kWarps * 32;
constexpr int kMaxBins = 34;
constexpr int kNumSums = 5;  // reduction slots per kernel
constexpr int kCtaRowMin = 256;  // rows with more entries are processed by a whole CTA
constexpr int kTileNnz = 1024;   // target nonzeros per warp task
constexpr int kIlp = 4;          // independent entries a lane loads before accumulating
constexpr unsigned kFull = 0xffffffffu;

struct Bin {
  int32_t row0, row1;     // rows [row0, row1) of the permuted matrix
  int32_t lanes;          // G: lanes per row (1, 2, 4, 8, 16 or 32)
  int32_t rows_per_tile;  // R: rows per warp task (<= 32)
  int32_t task0;          // index of the bin's first task
};

// Rows [0, cta_rows) are long (more than kCtaRowMin entries) and are handled one row per CTA;
// the bins cover the rest, one tile of rows per warp.
struct BinTable {
  int32_t nbins;
  int32_t ntasks;
  int32_t cta_rows;
  Bin bin[kMaxBins];
};

enum : int32_t { kOptimal = 1, kIterLimit = 2, kNumerical = 3, kInternalError = 6 };

// Scalar state of one solve; lives in device memory and is only touched by the last block of
// each iteration kernel (and read by all threads at kernel entry).
struct Ctl {
  double eta, omega, tau, sigma, inv_sigma;
  double ha, hb, he;  // z <- ha*zhat + hb*z + he*z0 (reflected Halpern weights)
  int32_t restart;    // decision taken at iteration t (applied by K2(t) and K1(t+1))
  int32_t done;
  int32_t status;
  int32_t restart_enabled;
  int64_t t, k, iters, restarts, max_iter, check_every, trace_cap, bodies;
  double tol;
  double r0, r_prev;
  double pid_integral, pid_eprev;
  int32_t pid_has_prev;
  int32_t pid_enabled;
  double sxx, sx0;       // |x - xhat|^2 and |xhat - x0|^2 for the coming iteration (from K2)
  double pres2, dobj_y;  // check-iteration sums from K1, finished by K2
  double omega_used;     // omega of the last iteration performed
  int64_t restarts_used; // restarts before the last iteration's decision
  double kkt[8];         // rel_gap, rel_pres, rel_dres, rel_kkt, pobj, dobj, pres, dres
  double lu_norm, c_norm;
  double gamma, beta_s, beta_n, beta_a, kp, ki, kd;
  unsigned int count0, count1, count2, count3;
};

__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return fmin(fmax(v, lo), hi);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

__device__ __forceinline__ int find_bin(const BinTable& bt, int task) {
  int b = 0;
  while (b + 1 < bt.nbins && task >= bt.bin[b + 1].task0) ++b;
  return b;
}

// L2 cache policies: the matrix is streamed once per iteration (evict first); the gathered
// vector is re-read by many rows (evict last).
struct LoadPolicy {
  uint64_t stream, keep;
};
__device__ __forceinline__ LoadPolicy make_policy() {
  LoadPolicy p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.stream));
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.keep));
  return p;
}
// Read-only streaming loads of the matrix: no L1 allocation, L2 evict-first.
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// Gathered vector entries: L2 evict-last.
__device__ __forceinline__ double ld_gather(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// Partial dot product of one lane: entries b+first, b+first+stride, ... < e, loaded kIlp at a
// time (all loads of a batch issued before any is used) and accumulated in entry order.
__device__ __forceinline__ double strided_dot(const int32_t* __restrict__ ci,
                                              const double* __restrict__ val,
                                              const double* __restrict__ xg, int first, int e,
                                              int stride, const LoadPolicy& pol) {
  double acc = 0.0;
  for (int k0 = first; k0 < e; k0 += kIlp * stride) {
    double v[kIlp];
    int c[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const int k = k0 + u * stride;
      if (k < e) {
        v[u] = ld_stream(val + k, pol.stream);
        c[u] = ld_stream(ci + k, pol.stream);
      } else {
        v[u] = 0.0;
        c[u] = -1;
      }
    }
    double xv[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) xv[u] = c[u] >= 0 ? ld_gather(xg + c[u], pol.keep) : 0.0;
#pragma unroll
    for (int u = 0; u < kIlp; ++u)
      if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
  }
  return acc;
}

// Dot products of the rows [row0, row0 + nrows) (nrows <= 32) of a CSR matrix with xg.
// G lanes per row, 32/G rows per pass; lane L returns the value of row L (garbage for
// L >= nrows).  Summation: each lane accumulates its strided entries in order, then a
// fixed xor butterfly over the G lanes (deterministic).
__device__ __forceinline__ double tile_spmv(const int32_t* __restrict__ rp,
                                            const int32_t* __restrict__ ci,
                                            const double* __restrict__ val,
                                            const double* __restrict__ xg, int row0, int nrows,
                                            int G, int lane, const LoadPolicy& pol) {
  const int rpp = 32 / G;  // rows per pass
  const int passes = (nrows + rpp - 1) / rpp;
  const int g = lane / G, sub = lane - g * G;
  // lane L's own row bounds, fetched once (coalesced), then passed around by shuffles
  int my_b = 0, my_e = 0;
  if (lane < nrows) {
    my_b = rp[row0 + lane];
    my_e = rp[row0 + lane + 1];
  }
  double mine = 0.0;
  for (int p = 0; p < passes; ++p) {
    const int q = p * rpp + g;  // row of this lane's group in this pass
    const int b = __shfl_sync(kFull, my_b, q & 31);
    const int e = __shfl_sync(kFull, my_e, q & 31);
    double acc = q < nrows ? strided_dot(ci, val, xg, b + sub, e, G, pol) : 0.0;
    for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    const double v = __shfl_sync(kFull, acc, (lane % rpp) * G);
    if (lane / rpp == p) mine = v;
  }
  return mine;
}

// Dot product of one long row with the whole block (all threads must call it): each thread
// takes every kThreads-th entry; the block's values are summed by a shared-memory halving tree
// down to one warp, then a warp butterfly (fixed order; about 12 warp-wide FP64 adds instead of
// one butterfly per warp).  The result is valid in thread 0.
__device__ __forceinline__ double cta_row_dot(const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ ci,
                                              const double* __restrict__ val,
                                              const double* __restrict__ xg, int row,
                                              const LoadPolicy& pol) {
  __shared__ double part[kThreads];
  const int tid = threadIdx.x;
  const int b = rp[row], e = rp[row + 1];
  part[tid] = strided_dot(ci, val, xg, b + tid, e, kThreads, pol);
  __syncthreads();
#pragma unroll
  for (int w = kThreads / 2; w >= 32; w >>= 1) {
    if (tid < w) part[tid] += part[tid + w];
    __syncthreads();
  }
  double v = 0.0;
  if (tid < 32) v = warp_sum(part[tid]);
  __syncthreads();
  return v;
}

// Visits every row of a binned CSR matrix once with its dot product against xg:
// epi(row, value) runs in thread 0 for the long rows (one per CTA, grid-strided) and in
// lane L < nrows of the owning warp for the binned rows.  Which block and lane handle a row
// depends only on the grid size, so all sums over rows are deterministic.
template <class Epi>
__device__ __forceinline__ void for_each_row(const BinTable& bins, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const double* __restrict__ val,
                                             const double* __restrict__ xg, const LoadPolicy& pol,
                                             Epi&& epi) {
  for (int r = blockIdx.x; r < bins.cta_rows; r += gridDim.x) {
    const double v = cta_row_dot(rp, ci, val, xg, r, pol);
    if (threadIdx.x == 0) epi(r, v);
  }
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kWarps;
  for (int task = blockIdx.x * kWarps + (threadIdx.x >> 5); task < bins.ntasks; task += nwarps) {
    const Bin B = bins.bin[find_bin(bins, task)];
    const int row0 = B.row0 + (task - B.task0) * B.rows_per_tile;
    const int nrows = min(B.rows_per_tile, B.row1 - row0);
    const double v = tile_spmv(rp, ci, val, xg, row0, nrows, B.lanes, lane, pol);
    if (lane < nrows) epi(row0 + lane, v);
  }
}

// Sums kNumSums per-thread values over the block (shared-memory halving tree down to one
// warp, then a warp butterfly, all in a fixed order), writes them to partials[blockIdx.x][*],
// and returns true in every thread of the block that finished last (all partials are then
// visible).  The whole block must call it; `counter` is reset by the caller's last block.
__device__ __forceinline__ bool block_sums_last(double (&s)[kNumSums], double* partials,
                                                unsigned int* counter) {
  __shared__ double red[kNumSums][kThreads];
  __shared__ bool is_last;
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) red[q][tid] = s[q];
  __syncthreads();
#pragma unroll
  for (int w = kThreads / 2; w >= 32; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) red[q][tid] += red[q][tid + w];
    }
    __syncthreads();
  }
  if (tid < 32) {
    double v[kNumSums];
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) v[q] = warp_sum(red[q][tid]);
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) partials[blockIdx.x * kNumSums + q] = v[q];
      __threadfence();
      const unsigned prev = atomicAdd(counter, 1u);
      is_last = (prev == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// In the last block's first warp: totals of the partials of all blocks, in a fixed order.
__device__ __forceinline__ void total_partials(const double* partials, int nblocks,
                                               double (&tot)[kNumSums]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) tot[q] = 0.0;
#pragma unroll 4
  for (int b = lane; b < nblocks; b += 32) {
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) tot[q] += __ldcg(partials + b * kNumSums + q);
  }
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) tot[q] = warp_sum(tot[q]);
}

}  // namespace pdhg
