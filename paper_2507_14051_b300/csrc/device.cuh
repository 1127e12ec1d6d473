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
// rows with more entries are split into chunk tasks; shorter ones are tiles of up to 32 lanes
// (on the MIPLIB-shaped LP, 1024 took the iteration from 29.7 to 28.6 us against 256: fewer
// chunked rows, whose partial sums every block adds after the barrier; 2048 and 4096 made the
// longest single tasks too long)
constexpr int kLongRowMin = 1024;
constexpr int kChunkNnz = 256;    // entries per chunk task of a long row
constexpr int kIlp = 8;           // independent entries a lane loads before accumulating
constexpr unsigned kFull = 0xffffffffu;

struct Bin {
  int32_t row0, row1;     // rows [row0, row1) of the permuted matrix
  int32_t lanes;          // G: lanes per row (1, 2, 4, 8, 16 or 32)
  int32_t rows_per_tile;  // R: rows per warp task (<= 32)
  int32_t task0;          // index of the bin's first task
  int32_t per_lane;       // most entries a lane reads in one task (ceil(Lc / G))
  int32_t sliced;         // 1: the bin's tiles are also stored sliced (BinTable::sell_*)
};

// Rows [0, long_rows) of the permuted order have more than kLongRowMin entries; each is split
// into chunks of kChunkNnz entries, one warp task per chunk (tasks [0, nchunks)).  chunk[q] =
// (row, first chunk of that row, number of chunks of the row, 0); part[q] holds the chunk's
// partial dot product and arrivals[row] counts finished chunks (the last one combines the
// partials in chunk order and rewinds the counter).  The bins cover the remaining rows, one
// tile of up to 32 rows per warp task (tasks [nchunks, nchunks + ntasks)).
struct BinTable {
  int32_t nbins;
  int32_t ntasks;
  int32_t long_rows;
  int32_t nchunks;
  const int4* chunk;
  double* part;
  unsigned int* arrivals;
  double* contrib;  // long row r's kNumSums epilogue contributions (added by the last block)
  // Sliced copy of the one-lane-per-row bins' 32-row tiles: tile task t (counted from the first
  // tile task) holds P = (sell_off[t + 1] - sell_off[t]) / 32 slots, and entry u of its row L
  // sits at sell_off[t] + 32 u + L (padding: column index -1), so a warp reads a slot of all 32
  // rows as one 128-byte line (FP32 values and indices) instead of 32 scattered words.  The
  // values are those of the matrix in the value type of the kernel that reads them (sell_val
  // points at doubles for the FP64 kernels, at floats for the FP32 ones).  sell_off NULL: none.
  const int32_t* sell_off;
  const int32_t* sell_ci;
  const void* sell_val;
  Bin bin[kMaxBins];
};

enum : int32_t { kOptimal = 1, kIterLimit = 2, kNumerical = 3, kStalled = 5, kInternalError = 6 };

// Scalar state of one solve; lives in device memory and is only touched by the last block of
// each iteration kernel (and read by all threads at kernel entry).
struct Ctl {
  double eta, omega, tau, sigma, inv_sigma;
  double w_over_eta, inv_eta_w;  // omega/eta and 1/(eta*omega): the weights of the P-norm
  double ha, hb, he;  // z <- ha*zhat + hb*z + he*z0 (reflected Halpern weights)
  int32_t restart;    // decision taken at iteration t (applied by K2(t) and K1(t+1))
  int32_t done;
  int32_t status;
  int32_t restart_enabled;
  int64_t t, k, iters, restarts, max_iter, check_every, trace_cap, bodies;
  double tol;
  double r0, r_prev;  // squared fixed-point residuals r_0^2 and r_{t-1}^2 of the epoch
  double pid_integral, pid_eprev;
  int32_t pid_has_prev;
  int32_t pid_enabled;
  double sxx, sx0;       // |x - xhat|^2 and |xhat - x0|^2 for the coming iteration (from K2)
  double pres2, dobj_y;  // check-iteration sums from K1, finished by K2
  double omega_used;     // omega of the last iteration performed
  int64_t iters32;       // mixed precision: iterations of the FP32 phase
  // FP32 phase stall guard: best relative KKT error seen at a check iteration, checks since,
  // and omega / PID state at that check (restored for the FP64 phase after a stall); the
  // check iterations store zhat in slot cand_slot of a two-slot buffer, best_slot holds the best
  int32_t patience, since_best, cand_slot, best_slot;
  double best_kkt, omega_best, integral_best, eprev_best;
  double kkt_best[8];
  int64_t restarts_used; // restarts before the last iteration's decision
  double kkt[8];         // rel_gap, rel_pres, rel_dres, rel_kkt, pobj, dobj, pres, dres
  double lu_norm, c_norm;
  double gamma, beta_s, beta_n, beta_a, kp, ki, kd;
  unsigned int count0, count1, count2, count3;
};

// An FP64 value's bits as a signed integer with the value's order (IEEE 754 sign-magnitude:
// negative values have their magnitude bits flipped), so that -inf < ... < -0 < +0 < ... < +inf.
__device__ __forceinline__ long long ord_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// min(max(v, lo), hi) by integer compares of ord_key: the same value as fmin(fmax(v, lo), hi)
// for every non-NaN v (infinite bounds included; -0 orders below +0).  On this GPU an FP64 min or max
// takes an FP64 pipe slot like an fma, and the loop kernels are bound by that pipe; integer
// compares and selects run on the integer pipes.  A NaN v goes to hi or lo by its sign bit.
__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  const long long kv = ord_key(v), kl = ord_key(lo), kh = ord_key(hi);
  const bool below = kv < kl;
  const long long kr = below ? kl : kv;
  const double r = below ? lo : v;
  return kr > kh ? hi : r;
}
__device__ __forceinline__ float clampd(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
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
// Read-only loads of the matrix: L2 evict-first (the matrix is streamed once per iteration), but
// allocated in L1: a lane reads its row's consecutive entries in successive steps, so one L1
// line serves several steps of several lanes instead of one L2 fetch per step (measured: FP32
// multicommodity iteration 156 -> 146 us, FP64 297 -> 288 us).
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
// Read-only loads of a sliced tile's slot (a whole line per warp, read once): evict-first in L2
// and not allocated in L1, where they would only displace the gathered vector's lines.
__device__ __forceinline__ double ld_slice(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_slice(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_slice(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
// Prefetch of the line holding *p into L1 (no register is written; the later load hits L1).
template <class T>
__device__ __forceinline__ void prefetch_l1(const T* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
// Gathered vector entries: L2 evict-last.  A coherent load (not .nc): the persistent kernels
// gather vectors that their previous phase wrote, after a grid or block barrier.
__device__ __forceinline__ double ld_gather(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_gather(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

// splitmix64 (Steele, Lea, Flood 2014; public-domain reference code by S. Vigna): output i
// of the stream started at `seed`; the start vector entry is uniform on [-1, 1) from the top
// 53 bits.  Entry j' of the permuted vector is the entry of original column col_perm[j'].
__device__ __forceinline__ double start_entry(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Read-only loads with the default L2 policy: for data the same SMs re-read every iteration (the
// cluster loops over a small instance), which should stay in L1 and L2.
__device__ __forceinline__ double ld_cached(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_cached(const float* p) { return __ldg(p); }
__device__ __forceinline__ int32_t ld_cached(const int32_t* p) { return __ldg(p); }

// Partial dot product of one lane: entries b+first, b+first+stride, ... < e, loaded ILP at a
// time (all loads of a batch issued before any is used) and accumulated in entry order.
// kCached: matrix loads without the L2 evict-first hint (ld_cached), for a matrix slice that the
// same SMs re-read every iteration.
template <int ILP, class V, bool kCached = false>
__device__ __forceinline__ V strided_dot_n(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                           const V* __restrict__ xg, int first, int e, int stride,
                                           const LoadPolicy& pol) {
  V acc = V(0);
  for (int k0 = first; k0 < e; k0 += ILP * stride) {
    V v[ILP];
    int c[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const int k = k0 + u * stride;
      if (k < e) {
        if (kCached) {
          v[u] = ld_cached(val + k);
          c[u] = ld_cached(ci + k);
        } else {
          v[u] = ld_stream(val + k, pol.stream);
          c[u] = ld_stream(ci + k, pol.stream);
        }
      } else {
        v[u] = V(0);
        c[u] = -1;
      }
    }
    V xv[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) xv[u] = c[u] >= 0 ? ld_gather(xg + c[u], pol.keep) : V(0);
#pragma unroll
    for (int u = 0; u < ILP; ++u)
      if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
  }
  return acc;
}

// The same with the batch sized to `per_lane`, the most entries any lane of the warp has
// (uniform across the warp): short rows then issue no FP64 fma for absent entries, which on
// this GPU's FP64 unit would cost as much as real ones.
template <class V, bool kCached = false>
__device__ __forceinline__ V strided_dot(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                         const V* __restrict__ xg, int first, int e, int stride,
                                         int per_lane, const LoadPolicy& pol) {
  if (per_lane <= 1) return strided_dot_n<1, V, kCached>(ci, val, xg, first, e, stride, pol);
  if (per_lane <= 2) return strided_dot_n<2, V, kCached>(ci, val, xg, first, e, stride, pol);
  if (per_lane <= 4) return strided_dot_n<4, V, kCached>(ci, val, xg, first, e, stride, pol);
  return strided_dot_n<kIlp, V, kCached>(ci, val, xg, first, e, stride, pol);
}

// One batch of N entries of a lane's strided slice (k0, k0 + stride, ...; entries at or past e
// are absent), all loads issued before any is used, accumulated into acc in entry order.
template <int N, class V, bool kCached>
__device__ __forceinline__ void dot_batch(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                          const V* __restrict__ xg, int k0, int e, int stride,
                                          const LoadPolicy& pol, V& acc) {
  V v[N];
  int c[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    const int k = k0 + u * stride;
    if (k < e) {
      if (kCached) {
        v[u] = ld_cached(val + k);
        c[u] = ld_cached(ci + k);
      } else {
        v[u] = ld_stream(val + k, pol.stream);
        c[u] = ld_stream(ci + k, pol.stream);
      }
    } else {
      v[u] = V(0);
      c[u] = -1;
    }
  }
  V xv[N];
#pragma unroll
  for (int u = 0; u < N; ++u) xv[u] = c[u] >= 0 ? ld_gather(xg + c[u], pol.keep) : V(0);
#pragma unroll
  for (int u = 0; u < N; ++u)
    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
}

// Partial dot product of one lane over exactly `slots` strided entries (warp-uniform: the most
// entries any lane of the warp has in this pass), in batches of 8 and one exact remainder
// batch: the warp issues one fma instruction per slot and none for slots no lane has (on this
// GPU an FP64 warp instruction costs the same pipe time whatever its active lanes).  The lane's
// entries are accumulated in entry order, as strided_dot does.
template <class V, bool kCached = false>
__device__ __forceinline__ V strided_dot_slots(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                               const V* __restrict__ xg, int first, int e, int stride,
                                               int slots, const LoadPolicy& pol) {
  V acc = V(0);
  int k0 = first;
  for (; slots >= kIlp; slots -= kIlp, k0 += kIlp * stride)
    dot_batch<kIlp, V, kCached>(ci, val, xg, k0, e, stride, pol, acc);
  switch (slots) {
    case 1: dot_batch<1, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 2: dot_batch<2, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 3: dot_batch<3, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 4: dot_batch<4, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 5: dot_batch<5, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 6: dot_batch<6, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    case 7: dot_batch<7, V, kCached>(ci, val, xg, k0, e, stride, pol, acc); break;
    default: break;
  }
  return acc;
}

// Two partial dot products of one lane, over [fa, ea) and [fb, eb) with the same stride, their
// loads issued together (twice the loads in flight of strided_dot_n); each is accumulated in
// entry order exactly as strided_dot_n would.
template <int ILP, class V>
__device__ __forceinline__ void strided_dot_pair(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                                 const V* __restrict__ xg, int fa, int ea, int fb, int eb,
                                                 int stride, const LoadPolicy& pol, V& ra, V& rb) {
  V acc_a = V(0), acc_b = V(0);
  for (int k0 = 0; fa + k0 < ea || fb + k0 < eb; k0 += ILP * stride) {
    V va[ILP], vb[ILP];
    int ca[ILP], cb[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const int ka = fa + k0 + u * stride, kb = fb + k0 + u * stride;
      if (ka < ea) {
        va[u] = ld_stream(val + ka, pol.stream);
        ca[u] = ld_stream(ci + ka, pol.stream);
      } else {
        va[u] = V(0);
        ca[u] = -1;
      }
      if (kb < eb) {
        vb[u] = ld_stream(val + kb, pol.stream);
        cb[u] = ld_stream(ci + kb, pol.stream);
      } else {
        vb[u] = V(0);
        cb[u] = -1;
      }
    }
    V xa[ILP], xb[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      xa[u] = ca[u] >= 0 ? ld_gather(xg + ca[u], pol.keep) : V(0);
      xb[u] = cb[u] >= 0 ? ld_gather(xg + cb[u], pol.keep) : V(0);
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u)
      if (ca[u] >= 0) acc_a = fma(va[u], xa[u], acc_a);
#pragma unroll
    for (int u = 0; u < ILP; ++u)
      if (cb[u] >= 0) acc_b = fma(vb[u], xb[u], acc_b);
  }
  ra = acc_a;
  rb = acc_b;
}

// One tile task of a BinTable: its rows, shape, and lane L's row bounds (L < nrows; 0 else).
// Largest entries per lane for which two tiles run side by side (tile_spmv_pair).
constexpr int kPairMaxPerLane = 4;

struct TileTask {
  int row0, nrows, lanes, per_lane, b, e;
  int sliced;  // the tile is read from the sliced copy: b = its first slot, e = its slot count
};

__device__ __forceinline__ TileTask tile_task(const BinTable& bins, const int32_t* __restrict__ rp, int task,
                                              int lane) {
  const Bin B = bins.bin[find_bin(bins, task - bins.nchunks)];
  TileTask t;
  t.row0 = B.row0 + (task - bins.nchunks - B.task0) * B.rows_per_tile;
  t.nrows = min(B.rows_per_tile, B.row1 - t.row0);
  t.lanes = B.lanes;
  t.per_lane = B.per_lane;
  t.sliced = B.sliced && bins.sell_off != nullptr;
  t.b = 0;
  t.e = 0;
  if (t.sliced) {
    const int q = task - bins.nchunks;
    t.b = bins.sell_off[q];
    t.e = (bins.sell_off[q + 1] - t.b) >> 5;
  } else if (lane < t.nrows) {
    t.b = rp[t.row0 + lane];
    t.e = rp[t.row0 + lane + 1];
  }
  return t;
}

// Dot products of a sliced tile (TileTask::sliced): lane L returns row L's value.  The lane
// accumulates its row's entries in entry order, as the CSR tile does, so both give the same
// bits; every load of a slot is one line for the whole warp.
template <int N, class V, bool kCached>
__device__ __forceinline__ void sliced_batch(const int32_t* __restrict__ sc, const V* __restrict__ sv,
                                             const V* __restrict__ xg, const LoadPolicy& pol, V& acc) {
  V v[N];
  int c[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
    if (kCached) {
      v[u] = ld_cached(sv + 32 * u);
      c[u] = ld_cached(sc + 32 * u);
    } else {
      v[u] = ld_slice(sv + 32 * u, pol.stream);
      c[u] = ld_slice(sc + 32 * u, pol.stream);
    }
  }
  V xv[N];
#pragma unroll
  for (int u = 0; u < N; ++u) xv[u] = c[u] >= 0 ? ld_gather(xg + c[u], pol.keep) : V(0);
#pragma unroll
  for (int u = 0; u < N; ++u)
    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
}

// kCached: the slots are read with the default cache policy (kept in L1 and L2), for a small LP
// whose tiles the same SMs re-read every iteration.
template <class V, bool kCached = false>
__device__ __forceinline__ V sliced_spmv(const BinTable& bins, const V* __restrict__ xg, const TileTask& a,
                                         int lane, const LoadPolicy& pol) {
  const V* __restrict__ sv = static_cast<const V*>(bins.sell_val) + a.b + lane;
  const int32_t* __restrict__ sc = bins.sell_ci + a.b + lane;
  V acc = V(0);
  int slots = a.e;
  for (; slots >= kIlp; slots -= kIlp, sv += 32 * kIlp, sc += 32 * kIlp)
    sliced_batch<kIlp, V, kCached>(sc, sv, xg, pol, acc);
  switch (slots) {
    case 1: sliced_batch<1, V, kCached>(sc, sv, xg, pol, acc); break;
    case 2: sliced_batch<2, V, kCached>(sc, sv, xg, pol, acc); break;
    case 3: sliced_batch<3, V, kCached>(sc, sv, xg, pol, acc); break;
    case 4: sliced_batch<4, V, kCached>(sc, sv, xg, pol, acc); break;
    case 5: sliced_batch<5, V, kCached>(sc, sv, xg, pol, acc); break;
    case 6: sliced_batch<6, V, kCached>(sc, sv, xg, pol, acc); break;
    case 7: sliced_batch<7, V, kCached>(sc, sv, xg, pol, acc); break;
    default: break;
  }
  return acc;
}

// Two sliced tiles side by side (their loads issued together): lane L returns row L's value of
// each; each accumulated exactly as sliced_spmv would.
template <class V>
__device__ __forceinline__ void sliced_spmv_pair(const BinTable& bins, const V* __restrict__ xg, const TileTask& a,
                                                 const TileTask& b, int lane, const LoadPolicy& pol, V& va, V& vb) {
  const V* __restrict__ vals = static_cast<const V*>(bins.sell_val);
  V acc_a = V(0), acc_b = V(0);
  const int slots = max(a.e, b.e);
  for (int u0 = 0; u0 < slots; u0 += kPairMaxPerLane) {
    V xa[kPairMaxPerLane], xb[kPairMaxPerLane], wa[kPairMaxPerLane], wb[kPairMaxPerLane];
    int ca[kPairMaxPerLane], cb[kPairMaxPerLane];
#pragma unroll
    for (int u = 0; u < kPairMaxPerLane; ++u) {
      const int ka = a.b + 32 * (u0 + u) + lane, kb = b.b + 32 * (u0 + u) + lane;
      ca[u] = -1;
      cb[u] = -1;
      wa[u] = V(0);
      wb[u] = V(0);
      if (u0 + u < a.e) {
        wa[u] = ld_slice(vals + ka, pol.stream);
        ca[u] = ld_slice(bins.sell_ci + ka, pol.stream);
      }
      if (u0 + u < b.e) {
        wb[u] = ld_slice(vals + kb, pol.stream);
        cb[u] = ld_slice(bins.sell_ci + kb, pol.stream);
      }
    }
#pragma unroll
    for (int u = 0; u < kPairMaxPerLane; ++u) {
      xa[u] = ca[u] >= 0 ? ld_gather(xg + ca[u], pol.keep) : V(0);
      xb[u] = cb[u] >= 0 ? ld_gather(xg + cb[u], pol.keep) : V(0);
    }
#pragma unroll
    for (int u = 0; u < kPairMaxPerLane; ++u)
      if (ca[u] >= 0) acc_a = fma(wa[u], xa[u], acc_a);
#pragma unroll
    for (int u = 0; u < kPairMaxPerLane; ++u)
      if (cb[u] >= 0) acc_b = fma(wb[u], xb[u], acc_b);
  }
  va = acc_a;
  vb = acc_b;
}

// Two single-pass tiles with the same lanes per row G (nrows * G <= 32 each, per_lane <=
// kPairMaxPerLane), their SpMVs interleaved: lane L returns row L's value of each (garbage for
// L >= nrows).  Each value is summed exactly as tile_spmv sums it.
template <class V>
__device__ __forceinline__ void tile_spmv_pair(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                               const V* __restrict__ xg, const TileTask& a, const TileTask& b,
                                               int lane, const LoadPolicy& pol, V& va, V& vb) {
  const int G = a.lanes, g = lane / G, sub = lane - g * G;
  const int ba = __shfl_sync(kFull, a.b, g), ea = __shfl_sync(kFull, a.e, g);
  const int bb = __shfl_sync(kFull, b.b, g), eb = __shfl_sync(kFull, b.e, g);
  V acc_a, acc_b;
  if (max(a.per_lane, b.per_lane) <= 2)
    strided_dot_pair<2, V>(ci, val, xg, ba + sub, ea, bb + sub, eb, G, pol, acc_a, acc_b);
  else
    strided_dot_pair<kPairMaxPerLane, V>(ci, val, xg, ba + sub, ea, bb + sub, eb, G, pol, acc_a, acc_b);
  for (int off = G >> 1; off > 0; off >>= 1) {
    acc_a += __shfl_xor_sync(kFull, acc_a, off);
    acc_b += __shfl_xor_sync(kFull, acc_b, off);
  }
  va = __shfl_sync(kFull, acc_a, (lane % (32 / G)) * G);
  vb = __shfl_sync(kFull, acc_b, (lane % (32 / G)) * G);
}

// Dot products of the rows [row0, row0 + nrows) (nrows <= 32) of a CSR matrix with xg.
// G lanes per row, 32/G rows per pass; lane L returns the value of row L (garbage for
// L >= nrows).  Each pass runs as many entry slots as its longest row needs (a warp maximum of
// the rows' own lengths; `per_lane`, the length class's bound, is not needed).  Summation: each
// lane accumulates its strided entries in order, then a fixed xor butterfly over the G lanes
// (deterministic).
template <class V, bool kCached = false>
__device__ __forceinline__ V tile_spmv_b(const int32_t* __restrict__ ci, const V* __restrict__ val,
                                         const V* __restrict__ xg, int my_b, int my_e, int nrows, int G,
                                         int per_lane, int lane, const LoadPolicy& pol) {
  (void)per_lane;
  const int rpp = 32 / G;  // rows per pass
  const int passes = (nrows + rpp - 1) / rpp;
  const int g = lane / G, sub = lane - g * G;
  V mine = V(0);
  for (int p = 0; p < passes; ++p) {
    const int q = p * rpp + g;  // row of this lane's group in this pass
    const int b = __shfl_sync(kFull, my_b, q & 31);
    const int e = __shfl_sync(kFull, my_e, q & 31);
    const int mine_slots = q < nrows && e > b + sub ? (e - b - sub + G - 1) / G : 0;
    const int slots = (int)__reduce_max_sync(kFull, (unsigned)mine_slots);
    V acc = q < nrows ? strided_dot_slots<V, kCached>(ci, val, xg, b + sub, e, G, slots, pol) : V(0);
    for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    const V v = __shfl_sync(kFull, acc, (lane % rpp) * G);
    if (lane / rpp == p) mine = v;
  }
  return mine;
}

// tile_spmv_b with lane L's row bounds (row L of the tile, L < nrows) fetched here, coalesced.
template <class V, bool kCached = false>
__device__ __forceinline__ V tile_spmv(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const V* __restrict__ val, const V* __restrict__ xg, int row0,
                                       int nrows, int G, int per_lane, int lane, const LoadPolicy& pol) {
  int my_b = 0, my_e = 0;
  if (lane < nrows) {
    my_b = rp[row0 + lane];
    my_e = rp[row0 + lane + 1];
  }
  return tile_spmv_b<V, kCached>(ci, val, xg, my_b, my_e, nrows, G, per_lane, lane, pol);
}

// Visits every row of a binned CSR matrix once with its dot product against xg and calls
// epi(row, value, in, acc) in exactly one lane: lane L < nrows of the warp that owns a tile (acc =
// that thread's running sums `s`; in = pre(row), issued before the tile's SpMV so that the
// row's own operands load while the SpMV runs), or lane 0 of the warp that finishes a long
// row's last chunk (acc = a zeroed array then stored in bins.contrib for the last block to add
// in row order; in = pre(row) loaded there).  Every sum therefore has a fixed order that
// depends only on the grid size: results are bit-reproducible run to run.
// kCached: matrix loads of single tiles with the default cache policy (ld_cached), for a small LP
// whose tiles the same SMs re-read every iteration (the cluster loop).
template <class V, class Pre, class Epi, bool kCached = false>
__device__ __forceinline__ void for_each_row_pf(const BinTable& bins, const int32_t* __restrict__ rp,
                                                const int32_t* __restrict__ ci, const V* __restrict__ val,
                                                const V* __restrict__ xg, const LoadPolicy& pol,
                                                double (&s)[kNumSums], Pre&& pre, Epi&& epi) {
  using In = decltype(pre(0));
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kWarps;
  const int total = bins.nchunks + bins.ntasks;
  // warp w of block b starts at task w * gridDim.x + b: a grid's first tasks go to different
  // blocks (a small LP's few tiles then run on as many SMs)
  for (int task = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; task < total; task += nwarps) {
    if (task < bins.nchunks) {
      const int4 ch = bins.chunk[task];
      const int b = rp[ch.x] + (task - ch.y) * kChunkNnz;
      const int e = min(rp[ch.x + 1], b + kChunkNnz);
      const V v = warp_sum(strided_dot(ci, val, xg, b + lane, e, 32, kChunkNnz / 32, pol));
      if (lane == 0) {
        bins.part[task] = (double)v;
        __threadfence();
        if (atomicAdd(bins.arrivals + ch.x, 1u) == (unsigned)ch.z - 1u) {
          __threadfence();
          double tot = 0.0;
          for (int q = 0; q < ch.z; ++q) tot += __ldcg(bins.part + ch.y + q);
          bins.arrivals[ch.x] = 0u;
          double c[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
          In in = pre(ch.x);
          epi(ch.x, (V)tot, in, c);
#pragma unroll
          for (int q = 0; q < kNumSums; ++q) bins.contrib[ch.x * kNumSums + q] = c[q];
        }
      }
      continue;
    }
    if constexpr (sizeof(V) != sizeof(float)) {
      // FP64 (bound by the FP64 pipe, not by loads in flight): one tile at a time
      const TileTask a = tile_task(bins, rp, task, lane);
      In in{};
      if (lane < a.nrows) in = pre(a.row0 + lane);
      const V v = a.sliced ? sliced_spmv<V, kCached>(bins, xg, a, lane, pol)
                           : tile_spmv_b<V, kCached>(ci, val, xg, a.b, a.e, a.nrows, a.lanes, a.per_lane, lane, pol);
      if (lane < a.nrows) epi(a.row0 + lane, v, in, s);
      continue;
    }
    // FP32 (bound by loads in flight): tiles two at a time (tasks t and t + nwarps, the same
    // tasks in the same order as one at a time); two short single-pass tiles of one shape run
    // their SpMVs side by side.
    const int task2 = task + nwarps;
    const TileTask a = tile_task(bins, rp, task, lane);
    const bool two = task2 < total;
    TileTask b{};
    if (two) b = tile_task(bins, rp, task2, lane);
    const bool pair = two && !a.sliced && !b.sliced && a.lanes == b.lanes && a.nrows * a.lanes <= 32 &&
                      b.nrows * b.lanes <= 32 && a.per_lane <= kPairMaxPerLane && b.per_lane <= kPairMaxPerLane;
    if (two && a.sliced && b.sliced) {
      In ia{}, ib{};
      if (lane < a.nrows) ia = pre(a.row0 + lane);
      if (lane < b.nrows) ib = pre(b.row0 + lane);
      V va, vb;
      sliced_spmv_pair(bins, xg, a, b, lane, pol, va, vb);
      if (lane < a.nrows) epi(a.row0 + lane, va, ia, s);
      if (lane < b.nrows) epi(b.row0 + lane, vb, ib, s);
    } else if (pair) {
      In ia{}, ib{};
      if (lane < a.nrows) ia = pre(a.row0 + lane);
      if (lane < b.nrows) ib = pre(b.row0 + lane);
      V va, vb;
      tile_spmv_pair(ci, val, xg, a, b, lane, pol, va, vb);
      if (lane < a.nrows) epi(a.row0 + lane, va, ia, s);
      if (lane < b.nrows) epi(b.row0 + lane, vb, ib, s);
    } else {
      {
        In in{};
        if (lane < a.nrows) in = pre(a.row0 + lane);
        const V v = a.sliced ? sliced_spmv<V, kCached>(bins, xg, a, lane, pol)
                             : tile_spmv_b<V, kCached>(ci, val, xg, a.b, a.e, a.nrows, a.lanes, a.per_lane, lane, pol);
        if (lane < a.nrows) epi(a.row0 + lane, v, in, s);
      }
      if (two) {
        In in{};
        if (lane < b.nrows) in = pre(b.row0 + lane);
        const V v = b.sliced ? sliced_spmv<V, kCached>(bins, xg, b, lane, pol)
                             : tile_spmv_b<V, kCached>(ci, val, xg, b.b, b.e, b.nrows, b.lanes, b.per_lane, lane, pol);
        if (lane < b.nrows) epi(b.row0 + lane, v, in, s);
      }
    }
    task = task2;  // the loop's increment moves on to task2 + nwarps
  }
}

struct NoOperands {};

// for_each_row_pf without per-row operands: epi(row, value, acc).
template <class V, class Epi, bool kCached = false>
__device__ __forceinline__ void for_each_row(const BinTable& bins, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci, const V* __restrict__ val,
                                             const V* __restrict__ xg, const LoadPolicy& pol,
                                             double (&s)[kNumSums], Epi&& epi) {
  auto pre = [](int) { return NoOperands{}; };
  auto e2 = [&](int i, V v, const NoOperands&, double (&acc)[kNumSums]) { epi(i, v, acc); };
  for_each_row_pf<V, decltype(pre)&, decltype(e2)&, kCached>(bins, rp, ci, val, xg, pol, s, pre, e2);
}

// Sums the first nsums (<= kNumSums <= kWarps) of each thread's v[] over the block in a fixed
// order: warp q adds sum q -- lane L the values of threads L, L + 32, ... as a pairwise tree,
// then a butterfly over the lanes -- so the sums' FP64 additions run on different warps at once
// (an FP64 warp instruction occupies the pipe as long as a full one whatever its active lanes,
// so a serial chain of them is what a block reduction costs).  The totals end in thread 0's
// v[] (v[q] = 0 for q >= nsums).  The whole block must call it.
__device__ __forceinline__ void block_reduce(double (&v)[kNumSums], int nsums) {
  static_assert(kNumSums <= kWarps && kWarps == 8, "one warp per sum, 8 values per lane");
  __shared__ double red[kNumSums][kThreads];
  __shared__ double out[kNumSums];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) red[q][tid] = v[q];
  __syncthreads();
  if (warp < nsums) {
    const double* r = red[warp];
    const double a = (r[lane] + r[lane + 32]) + (r[lane + 64] + r[lane + 96]);
    const double b = (r[lane + 128] + r[lane + 160]) + (r[lane + 192] + r[lane + 224]);
    const double t = warp_sum(a + b);
    if (lane == 0) out[warp] = t;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) v[q] = q < nsums ? out[q] : 0.0;
  }
  __syncthreads();
}

// Sums the block's per-thread values (block_reduce), writes them to partials[blockIdx.x][*],
// and returns true in every thread of the block that finished last (all partials are then
// visible).  The whole block must call it; `counter` is reset by the caller's last block.
__device__ __forceinline__ bool block_sums_last(double (&s)[kNumSums], int nsums, double* partials,
                                                unsigned int* counter) {
  __shared__ bool is_last;
  block_reduce(s, nsums);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) partials[blockIdx.x * kNumSums + q] = s[q];
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Totals over the blocks' partials and, if bins is given, the long rows' epilogue contributions
// (all threads of the block call it; every thread gets the totals).  Warp q adds sum q: lane L
// the partials of blocks L, L + 32, ... and then of long rows L, L + 32, ..., in that order,
// then a butterfly over the lanes.
__device__ __forceinline__ void block_totals(const double* partials, int nblocks, int nsums,
                                             const BinTable* bins, double (&tot)[kNumSums]) {
  __shared__ double out[kNumSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < nsums) {
    double a = 0.0;
#pragma unroll 4
    for (int b = lane; b < nblocks; b += 32) a += __ldcg(partials + b * kNumSums + warp);
    if (bins) {
#pragma unroll 4
      for (int r = lane; r < bins->long_rows; r += 32) a += __ldcg(bins->contrib + r * kNumSums + warp);
    }
    a = warp_sum(a);
    if (lane == 0) out[warp] = a;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kNumSums; ++q) tot[q] = q < nsums ? out[q] : 0.0;
  __syncthreads();
}

}  // namespace pdhg
