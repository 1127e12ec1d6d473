// Host helpers shared by the single-instance runtime (solver.cu) and the batched one (batch.cu).
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "lp.h"

// Sets the calling thread's lp_last_error message (defined in solver.cu).
void pdhg_set_last_error(const std::string& msg);

namespace pdhg_host {

using pdhg::kWarps;

inline lp_status fail(lp_status code, const std::string& msg) {
  pdhg_set_last_error(msg);
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      lp_status code_ = (e_ == cudaErrorMemoryAllocation) ? LP_ERR_OUT_OF_MEMORY : LP_ERR_CUDA; \
      return ::pdhg_host::fail(code_, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

// Blocks for a binned kernel: at least two warp tasks per warp where there is enough work (the
// block reduction is a fixed cost per block), every SM busy where there is work for it, and
// no more blocks than fit on the device at once.
inline int grid_for_tasks(int64_t warp_tasks, int num_sms, int max_blocks) {
  int64_t g = (warp_tasks + 2 * kWarps - 1) / (2 * kWarps);
  int64_t spread = (warp_tasks + kWarps - 1) / kWarps;
  if (spread > num_sms) spread = num_sms;
  if (g < spread) g = spread;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

constexpr int kPwBatch = 16;  // power-iteration steps per host synchronisation

inline int grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

inline int length_class(int64_t len) {
  if (len <= 1) return 0;
  int c = 0;
  while ((int64_t(1) << c) < len) ++c;
  return c;  // ceil(log2(len))
}

// Stable order of indices by decreasing length class (counting sort over 32 classes).
inline void order_by_class(const std::vector<int64_t>& len, std::vector<int32_t>& perm) {
  const int32_t N = (int32_t)len.size();
  std::vector<int64_t> count(33, 0);
  for (int32_t i = 0; i < N; ++i) count[length_class(len[i])]++;
  std::vector<int64_t> start(33, 0);
  int64_t acc = 0;
  for (int c = 32; c >= 0; --c) {
    start[c] = acc;
    acc += count[c];
  }
  perm.assign(N, 0);
  for (int32_t i = 0; i < N; ++i) perm[start[length_class(len[i])]++] = i;
}

inline lp_status validate(int32_t m, int32_t n, int64_t nnz, const int64_t* rp, const int32_t* ci,
                   const double* val, const double* c, const double* lc, const double* uc,
                   const double* lv, const double* uv) {
  if (rp[0] != 0) return fail(LP_ERR_INVALID_INPUT, "row_ptr[0] must be 0");
  for (int32_t i = 0; i < m; ++i)
    if (rp[i + 1] < rp[i]) return fail(LP_ERR_INVALID_INPUT, "row_ptr must be non-decreasing (row " + std::to_string(i) + ")");
  if (rp[m] != nnz) return fail(LP_ERR_INVALID_INPUT, "row_ptr[m] must equal nnz");
  for (int64_t p = 0; p < nnz; ++p) {
    if (ci[p] < 0 || ci[p] >= n) return fail(LP_ERR_INVALID_INPUT, "column index out of range at entry " + std::to_string(p));
    if (!std::isfinite(val[p])) return fail(LP_ERR_INVALID_INPUT, "non-finite matrix entry at " + std::to_string(p));
  }
  for (int32_t j = 0; j < n; ++j) {
    if (!std::isfinite(c[j])) return fail(LP_ERR_INVALID_INPUT, "non-finite objective entry " + std::to_string(j));
    if (std::isnan(lv[j]) || std::isnan(uv[j]) || lv[j] > uv[j] || lv[j] == INFINITY || uv[j] == -INFINITY)
      return fail(LP_ERR_INVALID_INPUT, "bad variable bounds at column " + std::to_string(j));
  }
  for (int32_t i = 0; i < m; ++i) {
    if (std::isnan(lc[i]) || std::isnan(uc[i]) || lc[i] > uc[i] || lc[i] == INFINITY || uc[i] == -INFINITY)
      return fail(LP_ERR_INVALID_INPUT, "bad row bounds at row " + std::to_string(i));
  }
  return LP_OK;
}

// Tile shape of a length class whose longest row has Lc entries: G lanes per row so that a lane
// reads at most lane_target entries in one pass (G a power of two <= 32), 32 / G rows per pass,
// and R rows per tile (a power of two, at least one pass's rows, at most 32): a tile takes
// R * G / 32 passes, and its epilogue runs in R lanes at once.
struct TileShape {
  int lanes, rows, per_lane;
};
inline TileShape tile_shape(int64_t Lc, int lane_target, int tile_rows) {
  const int64_t rr = (int64_t)32 * lane_target / Lc;
  int R0 = (int)(rr < 1 ? 1 : (rr > 32 ? 32 : rr));
  int p = 1;
  while (p * 2 <= R0) p *= 2;
  R0 = p;
  int R = tile_rows < 1 ? 1 : (tile_rows > 32 ? 32 : tile_rows);
  p = 1;
  while (p * 2 <= R) p *= 2;
  R = p > R0 ? p : R0;
  TileShape t;
  t.lanes = 32 / R0;
  t.rows = R;
  t.per_lane = (int)((Lc + t.lanes - 1) / t.lanes);
  return t;
}

// Stable order of indices by decreasing length (counting sort over the distinct lengths).  A
// length class is then a contiguous run, and inside it the rows of one tile pass have nearly
// equal lengths, so a pass issues few entry slots that only some of its rows use.
inline void order_by_length(const std::vector<int64_t>& len, std::vector<int32_t>& perm) {
  const int32_t N = (int32_t)len.size();
  int64_t maxlen = 0;
  for (int32_t i = 0; i < N; ++i) maxlen = len[i] > maxlen ? len[i] : maxlen;
  std::vector<int64_t> start(maxlen + 2, 0);
  for (int32_t i = 0; i < N; ++i) start[maxlen - len[i] + 1]++;
  for (int64_t L = 1; L <= maxlen + 1; ++L) start[L] += start[L - 1];
  perm.assign(N, 0);
  for (int32_t i = 0; i < N; ++i) perm[start[maxlen - len[i]]++] = i;
}

// Range checks of lp_params (shared by lp_create, lp_set_params and lp_batch_create).
inline lp_status check_params(const lp_params& p) {
  if (!(p.gamma >= 0.0 && p.gamma <= 1.0)) return fail(LP_ERR_INVALID_ARG, "gamma must be in [0, 1]");
  if (!(p.beta_sufficient >= 0.0) || !(p.beta_necessary >= 0.0) || !(p.beta_artificial >= 0.0))
    return fail(LP_ERR_INVALID_ARG, "restart betas must be >= 0");
  if (!std::isfinite(p.k_p) || !std::isfinite(p.k_i) || !std::isfinite(p.k_d))
    return fail(LP_ERR_INVALID_ARG, "PID gains must be finite");
  if (!std::isfinite(p.eta)) return fail(LP_ERR_INVALID_ARG, "eta must be finite");
  if (!(p.omega0 > 0.0) || !std::isfinite(p.omega0)) return fail(LP_ERR_INVALID_ARG, "omega0 must be > 0");
  if (p.check_every < 1) return fail(LP_ERR_INVALID_ARG, "check_every must be >= 1");
  if (!(p.power_tol >= 0.0) || p.power_max_iter < 1) return fail(LP_ERR_INVALID_ARG, "bad power iteration settings");
  if (p.ruiz_iters < 0 || p.ruiz_iters > 1000) return fail(LP_ERR_INVALID_ARG, "ruiz_iters must be in [0, 1000]");
  if (p.pc_enabled && !(p.pc_alpha >= 0.0 && p.pc_alpha <= 2.0)) return fail(LP_ERR_INVALID_ARG, "pc_alpha must be in [0, 2]");
  if (p.trace_cap < 0) return fail(LP_ERR_INVALID_ARG, "trace_cap must be >= 0");
  if (p.unroll < 1 || p.unroll > 64) return fail(LP_ERR_INVALID_ARG, "unroll must be in [1, 64]");
  if (p.lane_target < 0 || p.lane_target > 64) return fail(LP_ERR_INVALID_ARG, "lane_target must be in [0, 64]");
  if (p.persistent < -1 || p.persistent > 3) return fail(LP_ERR_INVALID_ARG, "persistent must be -1, 0, 1, 2 or 3");
  if (p.precision < 0 || p.precision > 2) return fail(LP_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
  if (!(p.switch_tol >= 0.0)) return fail(LP_ERR_INVALID_ARG, "switch_tol must be >= 0");
  if (p.fp32_patience < 0) return fail(LP_ERR_INVALID_ARG, "fp32_patience must be >= 0");
  if (p.batch_local_nnz < 0) return fail(LP_ERR_INVALID_ARG, "batch_local_nnz must be >= 0");
  if (p.rescale < 0 || p.rescale > 1) return fail(LP_ERR_INVALID_ARG, "rescale must be 0 or 1");
  if (p.tile_rows < 0 || p.tile_rows > 32) return fail(LP_ERR_INVALID_ARG, "tile_rows must be in [0, 32]");
  return LP_OK;
}

// ||c~||_2 / ||finite (l_c~, u_c~)||_2 of preconditioned data (each norm taken as 1 when 0): the
// initial-weight factor that makes the plain iteration equal to the bound/objective-rescaled one.
inline double rescale_ratio(const double* c, int64_t n, const double* lc, const double* uc, int64_t m) {
  double c2 = 0.0, b2 = 0.0;
  for (int64_t j = 0; j < n; ++j) c2 += c[j] * c[j];
  for (int64_t i = 0; i < m; ++i) {
    if (std::isfinite(lc[i])) b2 += lc[i] * lc[i];
    if (std::isfinite(uc[i])) b2 += uc[i] * uc[i];
  }
  const double gamma = c2 > 0.0 ? std::sqrt(c2) : 1.0, beta = b2 > 0.0 ? std::sqrt(b2) : 1.0;
  return gamma / beta;
}

// Contiguous slices of `rows` rows (offsets rp) for `parts` CTAs, balanced by nonzeros plus
// kSmRowCost per row (the epilogue's share): bounds[q] = first row of slice q.
constexpr int64_t kSmRowCost = 12;
inline void sm_slices(const std::vector<int32_t>& rp, int parts, int32_t* bounds) {
  const int64_t rows = (int64_t)rp.size() - 1;
  const int64_t total = rp[rows] + kSmRowCost * rows;
  int64_t r = 0;
  bounds[0] = 0;
  for (int q = 1; q < parts; ++q) {
    const int64_t target = total * q / parts;
    while (r < rows && rp[r] + kSmRowCost * r < target) ++r;
    bounds[q] = (int32_t)r;
  }
  bounds[parts] = (int32_t)rows;
}

// Longest row (or column) the shared-memory loop takes: a row gets at most 8 lanes, so its
// chain of dependent fmas grows with its length.
constexpr int32_t kSmMaxLen = 128;

}  // namespace pdhg_host
