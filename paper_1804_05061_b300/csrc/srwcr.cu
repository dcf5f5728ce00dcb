// libsrwcr: host runtime and C ABI (see include/srwcr.h).
//
// One context = one fixed/moving pair with its pyramid.  Per evaluation the
// stream sees: memset(accumulators) -> k_accumulate -> k_finalize ->
// k_reduce_D [-> memset(g) -> k_adjoint].  The fixed-image statistics
// P[r][a] = sum_x w(r,x) h(a - A(x)) are computed once in srwcr_create.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "srwcr.h"
#include "kernels.cuh"
#include "kernels_mas_a.cuh"
#include "kernels_rows.cuh"
#include "kernels_rows_mas_a.cuh"
#include "kernels_rigid.cuh"

using namespace srwcr;

namespace {

thread_local std::string g_err;

srwcr_status fail(srwcr_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
srwcr_status fail(srwcr_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? SRWCR_ENOMEM : SRWCR_ECUDA,         \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                  __LINE__);                                                             \
  } while (0)

#define CKL()                                                                            \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return fail(SRWCR_ECUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                   \
  } while (0)

#define RET_IF(x)                        \
  do {                                   \
    srwcr_status s_ = (x);               \
    if (s_ != SRWCR_OK) return s_;       \
  } while (0)

constexpr int kBlock = 256;
constexpr int kMinBinsPerPass = 8;  // value kernel: fewest compacted bins per pass
// Levels above this many voxels recompute the warp in the adjoint by default
// instead of storing 16 bytes per voxel between the two passes.
constexpr long long kKeepWarpMaxVoxels = 1LL << 25;
constexpr size_t kSmemBudget = 112 * 1024;  // per CTA, two CTAs per SM

struct Level {
  Geo g{};                            // geometry of the kernels that run per evaluation
  Geo gv{};                           // general-path geometry (create-time statistics)
  void* A = nullptr;                  // normalised fixed image (storage type)
  void* M = nullptr;                  // normalised moving image (storage type)
  unsigned long long* S = nullptr;    // [R][nbins][2] fixed-point S1, S2 (also P scratch)
  double* P = nullptr;                // [R][nbins] sum_x w h(a - A)
  double* Wr = nullptr;               // [2R] sum_a P[r][a], then its reciprocals
  int* nz_ptr = nullptr;              // [R+1] bins with P > 0, compressed rows
  int* nz_bin = nullptr;              // [nnz]
  double* nz_inv_p = nullptr;         // [nnz] 1 / P
  float* U = nullptr;                 // [R]
  float* V = nullptr;                 // [R]
  float* X = nullptr;                 // [R][nbins] (M as A: mu_r(a) / sigma_r^2)
  float* Y2 = nullptr;                // M as A: [R][nbins] mu_r(a)^2 / sigma_r^2
  float2* DY = nullptr;               // M as A: [R][nbins] (Y2[a+1] - Y2[a], X[a+1] - X[a])
  double* Dr = nullptr;               // [R] share of D
  double* stats = nullptr;            // [R][4]
  double* D = nullptr;                // device scalar
  int* ndeg = nullptr;                // device scalar
  double Z = 0.0;
  float s1 = 1.f, s2 = 1.f;           // fixed-point scales of S1, S2
  float s0 = 1.f;                     // M as A: fixed-point scale of P
  size_t smem_acc = 0, smem_adj = 0;
  bool tables = false;
  // Row-parallel fast path (32-wide tiles): static per-row lane permutation
  // ordering voxels by fixed-image bin, x-bins per row (4, 8 or 12), smem sizes.
  bool rows = false;
  int nxb_rows = 0;
  unsigned char* perm = nullptr;
  unsigned* binmask = nullptr;        // per tile: fixed-image bins present
  float4* bg = nullptr;               // per voxel (B, dM/dy) of the last kept warp
  unsigned char* rowdist = nullptr;   // per 32-voxel row: static distance to nonzero M (capped)
  unsigned char* rowlive = nullptr;   // per row: nonzero dM/dy at the last kept warp
  std::vector<unsigned char> rowdist_host;   // host copy of rowdist (tile order)
  int* order = nullptr;               // row kernels: tile of each CTA, costly first (or NULL)
  int order_len = 0;                  // tiles in order (a launch of another size ignores it)
  float* uvxz = nullptr;              // U, V, X contracted over z per image plane
  float2* dyz = nullptr;              // M as A: table differences contracted over z per plane
  int* ubins = nullptr;               // fixed-image bins present in the image (any tile)
  int nu = 0;
  size_t smem_acc_rows = 0, smem_adj_rows = 0;
  std::vector<int> nz_ptr_host;       // host copy of nz_ptr (finalisation cost model)
  int fin_lanes = 32;                 // lanes per region of the sparse finalisation
};

}  // namespace

struct srwcr_bend_levels;  // bending-energy work per level (bending.cuh)

struct srwcr_ctx {
  srwcr_config cfg{};
  int nlev = 0;
  Level lev[4];
  cudaStream_t stream = nullptr;
  // A value+gradient call sums D on this second stream while the gradient
  // runs (fork after the finalisation, join before anything reads D).
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int device = 0;
  double* D_host = nullptr;   // pinned
  int* flag_host = nullptr;   // pinned
  int* flag_dev = nullptr;
  float* c_stage = nullptr;   // device staging for the host-buffer entry point
  float* g_stage = nullptr;
  double* D_stage = nullptr;
  int64_t stage_len = 0;
  // Benchmark hooks: kernels launched so far, and (when enabled) CUDA-event
  // pairs around each kernel on the context's stream.
  long long launches = 0;
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
  srwcr_bend_levels* bend = nullptr;  // created on first use
  float* rigid_tab = nullptr;         // rigid model: per-evaluation table (kRigidTab floats)
  double* rigid_acc = nullptr;        // rigid model: FP64 gradient accumulators [6]
  float* rigid_c = nullptr;           // rigid model: FFD form of the transform (level 0 size)
  float* rigid_g = nullptr;           // rigid model: dD/dc of that FFD form
  // Host-buffer entry point: the whole call (copies, check, value, gradient,
  // copies back) as one CUDA graph for the last (level, c, g) it served with
  // page-locked host buffers; dropped when a level's kernels are re-selected.
  cudaGraphExec_t host_graph = nullptr;
  cudaStream_t capture_stream = nullptr;  // the legacy default stream cannot be captured
  int host_graph_level = -1;
  const float* host_graph_c = nullptr;
  float* host_graph_g = nullptr;
  long long host_graph_launches = 0;  // kernels per replay
  // Device entry point (srwcr_value_and_grad_async): the second consecutive
  // call with the same (level, c, D, g) captures the call as one CUDA graph,
  // replayed while the arguments stay the same; dropped with the host graph.
  cudaGraphExec_t async_graph = nullptr;
  int async_level = -1;
  const float* async_c = nullptr;
  double* async_D = nullptr;
  float* async_g = nullptr;
  int async_repeats = 0;               // consecutive calls with these arguments (-1: capture failed)
  long long async_graph_launches = 0;  // kernels per replay
};

namespace {

int ceil_log2(double v) {
  int e = 0;
  while (std::ldexp(1.0, e) < v) ++e;
  return e;
}

// Cells spanned by a tile along one axis: max over tiles of
// cell(last voxel) - cell(first voxel) + 4 (bins cell..cell+3 per voxel).
int max_bins_per_tile(int n, int tile, int num, int den) {
  int best = 0;
  for (int s = 0; s < n; s += tile) {
    const int e = std::min(n - 1, s + tile - 1);
    const int c0 = (int)((long long)s * den / num), c1 = (int)((long long)e * den / num);
    best = std::max(best, c1 - c0 + 4);
  }
  return best;
}

size_t acc_smem(const Geo& g, int nch) {
  return (size_t)g.hb[0] * g.hb[1] * g.hb[2] * g.nbins * nch * sizeof(unsigned long long);
}

// Row kernels need 32-wide tiles, at most 12 spatial x-bins and 11 FFD
// x-nodes per row (FFD spacing >= 5, spatial-bin spacing >= 5).
bool rows_geometry_ok(const Geo& g) {
  return g.tile[0] == 32 && g.hb[0] <= 12 && g.hf[0] <= kMaxRowNodes && g.tile[1] * g.tile[2] <= 256;
}

void set_tile(Geo& g, int ndim, int tx, int ty, int tz) {
  g.tile[0] = tx; g.tile[1] = ty; g.tile[2] = ndim == 3 ? tz : 1;
  for (int d = 0; d < 3; ++d) g.ntile[d] = (g.n[d] + g.tile[d] - 1) / g.tile[d];
  for (int d = 0; d < 3; ++d) {
    if (d < ndim) {
      g.hb[d] = max_bins_per_tile(g.n[d], g.tile[d], g.sbn[d], g.sbd[d]);
      g.hf[d] = max_bins_per_tile(g.n[d], g.tile[d], g.fsp[d], 1);
    } else {
      g.hb[d] = 1; g.hf[d] = 1;
    }
  }
}

// nch: histogram channels of the general value kernel (2, or 3 with M as A).
srwcr_status choose_tile(Geo& g, int ndim, const int* req, int nch) {
  if (req[0] > 0) {
    set_tile(g, ndim, req[0], std::max(1, req[1]), std::max(1, req[2]));
    // The create-time statistics always run on the general kernels (one
    // channel); a 32-wide tile may leave the evaluations to the row kernels,
    // which is checked once those are selected.
    const size_t need = acc_smem(g, req[0] == 32 ? 1 : nch);
    if (need > 220 * 1024)
      return fail(SRWCR_EINVAL, "requested tile needs %zu bytes of shared memory", need);
    return SRWCR_OK;
  }
  static const int cand3[][3] = {{32, 32, 8}, {32, 16, 8}, {32, 8, 8}, {32, 8, 4}, {32, 4, 4}, {32, 4, 2},
                                 {32, 2, 2}, {16, 2, 2}, {8, 2, 2}, {8, 1, 1}, {4, 1, 1}};
  static const int cand2[][3] = {{32, 64, 1}, {32, 32, 1}, {32, 16, 1}, {32, 8, 1}, {32, 4, 1},
                                 {16, 4, 1}, {8, 2, 1}, {4, 1, 1}};
  const int (*cand)[3] = ndim == 3 ? cand3 : cand2;
  const int nc = ndim == 3 ? 11 : 8;
  for (int i = 0; i < nc; ++i) {
    set_tile(g, ndim, cand[i][0], cand[i][1], cand[i][2]);
    if (acc_smem(g, nch) <= kSmemBudget) return SRWCR_OK;
  }
  for (int i = 0; i < nc; ++i) {
    set_tile(g, ndim, cand[i][0], cand[i][1], cand[i][2]);
    if (acc_smem(g, nch) <= 220 * 1024) return SRWCR_OK;
  }
  return fail(SRWCR_EINVAL, "no voxel tile fits the shared-memory histogram (nbins=%d)",
              g.nbins);
}

srwcr_status make_geo(const srwcr_config& cfg, const int dims[3], Geo& g) {
  memset(&g, 0, sizeof g);
  const int nd = cfg.ndim;
  if (cfg.spatial != SRWCR_SPATIAL_BSPLINE && cfg.spatial != SRWCR_SPATIAL_BOXCAR)
    return fail(SRWCR_EINVAL, "unknown spatial distribution");
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < nd ? dims[d] : 1;
    if (d < nd && g.n[d] < 2) return fail(SRWCR_EINVAL, "dimension %d has %d < 2 voxels", d, g.n[d]);
    g.fsp[d] = d < nd ? cfg.ffd_spacing[d] : 1;
    g.nf[d] = d < nd ? (g.n[d] - 1) / g.fsp[d] + 4 : 1;
    if (d < nd && cfg.spatial == SRWCR_SPATIAL_BOXCAR && cfg.sbin_intervals[d] < 1)
      return fail(SRWCR_EINVAL, "boxcar patches need sbin_intervals > 0 on axis %d", d);
    if (d < nd && cfg.sbin_intervals[d] > 0) {
      if (cfg.sbin_intervals[d] > g.n[d])
        return fail(SRWCR_EINVAL, "more spatial-bin intervals than voxels on axis %d", d);
      g.sbn[d] = g.n[d];
      g.sbd[d] = cfg.sbin_intervals[d];
    } else {
      g.sbn[d] = d < nd ? g.fsp[d] : 1;
      g.sbd[d] = 1;
    }
    if ((long long)(g.n[d] - 1) * g.sbd[d] >= (1LL << 31))
      return fail(SRWCR_EINVAL, "spatial-bin arithmetic would overflow on axis %d", d);
    g.nsb[d] = d < nd ? (int)((long long)(g.n[d] - 1) * g.sbd[d] / g.sbn[d]) + 4 : 1;
    if (d < nd && cfg.spatial == SRWCR_SPATIAL_BOXCAR) g.nsb[d] = cfg.sbin_intervals[d];
  }
  g.boxcar = cfg.spatial == SRWCR_SPATIAL_BOXCAR ? 1 : 0;
  g.nbins = cfg.n_intensity_bins;
  g.nvox = (long long)g.n[0] * g.n[1] * g.n[2];
  g.ncoef = (long long)g.nf[0] * g.nf[1] * g.nf[2];
  g.R = (long long)g.nsb[0] * g.nsb[1] * g.nsb[2];
  g.nabin = g.nbins;
  g.cbin = g.nbins;
  return choose_tile(g, nd, cfg.tile, cfg.role == SRWCR_ROLE_M_AS_A ? 3 : 2);
}

// Fixed-point scales: every per-(r,a) total stays below 2^62.  A bin's
// support covers at most ~4 spacings per axis, so totals are bounded by that
// box's voxel count times the largest per-voxel term (1, L, L^2).
void fixed_scales(const Geo& g, int ndim, double* sP, double* s1, double* s2) {
  double box = 1.0;
  for (int d = 0; d < ndim; ++d) {
    const double span = std::min((double)g.n[d], std::floor(4.0 * g.sbn[d] / g.sbd[d]) + 2.0);
    box *= span;
  }
  box = std::min(box, (double)g.nvox);
  const double L = g.nbins - 1;
  *sP = std::ldexp(1.0, 62 - ceil_log2(box));
  *s1 = std::ldexp(1.0, 62 - ceil_log2(box * L));
  *s2 = std::ldexp(1.0, 62 - ceil_log2(box * L * L));
  // The row kernels add sums over at most two 32-voxel row segments (terms
  // <= L, L^2) into two 32-bit words (bits 0-23, 24-47), at most 256
  // updates per word per CTA: one update stays below 2^48, so no word
  // overflows.
  *s1 = std::min(*s1, std::ldexp(1.0, 48 - ceil_log2(64.0 * L)));
  *s2 = std::min(*s2, std::ldexp(1.0, 48 - ceil_log2(64.0 * L * L)));
}

// keep_warp: the value pass stores (B, dM/dy) per voxel for an adjoint at
// the same coefficients, which then reads it instead of recomputing the warp.
AccArgs acc_args(const Level& lv, const float* c, bool keep_warp) {
  AccArgs a;
  a.A = lv.A; a.M = lv.M; a.c = c; a.perm = lv.perm; a.binmask = lv.binmask;
  a.acc = lv.S; a.bg = keep_warp ? lv.bg : nullptr; a.s1 = lv.s1; a.s2 = lv.s2;
  a.rowdist = lv.rowdist;
  a.rowlive = keep_warp ? lv.rowlive : nullptr;
  return a;
}

AdjArgs adj_args(const Level& lv, const float* c, const float* gD, float* g, bool kept_warp) {
  AdjArgs a;
  a.A = lv.A; a.M = lv.M; a.c = c; a.perm = lv.perm; a.binmask = lv.binmask;
  a.U = lv.U; a.V = lv.V; a.X = lv.X; a.gscale = gD; a.bg = kept_warp ? lv.bg : nullptr;
  a.rowlive = kept_warp ? lv.rowlive : nullptr;
  a.uvxz = lv.uvxz;
  a.invZ = (float)(1.0 / lv.Z); a.grad = g;
  return a;
}

// The level's tile order if it was built for a launch of nblk tiles (the
// kernels read order[blockIdx.x]), else NULL: index order.
const int* tile_order(const Level& lv, int nblk) {
  return lv.order && lv.order_len == nblk ? lv.order : nullptr;
}

template <int DIM, typename T, bool SKIP>
void launch_rows_acc_s(srwcr_ctx* ctx, Level& lv, const AccArgs& a, int nblk) {
  const int* ord = tile_order(lv, nblk);
  if (lv.nxb_rows == 4)
    k_accumulate_rows<DIM, T, 4, SKIP><<<nblk, kAccWarps * 32, lv.smem_acc_rows, ctx->stream>>>(lv.g, a, ord);
  else if (lv.nxb_rows == 8)
    k_accumulate_rows<DIM, T, 8, SKIP><<<nblk, kAccWarps * 32, lv.smem_acc_rows, ctx->stream>>>(lv.g, a, ord);
  else
    k_accumulate_rows<DIM, T, 12, SKIP><<<nblk, kAccWarps * 32, lv.smem_acc_rows, ctx->stream>>>(lv.g, a, ord);
}

// Levels without the per-row records run the kernel with the per-row tests
// compiled out.
template <int DIM, typename T>
void launch_rows_acc(srwcr_ctx* ctx, Level& lv, const float* c, int nblk, bool keep) {
  const AccArgs a = acc_args(lv, c, keep);
  if (lv.rowdist) launch_rows_acc_s<DIM, T, true>(ctx, lv, a, nblk);
  else launch_rows_acc_s<DIM, T, false>(ctx, lv, a, nblk);
}

template <int DIM, typename T>
void launch_rows_adj(srwcr_ctx* ctx, Level& lv, const float* c, const float* gD, float* g,
                     int nblk, bool kept) {
  const AdjArgs a = adj_args(lv, c, gD, g, kept);
  const int* ord = tile_order(lv, nblk);
  if (lv.nxb_rows == 4)
    k_adjoint_rows<DIM, T, 4><<<nblk, kAdjWarps * 32, lv.smem_adj_rows, ctx->stream>>>(lv.g, a, ord);
  else if (lv.nxb_rows == 8)
    k_adjoint_rows<DIM, T, 8><<<nblk, kAdjWarps * 32, lv.smem_adj_rows, ctx->stream>>>(lv.g, a, ord);
  else
    k_adjoint_rows<DIM, T, 12><<<nblk, kAdjWarps * 32, lv.smem_adj_rows, ctx->stream>>>(lv.g, a, ord);
}

AccArgsA acc_args_a(const Level& lv, const float* c, bool keep_warp) {
  AccArgsA a;
  a.F = lv.A; a.M = lv.M; a.c = c; a.acc = lv.S; a.bg = keep_warp ? lv.bg : nullptr;
  a.rowdist = lv.rowdist; a.rowlive = keep_warp ? lv.rowlive : nullptr;
  a.s0 = lv.s0; a.s1 = lv.s1; a.s2 = lv.s2;
  return a;
}

template <int DIM, typename T>
void launch_rows_acc_mas_a(srwcr_ctx* ctx, Level& lv, const float* c, int nblk, bool keep) {
  const AccArgsA a = acc_args_a(lv, c, keep);
  const int* ord = tile_order(lv, nblk);
  const size_t sm = lv.smem_acc_rows;
  if (lv.nxb_rows == 4) k_accumulate_rows_mas_a<DIM, T, 4><<<nblk, kAccWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
  else if (lv.nxb_rows == 8) k_accumulate_rows_mas_a<DIM, T, 8><<<nblk, kAccWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
  else k_accumulate_rows_mas_a<DIM, T, 12><<<nblk, kAccWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
}

template <int DIM, typename T>
void launch_rows_adj_mas_a(srwcr_ctx* ctx, Level& lv, const float* c, const float* gD, float* g,
                           int nblk, bool kept) {
  AdjArgsA a;
  a.F = lv.A; a.M = lv.M; a.c = c; a.dyz = lv.dyz; a.gscale = gD;
  a.bg = kept ? lv.bg : nullptr; a.rowlive = kept ? lv.rowlive : nullptr;
  a.invZ = (float)(1.0 / lv.Z); a.grad = g;
  const int* ord = tile_order(lv, nblk);
  const size_t sm = lv.smem_adj_rows;
  if (lv.nxb_rows == 4) k_adjoint_rows_mas_a<DIM, T, 4><<<nblk, kAdjWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
  else if (lv.nxb_rows == 8) k_adjoint_rows_mas_a<DIM, T, 8><<<nblk, kAdjWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
  else k_adjoint_rows_mas_a<DIM, T, 12><<<nblk, kAdjWarps * 32, sm, ctx->stream>>>(lv.g, a, ord);
}

template <typename T>
srwcr_status launch_accumulate(srwcr_ctx* ctx, Level& lv, const float* c, bool stat, float s0,
                               float s1, bool keep_warp = false) {
  const Geo& gg = stat ? lv.gv : lv.g;
  const int nblk = gg.ntile[0] * gg.ntile[1] * gg.ntile[2];
  const T* A = (const T*)lv.A;
  const T* M = (const T*)lv.M;
  if (!stat && lv.rows) {
    if (ctx->cfg.role == SRWCR_ROLE_M_AS_A) {
      if (ctx->cfg.ndim == 3) launch_rows_acc_mas_a<3, T>(ctx, lv, c, nblk, keep_warp);
      else launch_rows_acc_mas_a<2, T>(ctx, lv, c, nblk, keep_warp);
    } else if (ctx->cfg.ndim == 3) {
      launch_rows_acc<3, T>(ctx, lv, c, nblk, keep_warp);
    } else {
      launch_rows_acc<2, T>(ctx, lv, c, nblk, keep_warp);
    }
    CKL();
    return SRWCR_OK;
  }
  if (!stat && ctx->cfg.role == SRWCR_ROLE_M_AS_A) {
    if (ctx->cfg.ndim == 3)
      k_accumulate_mas_a<3, T><<<nblk, kBlock, lv.smem_acc, ctx->stream>>>(gg, A, M, c, lv.S, lv.s0,
                                                                            lv.s1, lv.s2);
    else
      k_accumulate_mas_a<2, T><<<nblk, kBlock, lv.smem_acc, ctx->stream>>>(gg, A, M, c, lv.S, lv.s0,
                                                                            lv.s1, lv.s2);
    CKL();
    return SRWCR_OK;
  }
  const size_t sm = stat ? acc_smem(gg, 1) : lv.smem_acc;
  if (ctx->cfg.ndim == 3) {
    if (stat) k_accumulate<3, T, true><<<nblk, kBlock, sm, ctx->stream>>>(gg, A, M, c, lv.S, s0, s1);
    else k_accumulate<3, T, false><<<nblk, kBlock, sm, ctx->stream>>>(gg, A, M, c, lv.S, s0, s1);
  } else {
    if (stat) k_accumulate<2, T, true><<<nblk, kBlock, sm, ctx->stream>>>(gg, A, M, c, lv.S, s0, s1);
    else k_accumulate<2, T, false><<<nblk, kBlock, sm, ctx->stream>>>(gg, A, M, c, lv.S, s0, s1);
  }
  CKL();
  return SRWCR_OK;
}

template <typename T>
srwcr_status launch_adjoint(srwcr_ctx* ctx, Level& lv, const float* c, const float* gD, float* g,
                            bool kept_warp) {
  const int nblk = lv.g.ntile[0] * lv.g.ntile[1] * lv.g.ntile[2];
  const float invZ = (float)(1.0 / lv.Z);
  if (lv.rows && ctx->cfg.role == SRWCR_ROLE_M_AS_A) {
    // Per-plane z-contraction of the table differences, then the adjoint.
    const long long nz = zcontract_dy_len(lv.g);
    const int zb = (int)std::min<long long>(148 * 16, (nz + 255) / 256);
    if (ctx->cfg.ndim == 3) k_zcontract_dy<3><<<zb, 256, 0, ctx->stream>>>(lv.g, lv.DY, lv.dyz);
    else k_zcontract_dy<2><<<zb, 256, 0, ctx->stream>>>(lv.g, lv.DY, lv.dyz);
    CKL();
    ctx->launches += 1;
    if (ctx->cfg.ndim == 3) launch_rows_adj_mas_a<3, T>(ctx, lv, c, gD, g, nblk, kept_warp);
    else launch_rows_adj_mas_a<2, T>(ctx, lv, c, gD, g, nblk, kept_warp);
    CKL();
    return SRWCR_OK;
  }
  if (lv.rows) {
    // Per-plane z-contraction of the region tables, then the adjoint.
    // The contraction also clears g (see run_grad).  Blocks of 256 threads,
    // about 2 entries per thread (each entry waits on L2 loads), per image
    // plane.
    const long long ng = lv.g.ncoef * ctx->cfg.ndim;
    const long long per = (2LL + lv.nu) * lv.g.nsb[1] * lv.g.nsb[0];
    const dim3 zgrid((unsigned)std::max<long long>(1, std::min<long long>(128, (per + 511) / 512)),
                     (unsigned)lv.g.n[2]);
    if (ctx->cfg.ndim == 3)
      k_zcontract<3><<<zgrid, 256, 0, ctx->stream>>>(lv.g, lv.ubins, lv.nu, lv.U, lv.V, lv.X, lv.uvxz,
                                                     g, ng);
    else
      k_zcontract<2><<<zgrid, 256, 0, ctx->stream>>>(lv.g, lv.ubins, lv.nu, lv.U, lv.V, lv.X, lv.uvxz,
                                                     g, ng);
    CKL();
    ctx->launches += 1;
    if (ctx->cfg.ndim == 3) launch_rows_adj<3, T>(ctx, lv, c, gD, g, nblk, kept_warp);
    else launch_rows_adj<2, T>(ctx, lv, c, gD, g, nblk, kept_warp);
    CKL();
    return SRWCR_OK;
  }
  if (ctx->cfg.role == SRWCR_ROLE_M_AS_A) {
    if (ctx->cfg.ndim == 3)
      k_adjoint_mas_a<3, T><<<nblk, kBlock, lv.smem_adj, ctx->stream>>>(
          lv.g, (const T*)lv.A, (const T*)lv.M, c, lv.DY, gD, invZ, g);
    else
      k_adjoint_mas_a<2, T><<<nblk, kBlock, lv.smem_adj, ctx->stream>>>(
          lv.g, (const T*)lv.A, (const T*)lv.M, c, lv.DY, gD, invZ, g);
    CKL();
    return SRWCR_OK;
  }
  if (ctx->cfg.ndim == 3)
    k_adjoint<3, T><<<nblk, kBlock, lv.smem_adj, ctx->stream>>>(
        lv.g, (const T*)lv.A, (const T*)lv.M, c, lv.U, lv.V, lv.X, gD, invZ, g);
  else
    k_adjoint<2, T><<<nblk, kBlock, lv.smem_adj, ctx->stream>>>(
        lv.g, (const T*)lv.A, (const T*)lv.M, c, lv.U, lv.V, lv.X, gD, invZ, g);
  CKL();
  return SRWCR_OK;
}

template <typename T>
srwcr_status set_smem_limits() {
  const int mx = 227 * 1024;
  CK(cudaFuncSetAttribute(k_accumulate<3, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate<3, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate<2, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate<2, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate<3, T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate<2, T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_mas_a<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_mas_a<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_mas_a<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_mas_a<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 12, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 12, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 12, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 12, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<3, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<2, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<3, T, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows<2, T, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<3, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<3, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<2, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows<2, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<3, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<3, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<3, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<2, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<2, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_mas_a<2, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<3, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<3, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<3, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<2, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<2, T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_mas_a<2, T, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  return SRWCR_OK;
}

bool is_bf16(const srwcr_ctx* ctx) { return ctx->cfg.storage == SRWCR_STORAGE_BF16; }

// Kernel kinds reported by srwcr_profile_read.
enum { kProfAccumulate = 0, kProfFinalize = 1, kProfAdjoint = 2, kProfKinds = 3 };

// The cached host-call graph holds the kernels and buffers a level had when
// it was captured.
void drop_async_graph(srwcr_ctx* ctx) {
  if (ctx->async_graph) cudaGraphExecDestroy(ctx->async_graph);
  ctx->async_graph = nullptr;
  ctx->async_level = -1;
  ctx->async_c = nullptr;
  ctx->async_D = nullptr;
  ctx->async_g = nullptr;
  ctx->async_repeats = 0;
}

void drop_host_graph(srwcr_ctx* ctx) {
  if (ctx->host_graph) cudaGraphExecDestroy(ctx->host_graph);
  ctx->host_graph = nullptr;
  ctx->host_graph_level = -1;
  ctx->host_graph_c = nullptr;
  ctx->host_graph_g = nullptr;
  drop_async_graph(ctx);
}

cudaEvent_t prof_begin(srwcr_ctx* ctx) {
  if (!ctx->profiling) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, ctx->stream);
  return e;
}

void prof_end(srwcr_ctx* ctx, int kind, cudaEvent_t begin) {
  if (!ctx->profiling || !begin) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaEventDestroy(begin); return; }
  cudaEventRecord(e, ctx->stream);
  ctx->prof.push_back({kind, {begin, e}});
}

srwcr_status check_level(const srwcr_ctx* ctx, int level) {
  if (!ctx) return fail(SRWCR_EINVAL, "null context");
  if (level < 0 || level >= ctx->nlev)
    return fail(SRWCR_EINVAL, "level %d out of range [0, %d)", level, ctx->nlev);
  return SRWCR_OK;
}

RegionStatic region_static(const Level& lv) {
  RegionStatic rs;
  rs.W = lv.Wr;
  rs.inv_w = lv.Wr + lv.g.R;
  rs.ptr = lv.nz_ptr;
  rs.bin = lv.nz_bin;
  rs.inv_p = lv.nz_inv_p;
  return rs;
}

// FP64 issue model of the sparse finalisation with G lanes per region over
// the regions whose compressed-row offsets are `ptr`: a warp serves 32/G
// consecutive regions and issues, per group, a fixed ~32 FP64 operations
// (moments, one reciprocal, the region's outputs), ~6 per list entry over
// ceil(nnz / G) rounds of its slowest group, and ~1.5 per shuffle round.
// Returns the summed warp costs and raises *longest to the largest one.
double finalize_cost(const std::vector<int>& ptr, int G, double* longest) {
  const long long R = (long long)ptr.size() - 1;
  const int per = 32 / G;
  int lg = 0;
  while ((1 << lg) < G) ++lg;
  double sum = 0.0;
  for (long long w0 = 0; w0 < R; w0 += per) {
    int rounds = 0;
    for (long long r = w0; r < std::min(R, w0 + per); ++r)
      rounds = std::max(rounds, (ptr[r + 1] - ptr[r] + G - 1) / G);
    const double c = 32.0 + 6.0 * rounds + 1.5 * lg;
    sum += c;
    *longest = std::max(*longest, c);
  }
  return sum;
}

// Lanes per region minimising max(sum of warp costs / SM sub-partitions,
// longest warp) over one or more region lists (one per batch pair).
int finalize_lanes_auto(const std::vector<const std::vector<int>*>& lists, int device) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int best = 32;
  double best_t = 0.0;
  for (int G : kFinLanes) {
    double sum = 0.0, longest = 0.0;
    for (const auto* l : lists) sum += finalize_cost(*l, G, &longest);
    const double t = std::max(sum / (4.0 * sms), longest);
    if (G == kFinLanes[0] || t < best_t) {
      best = G;
      best_t = t;
    }
  }
  return best;
}

#define SRWCR_FIN_LANES_SWITCH(G, CALL) \
  switch (G) {                          \
    case 1: CALL(1); break;             \
    case 2: CALL(2); break;             \
    case 4: CALL(4); break;             \
    case 8: CALL(8); break;             \
    case 16: CALL(16); break;           \
    default: CALL(32); break;           \
  }

// Two warps per block for the finalisations: their lane groups are
// independent (no shared memory, no block barrier), and small blocks spread
// their few warps over every SM's FP64 unit (256-thread blocks left most SMs
// idle: 53 blocks for 847 regions at 16 lanes).
constexpr int kFinBlock = 64;

void launch_finalize_sparse(srwcr_ctx* ctx, const Level& lv) {
  const long long threads = ((lv.g.R * lv.fin_lanes + 31) / 32) * 32;
  const int blocks = (int)((threads + kFinBlock - 1) / kFinBlock);
  const RegionStatic rs = region_static(lv);
#define SRWCR_FIN_CALL(G)                                                                 \
  k_finalize_sparse<G><<<blocks, kFinBlock, 0, ctx->stream>>>(lv.g.R, lv.g.nbins, rs, lv.S,  \
                                                           1.0 / lv.s1, 1.0 / lv.s2,       \
                                                           1.0 / lv.Z, lv.U, lv.V, lv.X, \
                                                           lv.Dr, lv.stats)
  SRWCR_FIN_LANES_SWITCH(lv.fin_lanes, SRWCR_FIN_CALL)
#undef SRWCR_FIN_CALL
}

// (a) + (b): value into lv.D, tables into lv.U/V/X.  keep_warp: also store
// the per-voxel warp for a following run_grad(..., true) at the same c.
srwcr_status run_value(srwcr_ctx* ctx, Level& lv, const float* c, bool keep_warp,
                       bool reduce = true) {
  const bool mas_a = ctx->cfg.role == SRWCR_ROLE_M_AS_A;
  const size_t sbytes = (size_t)lv.g.R * lv.g.nbins * (mas_a ? 3 : 2) * sizeof(unsigned long long);
  CK(cudaMemsetAsync(lv.S, 0, sbytes, ctx->stream));
  cudaEvent_t ev = prof_begin(ctx);
  srwcr_status st =
      is_bf16(ctx) ? launch_accumulate<__nv_bfloat16>(ctx, lv, c, false, lv.s1, lv.s2, keep_warp)
                   : launch_accumulate<float>(ctx, lv, c, false, lv.s1, lv.s2, keep_warp);
  if (st != SRWCR_OK) return st;
  prof_end(ctx, kProfAccumulate, ev);
  const int fblk = (int)((lv.g.R * 32 + kFinBlock - 1) / kFinBlock);
  ev = prof_begin(ctx);
  if (mas_a)
    k_finalize_mas_a<<<fblk, kFinBlock, 0, ctx->stream>>>(lv.g, lv.S, 1.0 / lv.s0, 1.0 / lv.s1,
                                                       1.0 / lv.s2, 1.0 / lv.Z, lv.X, lv.Y2, lv.DY, lv.Dr,
                                                       lv.stats);
  else
    launch_finalize_sparse(ctx, lv);
  CKL();
  if (reduce) {
    k_reduce_D<<<1, 1024, 0, ctx->stream>>>(lv.Dr, lv.stats, lv.g.R, lv.D, lv.ndeg);
    CKL();
  }
  prof_end(ctx, kProfFinalize, ev);
  ctx->launches += 3;
  lv.tables = true;
  return SRWCR_OK;
}

// (c): gradient; kept_warp reads the warp stored by the preceding value pass
// at the same coefficients instead of recomputing it.
srwcr_status run_grad(srwcr_ctx* ctx, Level& lv, const float* c, const float* gD, float* g,
                      bool kept_warp) {
  // On row-kernel levels with the moving image as B the table contraction
  // that precedes the adjoint clears g itself.
  if (!(lv.rows && ctx->cfg.role == SRWCR_ROLE_M_AS_B))
    CK(cudaMemsetAsync(g, 0, sizeof(float) * lv.g.ncoef * ctx->cfg.ndim, ctx->stream));
  cudaEvent_t ev = prof_begin(ctx);
  RET_IF(is_bf16(ctx) ? launch_adjoint<__nv_bfloat16>(ctx, lv, c, gD, g, kept_warp)
                      : launch_adjoint<float>(ctx, lv, c, gD, g, kept_warp));
  prof_end(ctx, kProfAdjoint, ev);
  ctx->launches += 1;
  return SRWCR_OK;
}

// Value and gradient at the same c (the warp kept by the value pass where
// the level keeps it).  The value's final sum only feeds D, so it runs on
// the auxiliary stream beside the table contraction and the adjoint; the
// context's stream waits for it before returning, so whatever follows on
// that stream (D copies, line-search tests, a graph's end) sees D.  Inside
// a stream capture the fork and join become graph edges.
// D_copy: optional second place for D (see reduce_D_block).
srwcr_status run_value_and_grad(srwcr_ctx* ctx, Level& lv, const float* c, float* g,
                                double* D_copy = nullptr) {
  RET_IF(run_value(ctx, lv, c, true, false));
  CK(cudaEventRecord(ctx->fork_ev, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->fork_ev, 0));
  k_reduce_D<<<1, 1024, 0, ctx->aux_stream>>>(lv.Dr, lv.stats, lv.g.R, lv.D, lv.ndeg, D_copy);
  CKL();
  CK(cudaEventRecord(ctx->join_ev, ctx->aux_stream));
  const srwcr_status st = run_grad(ctx, lv, c, nullptr, g, true);
  CK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
  return st;
}

// Rigid model on the general kernels of the level: value into lv.D (and
// the tables); with g, dD/dmu (ndim translations, then the angles; an angle
// is mu * ang_scale radians).
template <typename T>
srwcr_status launch_rigid(srwcr_ctx* ctx, Level& lv, const float* g_unused, bool grad) {
  (void)g_unused;
  const Geo& gv = lv.gv;
  const int nblk = gv.ntile[0] * gv.ntile[1] * gv.ntile[2];
  const T* A = (const T*)lv.A;
  const T* M = (const T*)lv.M;
  if (!grad) {
    if (ctx->cfg.ndim == 3)
      k_accumulate<3, T, false, true><<<nblk, kBlock, lv.smem_acc, ctx->stream>>>(
          gv, A, M, ctx->rigid_tab, lv.S, lv.s1, lv.s2);
    else
      k_accumulate<2, T, false, true><<<nblk, kBlock, lv.smem_acc, ctx->stream>>>(
          gv, A, M, ctx->rigid_tab, lv.S, lv.s1, lv.s2);
  } else {
    const float invZ = (float)(1.0 / lv.Z);
    if (ctx->cfg.ndim == 3)
      k_adjoint_rigid<3, T><<<nblk, kBlock, 0, ctx->stream>>>(gv, A, M, ctx->rigid_tab, lv.U, lv.V,
                                                              lv.X, nullptr, invZ, ctx->rigid_acc);
    else
      k_adjoint_rigid<2, T><<<nblk, kBlock, 0, ctx->stream>>>(gv, A, M, ctx->rigid_tab, lv.U, lv.V,
                                                              lv.X, nullptr, invZ, ctx->rigid_acc);
  }
  CKL();
  return SRWCR_OK;
}

srwcr_status ensure_rigid(srwcr_ctx* ctx) {
  if (ctx->cfg.role != SRWCR_ROLE_M_AS_B)
    return fail(SRWCR_EINVAL, "the rigid model takes the moving image as B only");
  if (!ctx->rigid_tab) CK(cudaMalloc((void**)&ctx->rigid_tab, sizeof(float) * kRigidTab));
  if (!ctx->rigid_acc) CK(cudaMalloc((void**)&ctx->rigid_acc, sizeof(double) * 8));
  const size_t nc = (size_t)ctx->lev[0].g.ncoef * ctx->cfg.ndim;  // level 0 is the largest
  if (!ctx->rigid_c) CK(cudaMalloc((void**)&ctx->rigid_c, sizeof(float) * nc));
  if (!ctx->rigid_g) CK(cudaMalloc((void**)&ctx->rigid_g, sizeof(float) * nc));
  return SRWCR_OK;
}

// Value (and, with g != NULL, gradient) of the rigid model at mu.  On a
// row-parallel level the transform runs through the FFD kernels in its exact
// FFD form (the affine displacement sampled at the control nodes, which the
// cubic B-spline reproduces at every voxel, so D is the same function of mu)
// and dD/dmu is dD/dc chained through that form; otherwise the general
// per-voxel kernels take the rigid map directly.
srwcr_status run_rigid(srwcr_ctx* ctx, Level& lv, const float* mu, float* g, double ang_scale) {
  RET_IF(ensure_rigid(ctx));
  const Geo& gv = lv.gv;
  const int nd = ctx->cfg.ndim;
  k_rigid_setup<<<1, 32, 0, ctx->stream>>>(mu, nd, 0.5 * (gv.n[0] - 1), 0.5 * (gv.n[1] - 1),
                                           nd == 3 ? 0.5 * (gv.n[2] - 1) : 0.0, ang_scale,
                                           ctx->rigid_tab);
  CKL();
  ctx->launches += 1;
  if (lv.rows) {
    const int cb = (int)std::min<long long>(148 * 4, (gv.ncoef + 255) / 256);
    k_rigid_to_ffd<<<cb, 256, 0, ctx->stream>>>(gv, nd, ctx->rigid_tab, ctx->rigid_c);
    CKL();
    ctx->launches += 1;
    RET_IF(run_value(ctx, lv, ctx->rigid_c, g != nullptr));
    if (!g) return SRWCR_OK;
    RET_IF(run_grad(ctx, lv, ctx->rigid_c, nullptr, ctx->rigid_g, true));
    CK(cudaMemsetAsync(ctx->rigid_acc, 0, sizeof(double) * 8, ctx->stream));
    if (nd == 3) k_rigid_chain<3><<<cb, 256, 0, ctx->stream>>>(gv, ctx->rigid_tab, ctx->rigid_g, ctx->rigid_acc);
    else k_rigid_chain<2><<<cb, 256, 0, ctx->stream>>>(gv, ctx->rigid_tab, ctx->rigid_g, ctx->rigid_acc);
    CKL();
    k_rigid_grad_out<<<1, 32, 0, ctx->stream>>>(ctx->rigid_acc, nd, ang_scale, g);
    CKL();
    ctx->launches += 2;
    return SRWCR_OK;
  }
  CK(cudaMemsetAsync(lv.S, 0, (size_t)lv.g.R * lv.g.nbins * 2 * sizeof(unsigned long long),
                     ctx->stream));
  cudaEvent_t ev = prof_begin(ctx);
  RET_IF(is_bf16(ctx) ? launch_rigid<__nv_bfloat16>(ctx, lv, nullptr, false)
                      : launch_rigid<float>(ctx, lv, nullptr, false));
  prof_end(ctx, kProfAccumulate, ev);
  ev = prof_begin(ctx);
  launch_finalize_sparse(ctx, lv);
  CKL();
  k_reduce_D<<<1, 1024, 0, ctx->stream>>>(lv.Dr, lv.stats, lv.g.R, lv.D, lv.ndeg);
  CKL();
  prof_end(ctx, kProfFinalize, ev);
  ctx->launches += 3;
  lv.tables = true;
  if (!g) return SRWCR_OK;
  CK(cudaMemsetAsync(ctx->rigid_acc, 0, sizeof(double) * 8, ctx->stream));
  ev = prof_begin(ctx);
  RET_IF(is_bf16(ctx) ? launch_rigid<__nv_bfloat16>(ctx, lv, nullptr, true)
                      : launch_rigid<float>(ctx, lv, nullptr, true));
  prof_end(ctx, kProfAdjoint, ev);
  k_rigid_grad_out<<<1, 32, 0, ctx->stream>>>(ctx->rigid_acc, nd, ang_scale, g);
  CKL();
  ctx->launches += 2;
  return SRWCR_OK;
}

__global__ void k_check_finite(const float* __restrict__ c, long long n, int* __restrict__ flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(c[i])) flag[0] = 1;
}

// Copies n coefficients from page-locked host memory (read through its
// device mapping) into the device staging buffer, and stores 1 into the
// mapped host flag if any is not finite (the host clears the flag before
// the launch): the upload and the check of a host-buffer call in one kernel.
__global__ void k_stage_checked(const float* src, float* __restrict__ dst, long long n, int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = src[i];
    dst[i] = v;
    bad |= !isfinite(v);
  }
  if (bad) *reinterpret_cast<volatile int*>(flag) = 1;
}

// Copies n floats from device memory into page-locked host memory through
// its device mapping (coalesced stores over the bus): the gradient of a
// host-buffer call, without a copy-engine transfer.
__global__ void k_copy_to_mapped(const float* __restrict__ src, float* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

srwcr_status check_finite_async(srwcr_ctx* ctx, const float* c, long long n) {
  CK(cudaMemsetAsync(ctx->flag_dev, 0, sizeof(int), ctx->stream));
  k_check_finite<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, ctx->stream>>>(c, n, ctx->flag_dev);
  CKL();
  CK(cudaMemcpyAsync(ctx->flag_host, ctx->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  return SRWCR_OK;
}

srwcr_status finish_sync(srwcr_ctx* ctx, Level& lv, double* D_host) {
  CK(cudaMemcpyAsync(ctx->D_host, lv.D, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->flag_host[0]) return fail(SRWCR_ENUMERIC, "non-finite FFD coefficients");
  if (!std::isfinite(ctx->D_host[0])) return fail(SRWCR_ENUMERIC, "non-finite SRWCR value");
  if (D_host) *D_host = ctx->D_host[0];
  return SRWCR_OK;
}

void free_level(Level& lv) {
  void* ptrs[] = {lv.A, lv.M, lv.S, lv.P, lv.U, lv.V, lv.X, lv.Dr, lv.stats, lv.D, lv.ndeg, lv.perm,
                  lv.binmask, lv.Wr, lv.nz_ptr, lv.nz_bin, lv.nz_inv_p, lv.bg, lv.uvxz,
                  lv.ubins, lv.Y2, lv.DY, lv.rowdist, lv.rowlive, lv.dyz, lv.order};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  lv = Level();
}

template <typename T>
srwcr_status normalise_into(srwcr_ctx* ctx, const float* src_dev, long long n, T* out,
                            float* part, int nparts) {
  k_minmax_partial<<<nparts, 256, 0, ctx->stream>>>(src_dev, n, part);
  CKL();
  const double L = ctx->cfg.n_intensity_bins - 1;
  k_normalise<T><<<1024, 256, 0, ctx->stream>>>(src_dev, n, part, nparts, L, out);
  CKL();
  return SRWCR_OK;
}

}  // namespace

namespace {

template <typename T>
void launch_tile_binmask(srwcr_ctx* ctx, const Geo& g, const void* A, unsigned* mask) {
  if (ctx->cfg.ndim == 3) k_tile_binmask<3, T><<<1024, 256, 0, ctx->stream>>>(g, (const T*)A, mask);
  else k_tile_binmask<2, T><<<1024, 256, 0, ctx->stream>>>(g, (const T*)A, mask);
}

// Pick the largest 32-wide tile whose row kernels fit in shared memory.  The
// value kernel's histogram holds only the fixed-image bins a tile uses, so
// each candidate's per-tile masks are built on the device and the largest
// per-tile count sizes the histogram.  Levels without such a tile keep the
// general path.
// The row-parallel kernels serve both roles (either spatial distribution):
// with the moving image as B each row is ordered by the static fixed-image
// bin; with the moving image as A the lanes are grouped by the warped bin at
// every evaluation and the histogram holds every intensity bin.
bool rows_allowed(const srwcr_config& cfg) {
  return cfg.role == SRWCR_ROLE_M_AS_B || cfg.role == SRWCR_ROLE_M_AS_A;
}

// Moving image as A: the largest listed tile whose histogram (every bin)
// and tables fit in shared memory, with at most 128 rows per plane (an entry
// takes up to two updates per row, each < 2^48 in two 24-bit words).
srwcr_status build_tile_order(srwcr_ctx* ctx, Level& lv);

srwcr_status select_rows_path_mas_a(srwcr_ctx* ctx, Level& lv, const int* force_tile) {
  const srwcr_config& cfg = ctx->cfg;
  const int nd = cfg.ndim;
  static const int cand3[][3] = {{32, 64, 1}, {32, 32, 2}, {32, 16, 4}, {32, 32, 1}, {32, 16, 2},
                                 {32, 8, 4}, {32, 8, 2}, {32, 4, 2}, {32, 2, 2}, {32, 1, 1}};
  static const int cand2[][3] = {{32, 64, 1}, {32, 32, 1}, {32, 16, 1}, {32, 8, 1}, {32, 4, 1},
                                 {32, 1, 1}};
  std::vector<std::array<int, 3>> cands;
  if (force_tile) cands.push_back({force_tile[0], force_tile[1], force_tile[2]});
  else if (cfg.tile[0] > 0) {
    if (cfg.tile[0] == 32) cands.push_back({32, std::max(1, cfg.tile[1]), std::max(1, cfg.tile[2])});
  } else if (nd == 3) {
    for (auto& t : cand3) cands.push_back({t[0], t[1], t[2]});
  } else {
    for (auto& t : cand2) cands.push_back({t[0], t[1], t[2]});
  }
  for (const auto& t : cands) {
    Geo g = lv.gv;
    set_tile(g, nd, t[0], t[1], t[2]);
    if (!rows_geometry_ok(g) || g.tile[1] > 128) continue;
    const int nxb = g.hb[0] <= 4 ? 4 : (g.hb[0] <= 8 ? 8 : 12);
    const size_t sa = acc_rows_mas_a_smem_bytes(g, nd, nxb), sj = adj_rows_mas_a_smem_bytes(g, nd, nxb);
    if (sa > 220 * 1024 || sj > 220 * 1024) continue;
    lv.g = g;
    lv.rows = true;
    lv.nxb_rows = nxb;
    lv.smem_acc_rows = sa;
    lv.smem_adj_rows = sj;
    if (!lv.dyz) CK(cudaMalloc((void**)&lv.dyz, sizeof(float2) * zcontract_dy_len(g)));
    return build_tile_order(ctx, lv);   // a no-op before the row distances exist
  }
  return SRWCR_OK;
}

// Rows within this L-infinity distance of a nonzero moving-image voxel count
// toward a tile's cost in the launch order below.
constexpr unsigned char kOrderDist = 8;

// Launch order of the row kernels' tiles, on the host (see srwcr_tile_order):
// a tile's cost is its number of rows within kOrderDist of a nonzero
// moving-image voxel (the rows whose warp the value pass computes at
// moderate displacements; the adjoint visits the subset with a nonzero
// moving-image gradient), the tiles go out costly first (longest-first
// scheduling, so the launch ends on cheap tiles) in 16 cost classes, and
// tiles of one class keep their index order (neighbouring tiles, which read
// nearby moving-image voxels, still run close together in time).  n: voxels
// per axis (1 for an absent axis); tile: 32 x tile[1] x tile[2]; rowdist:
// [z][y][x block] with ceil(n[0] / 32) blocks per row; tiles numbered x
// block fastest, then y, then z, as the kernels number their CTAs.
void tile_order_host(const unsigned char* rowdist, const int n[3], const int tile[3],
                     std::vector<int>* order, std::vector<int>* cost) {
  const int nt0 = (n[0] + 31) / 32, nt1 = (n[1] + tile[1] - 1) / tile[1];
  const int nt2 = (n[2] + tile[2] - 1) / tile[2];
  const int ntiles = nt0 * nt1 * nt2;
  cost->assign(ntiles, 0);
  for (int t = 0; t < ntiles; ++t) {
    const int tx = t % nt0, ty = (t / nt0) % nt1, tz = t / (nt0 * nt1);
    const int y1 = std::min(n[1], (ty + 1) * tile[1]), z1 = std::min(n[2], (tz + 1) * tile[2]);
    int c = 0;
    for (int z = tz * tile[2]; z < z1; ++z)
      for (int y = ty * tile[1]; y < y1; ++y)
        c += rowdist[((size_t)z * n[1] + y) * nt0 + tx] <= kOrderDist;
    (*cost)[t] = c;
  }
  const long long cmax = *std::max_element(cost->begin(), cost->end());
  const std::vector<int>& cs = *cost;
  order->resize(ntiles);
  for (int t = 0; t < ntiles; ++t) (*order)[t] = t;
  std::stable_sort(order->begin(), order->end(), [&](int a, int b) {
    return cs[a] * 16LL / (cmax + 1) > cs[b] * 16LL / (cmax + 1);
  });
}

// The level's tile order on the device (levels with the per-row distances;
// others launch in index order).
srwcr_status build_tile_order(srwcr_ctx* ctx, Level& lv) {
  (void)ctx;
  if (lv.order) cudaFree(lv.order);
  lv.order = nullptr;
  lv.order_len = 0;
  if (!lv.rows || !lv.rowdist || lv.rowdist_host.empty()) return SRWCR_OK;
  std::vector<int> order, cost;
  tile_order_host(lv.rowdist_host.data(), lv.g.n, lv.g.tile, &order, &cost);
  const int ntiles = (int)order.size();
  if (ntiles != lv.g.ntile[0] * lv.g.ntile[1] * lv.g.ntile[2])
    return fail(SRWCR_EINVAL, "tile order: %d tiles against %d (internal)", ntiles,
                lv.g.ntile[0] * lv.g.ntile[1] * lv.g.ntile[2]);
  CK(cudaMalloc((void**)&lv.order, sizeof(int) * ntiles));
  CK(cudaMemcpy(lv.order, order.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice));
  lv.order_len = ntiles;
  return SRWCR_OK;
}

srwcr_status select_rows_path(srwcr_ctx* ctx, Level& lv, const int* force_tile = nullptr) {
  const srwcr_config& cfg = ctx->cfg;
  if (cfg.role == SRWCR_ROLE_M_AS_A) return select_rows_path_mas_a(ctx, lv, force_tile);
  const int nd = cfg.ndim;
  static const int cand3[][3] = {{32, 32, 4}, {32, 16, 4}, {32, 8, 4}, {32, 8, 2}, {32, 4, 2},
                                 {32, 2, 2}, {32, 1, 1}};
  static const int cand2[][3] = {{32, 64, 1}, {32, 32, 1}, {32, 16, 1}, {32, 8, 1}, {32, 4, 1},
                                 {32, 1, 1}};
  std::vector<std::array<int, 3>> cands;
  if (force_tile) {
    cands.push_back({force_tile[0], force_tile[1], force_tile[2]});
  } else if (cfg.tile[0] > 0) {
    if (cfg.tile[0] == 32) cands.push_back({32, std::max(1, cfg.tile[1]), std::max(1, cfg.tile[2])});
  } else if (nd == 3) {
    for (auto& t : cand3) cands.push_back({t[0], t[1], t[2]});
  } else {
    for (auto& t : cand2) cands.push_back({t[0], t[1], t[2]});
  }
  const int words = (lv.g.nbins + 31) / 32;
  std::vector<unsigned> hmask;
  for (const auto& t : cands) {
    Geo g = lv.gv;
    set_tile(g, nd, t[0], t[1], t[2]);
    if (!rows_geometry_ok(g)) continue;
    const size_t ntiles = (size_t)g.ntile[0] * g.ntile[1] * g.ntile[2];
    unsigned* mask = nullptr;
    CK(cudaMalloc((void**)&mask, sizeof(unsigned) * ntiles * words));
    CK(cudaMemsetAsync(mask, 0, sizeof(unsigned) * ntiles * words, ctx->stream));
    if (is_bf16(ctx)) launch_tile_binmask<__nv_bfloat16>(ctx, g, lv.A, mask);
    else launch_tile_binmask<float>(ctx, g, lv.A, mask);
    cudaError_t e = cudaGetLastError();
    hmask.assign(ntiles * words, 0u);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hmask.data(), mask, sizeof(unsigned) * ntiles * words,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      cudaFree(mask);
      return fail(SRWCR_ECUDA, "tile bin masks: %s", cudaGetErrorString(e));
    }
    int nab = 1;
    for (size_t tt = 0; tt < ntiles; ++tt) {
      int cnt = 0;
      for (int w = 0; w < words; ++w) cnt += __builtin_popcount(hmask[tt * words + w]);
      nab = std::max(nab, cnt);
    }
    if (!lv.ubins) {
      // Bins present anywhere in the image (the same for every tiling).
      std::vector<int> ub;
      for (int a = 0; a < lv.g.nbins; ++a) {
        bool any = false;
        for (size_t tt = 0; tt < ntiles && !any; ++tt) any = (hmask[tt * words + (a >> 5)] >> (a & 31)) & 1u;
        if (any) ub.push_back(a);
      }
      if (ub.empty()) ub.push_back(0);
      CK(cudaMalloc((void**)&lv.ubins, sizeof(int) * ub.size()));
      CK(cudaMemcpy(lv.ubins, ub.data(), sizeof(int) * ub.size(), cudaMemcpyHostToDevice));
      lv.nu = (int)ub.size();
    }
    g.nabin = nab;
    const int nxb = g.hb[0] <= 4 ? 4 : (g.hb[0] <= 8 ? 8 : 12);
    // Compacted bins per pass of the value kernel: all of them when they fit,
    // else the most that fit (a tile using more takes several passes).
    g.cbin = cfg.bins_per_pass > 0 ? std::min(nab, cfg.bins_per_pass) : nab;
    while (g.cbin > kMinBinsPerPass && acc_rows_smem_bytes(g, nd, nxb) > 220 * 1024) --g.cbin;
    const size_t sa = acc_rows_smem_bytes(g, nd, nxb), sj = adj_rows_smem_bytes(g, nd, nxb);
    if (sa > 220 * 1024 || sj > 220 * 1024) {
      cudaFree(mask);
      continue;
    }
    lv.g = g;
    lv.rows = true;
    lv.nxb_rows = nxb;
    lv.binmask = mask;
    lv.smem_acc_rows = sa;
    lv.smem_adj_rows = sj;
    const long long nrows = (long long)((g.n[0] + 31) / 32) * g.n[1] * g.n[2];
    CK(cudaMalloc((void**)&lv.perm, 32 * nrows));
    if (is_bf16(ctx)) k_row_perm<__nv_bfloat16><<<1024, 256, 0, ctx->stream>>>(g, (const __nv_bfloat16*)lv.A, lv.perm);
    else k_row_perm<float><<<1024, 256, 0, ctx->stream>>>(g, (const float*)lv.A, lv.perm);
    CKL();
    return build_tile_order(ctx, lv);   // a no-op before the row distances exist
  }
  return SRWCR_OK;
}

// Static per-row distance to the nearest nonzero moving-image voxel (the
// value pass skips rows that provably read only zeros) and the per-row
// record of a nonzero moving-image gradient the adjoint visits.
srwcr_status build_row_dist(srwcr_ctx* ctx, Level& lv) {
  const Geo& g = lv.g;
  const long long nrows = (long long)((g.n[0] + 31) / 32) * g.n[1] * g.n[2];
  CK(cudaMalloc((void**)&lv.rowdist, nrows));
  CK(cudaMalloc((void**)&lv.rowlive, nrows));
  CK(cudaMemsetAsync(lv.rowlive, 1, nrows, ctx->stream));
  unsigned char* d[2] = {nullptr, nullptr};
  CK(cudaMalloc((void**)&d[0], g.nvox));
  cudaError_t e = cudaMalloc((void**)&d[1], g.nvox);
  if (e != cudaSuccess) { cudaFree(d[0]); return fail(SRWCR_ENOMEM, "cudaMalloc failed"); }
  const int nb = (int)std::min<long long>(148 * 8, (g.nvox + 255) / 256);
  if (is_bf16(ctx)) k_mdist_x<__nv_bfloat16><<<nb, 256, 0, ctx->stream>>>(g, (const __nv_bfloat16*)lv.M, d[0]);
  else k_mdist_x<float><<<nb, 256, 0, ctx->stream>>>(g, (const float*)lv.M, d[0]);
  int cur = 0;
  for (int axis = 1; axis < ctx->cfg.ndim; ++axis, cur ^= 1)
    k_mdist_pass<<<nb, 256, 0, ctx->stream>>>(g, axis, d[cur], d[cur ^ 1]);
  k_row_dist<<<(int)std::min<long long>(148 * 8, (nrows + 255) / 256), 256, 0, ctx->stream>>>(g, d[cur], lv.rowdist);
  e = cudaGetLastError();
  std::vector<unsigned char> hd;
  if (e == cudaSuccess) {
    hd.resize(nrows);
    e = cudaMemcpyAsync(hd.data(), lv.rowdist, nrows, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d[0]);
  cudaFree(d[1]);
  if (e != cudaSuccess) return fail(SRWCR_ECUDA, "row distances: %s", cudaGetErrorString(e));
  // A level where no row lies farther than the stencil's reach from a
  // nonzero moving-image voxel can never skip a row: both records are
  // dropped there (every row is processed, without the per-row tests).
  const unsigned char far = *std::max_element(hd.begin(), hd.end());
  if ((float)far <= kDeadRowMargin) {
    cudaFree(lv.rowdist);
    cudaFree(lv.rowlive);
    lv.rowdist = nullptr;
    lv.rowlive = nullptr;
    return SRWCR_OK;
  }
  lv.rowdist_host = std::move(hd);
  return build_tile_order(ctx, lv);
}

void free_bend(srwcr_ctx* ctx);  // bending.cuh

}  // namespace

extern "C" {

const char* srwcr_last_error(void) { return g_err.c_str(); }

void srwcr_destroy(srwcr_ctx* ctx) {
  if (!ctx) return;
  free_bend(ctx);
  if (ctx->rigid_tab) cudaFree(ctx->rigid_tab);
  if (ctx->rigid_acc) cudaFree(ctx->rigid_acc);
  if (ctx->rigid_c) cudaFree(ctx->rigid_c);
  if (ctx->rigid_g) cudaFree(ctx->rigid_g);
  if (ctx->host_graph) cudaGraphExecDestroy(ctx->host_graph);
  if (ctx->async_graph) cudaGraphExecDestroy(ctx->async_graph);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  for (int l = 0; l < ctx->nlev; ++l) free_level(ctx->lev[l]);
  if (ctx->D_host) cudaFreeHost(ctx->D_host);
  if (ctx->flag_host) cudaFreeHost(ctx->flag_host);
  if (ctx->flag_dev) cudaFree(ctx->flag_dev);
  if (ctx->c_stage) cudaFree(ctx->c_stage);
  if (ctx->g_stage) cudaFree(ctx->g_stage);
  if (ctx->D_stage) cudaFree(ctx->D_stage);
  for (auto& p : ctx->prof) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  delete ctx;
}

static srwcr_status create_impl(const srwcr_config* cfg, const float* fixed, const float* moving,
                                int on_device, void* stream, srwcr_ctx* ctx) {
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)stream;
  CK(cudaGetDevice(&ctx->device));
  CK(cudaMallocHost((void**)&ctx->D_host, sizeof(double)));
  CK(cudaMallocHost((void**)&ctx->flag_host, sizeof(int)));
  ctx->flag_host[0] = 0;
  CK(cudaMalloc((void**)&ctx->flag_dev, sizeof(int)));
  CK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
  RET_IF(set_smem_limits<float>());
  RET_IF(set_smem_limits<__nv_bfloat16>());
  const size_t esz = is_bf16(ctx) ? 2 : 4;

  // Level geometry: level l halves every axis of level l-1 (floor).
  int dims[3] = {cfg->dims[0], cfg->dims[1], cfg->ndim == 3 ? cfg->dims[2] : 1};
  ctx->nlev = cfg->pyramid_levels;
  for (int l = 0; l < ctx->nlev; ++l) {
    if (l > 0)
      for (int d = 0; d < cfg->ndim; ++d) dims[d] /= 2;
    Level& lv = ctx->lev[l];
    RET_IF(make_geo(*cfg, dims, lv.g));
    const Geo& g = lv.g;
    CK(cudaMalloc(&lv.A, esz * g.nvox));
    CK(cudaMalloc(&lv.M, esz * g.nvox));
    const int nch = cfg->role == SRWCR_ROLE_M_AS_A ? 3 : 2;
    CK(cudaMalloc((void**)&lv.S, sizeof(unsigned long long) * g.R * g.nbins * nch));
    CK(cudaMalloc((void**)&lv.P, sizeof(double) * g.R * g.nbins));
    CK(cudaMalloc((void**)&lv.U, sizeof(float) * g.R));
    CK(cudaMalloc((void**)&lv.V, sizeof(float) * g.R));
    CK(cudaMalloc((void**)&lv.X, sizeof(float) * g.R * g.nbins));
    if (nch == 3) CK(cudaMalloc((void**)&lv.Y2, sizeof(float) * g.R * g.nbins));
    if (nch == 3) CK(cudaMalloc((void**)&lv.DY, sizeof(float2) * g.R * g.nbins));
    if (nch == 3) CK(cudaMemsetAsync(lv.DY, 0, sizeof(float2) * g.R * g.nbins, ctx->stream));
    CK(cudaMalloc((void**)&lv.Dr, sizeof(double) * g.R));
    CK(cudaMalloc((void**)&lv.stats, sizeof(double) * g.R * 4));
    CK(cudaMalloc((void**)&lv.D, sizeof(double)));
    CK(cudaMalloc((void**)&lv.ndeg, sizeof(int)));
    lv.smem_acc = acc_smem(g, nch);
    lv.smem_adj = sizeof(float) * cfg->ndim * g.hf[0] * g.hf[1] * g.hf[2];
    lv.gv = g;
  }

  // Normalise the two images into level 0 (Sec. II: [0, L_eps]).
  const long long n0 = ctx->lev[0].g.nvox;
  float* tmp = nullptr;
  float* part = nullptr;
  const int nparts = 512;
  CK(cudaMalloc((void**)&tmp, sizeof(float) * n0));
  cudaError_t e = cudaMalloc((void**)&part, sizeof(float) * 2 * nparts);
  if (e != cudaSuccess) { cudaFree(tmp); return fail(SRWCR_ENOMEM, "cudaMalloc failed"); }
  srwcr_status st = SRWCR_OK;
  const float* src[2] = {fixed, moving};
  void* dst[2] = {ctx->lev[0].A, ctx->lev[0].M};
  for (int im = 0; im < 2 && st == SRWCR_OK; ++im) {
    e = cudaMemcpyAsync(tmp, src[im], sizeof(float) * n0,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) { st = fail(SRWCR_ECUDA, "image upload: %s", cudaGetErrorString(e)); break; }
    // Reject constant images (max == min) before dividing by zero.
    k_minmax_partial<<<nparts, 256, 0, ctx->stream>>>(tmp, n0, part);
    float hpart[2 * nparts];
    e = cudaMemcpyAsync(hpart, part, sizeof hpart, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { st = fail(SRWCR_ECUDA, "min/max: %s", cudaGetErrorString(e)); break; }
    float mn = INFINITY, mx = -INFINITY;
    for (int i = 0; i < nparts; ++i) { mn = std::min(mn, hpart[2 * i]); mx = std::max(mx, hpart[2 * i + 1]); }
    if (!(mx > mn) || !std::isfinite(mn) || !std::isfinite(mx)) {
      st = fail(SRWCR_EINVAL, "%s image is constant or not finite", im ? "moving" : "fixed");
      break;
    }
    st = is_bf16(ctx) ? normalise_into(ctx, tmp, n0, (__nv_bfloat16*)dst[im], part, nparts)
                      : normalise_into(ctx, tmp, n0, (float*)dst[im], part, nparts);
    if (st == SRWCR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      st = fail(SRWCR_ECUDA, "normalisation failed");
  }
  cudaFree(tmp);
  cudaFree(part);
  RET_IF(st);

  // Pyramid.
  for (int l = 1; l < ctx->nlev; ++l) {
    const Geo& gi = ctx->lev[l - 1].g;
    const Geo& go = ctx->lev[l].g;
    for (int im = 0; im < 2; ++im) {
      const void* in = im ? ctx->lev[l - 1].M : ctx->lev[l - 1].A;
      void* out = im ? ctx->lev[l].M : ctx->lev[l].A;
      if (cfg->ndim == 3) {
        if (is_bf16(ctx)) k_downsample<3, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>((const __nv_bfloat16*)in, gi.n[0], gi.n[1], (__nv_bfloat16*)out, go.n[0], go.n[1], go.n[2]);
        else k_downsample<3, float><<<1024, 256, 0, ctx->stream>>>((const float*)in, gi.n[0], gi.n[1], (float*)out, go.n[0], go.n[1], go.n[2]);
      } else {
        if (is_bf16(ctx)) k_downsample<2, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>((const __nv_bfloat16*)in, gi.n[0], gi.n[1], (__nv_bfloat16*)out, go.n[0], go.n[1], go.n[2]);
        else k_downsample<2, float><<<1024, 256, 0, ctx->stream>>>((const float*)in, gi.n[0], gi.n[1], (float*)out, go.n[0], go.n[1], go.n[2]);
      }
      CKL();
    }
  }

  // Row-parallel path: tile, per-tile fixed-image bin masks and per-row
  // lane permutations (A is fixed); storage for the warp the value pass
  // keeps for the adjoint (16 bytes per voxel).
  for (int l = 0; l < ctx->nlev; ++l) {
    Level& lv = ctx->lev[l];
    // The row kernels sort each row's voxels by the static fixed-image bin;
    // with the moving image as A the binned image moves, so the general
    // per-voxel kernels run.
    if (rows_allowed(*cfg)) RET_IF(select_rows_path(ctx, lv));
    if (!lv.rows && lv.smem_acc > 220 * 1024)
      return fail(SRWCR_EINVAL,
                  "requested tile needs %zu bytes of shared memory on the general kernels, and the "
                  "row kernels cannot take level %d", lv.smem_acc, l);
    if (lv.rows) {
      const bool keep = cfg->keep_warp > 0 || (cfg->keep_warp == 0 && lv.g.nvox <= kKeepWarpMaxVoxels);
      if (keep) CK(cudaMalloc((void**)&lv.bg, sizeof(float4) * lv.g.nvox));
      CK(cudaMalloc((void**)&lv.uvxz, sizeof(float) * zcontract_len(lv.g)));
      RET_IF(build_row_dist(ctx, lv));
    }
  }

  // Static fixed-image statistics P[r][a] and Z = sum P.
  for (int l = 0; l < ctx->nlev; ++l) {
    Level& lv = ctx->lev[l];
    double sP, s1, s2;
    fixed_scales(lv.g, cfg->ndim, &sP, &s1, &s2);
    lv.s1 = (float)s1;
    lv.s0 = (float)sP;
    lv.s2 = (float)s2;
    // Moving image as A on the row kernels: P is accumulated per evaluation
    // from sums over at most 64 voxels of weights <= 1 per row update, each
    // kept below 2^48 like the moments.
    if (cfg->role == SRWCR_ROLE_M_AS_A && lv.rows) lv.s0 = (float)std::min(sP, std::ldexp(1.0, 42));
    CK(cudaMemsetAsync(lv.S, 0, sizeof(unsigned long long) * lv.g.R * lv.g.nbins, ctx->stream));
    RET_IF(is_bf16(ctx) ? launch_accumulate<__nv_bfloat16>(ctx, lv, nullptr, true, (float)sP, 0.f)
                        : launch_accumulate<float>(ctx, lv, nullptr, true, (float)sP, 0.f));
    const long long n = lv.g.R * lv.g.nbins;
    k_fixed_to_double<<<256, 256, 0, ctx->stream>>>(lv.S, 1.0 / sP, lv.P, n);
    CKL();
    double* hP = (double*)malloc(sizeof(double) * n);
    if (!hP) return fail(SRWCR_ENOMEM, "host allocation failed");
    e = cudaMemcpyAsync(hP, lv.P, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free(hP); return fail(SRWCR_ECUDA, "P readback: %s", cudaGetErrorString(e)); }
    double Z = 0.0;
    for (long long i = 0; i < n; ++i) Z += hP[i];
    // Static per-region data of the finalisation (bins with P > 0).
    const int nb = lv.g.nbins;
    std::vector<double> Wr(2 * lv.g.R), inv_p;
    std::vector<int> ptr(lv.g.R + 1, 0), bin;
    for (long long r = 0; r < lv.g.R; ++r) {
      double w = 0.0;
      for (int a = 0; a < nb; ++a) {
        const double p = hP[r * nb + a];
        w += p;
        if (p > 0.0) {
          bin.push_back(a);
          inv_p.push_back(1.0 / p);
        }
      }
      Wr[r] = w;
      Wr[lv.g.R + r] = w > 0.0 ? 1.0 / w : 0.0;
      ptr[r + 1] = (int)bin.size();
    }
    free(hP);
    const size_t nnz = std::max<size_t>(bin.size(), 1);
    CK(cudaMalloc((void**)&lv.Wr, sizeof(double) * 2 * lv.g.R));
    CK(cudaMalloc((void**)&lv.nz_ptr, sizeof(int) * (lv.g.R + 1)));
    CK(cudaMalloc((void**)&lv.nz_bin, sizeof(int) * nnz));
    CK(cudaMalloc((void**)&lv.nz_inv_p, sizeof(double) * nnz));
    CK(cudaMemcpy(lv.Wr, Wr.data(), sizeof(double) * 2 * lv.g.R, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(lv.nz_ptr, ptr.data(), sizeof(int) * (lv.g.R + 1), cudaMemcpyHostToDevice));
    if (!bin.empty()) {
      CK(cudaMemcpy(lv.nz_bin, bin.data(), sizeof(int) * bin.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(lv.nz_inv_p, inv_p.data(), sizeof(double) * bin.size(), cudaMemcpyHostToDevice));
    }
    lv.fin_lanes = cfg->finalize_lanes > 0 ? cfg->finalize_lanes
                                           : finalize_lanes_auto({&ptr}, ctx->device);
    lv.nz_ptr_host = std::move(ptr);
    // X entries of bins with P = 0 are never written by the finalisation.
    CK(cudaMemsetAsync(lv.X, 0, sizeof(float) * lv.g.R * nb, ctx->stream));
    lv.Z = Z;
    if (!(Z > 0.0)) return fail(SRWCR_EINVAL, "empty fixed-image statistics at level %d", l);
  }
  return SRWCR_OK;
}

srwcr_status srwcr_create(const srwcr_config* cfg, const float* fixed, const float* moving,
                          int images_on_device, void* stream, srwcr_ctx** out) {
  if (!out) return fail(SRWCR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !fixed || !moving) return fail(SRWCR_EINVAL, "null argument");
  if (cfg->ndim != 2 && cfg->ndim != 3) return fail(SRWCR_EINVAL, "ndim must be 2 or 3");
  if (cfg->n_intensity_bins < 2 || cfg->n_intensity_bins > 256)
    return fail(SRWCR_EINVAL, "n_intensity_bins must be in [2, 256]");
  if (cfg->storage != SRWCR_STORAGE_F32 && cfg->storage != SRWCR_STORAGE_BF16)
    return fail(SRWCR_EINVAL, "unknown storage type");
  if (cfg->pyramid_levels < 1 || cfg->pyramid_levels > 4)
    return fail(SRWCR_EINVAL, "pyramid_levels must be in [1, 4]");
  for (int d = 0; d < cfg->ndim; ++d) {
    if (cfg->dims[d] < 2 || cfg->dims[d] > 65535) return fail(SRWCR_EINVAL, "dims[%d] out of range", d);
    if (cfg->ffd_spacing[d] < 1 || cfg->ffd_spacing[d] > cfg->dims[d])
      return fail(SRWCR_EINVAL, "ffd_spacing[%d] out of range", d);
    if (cfg->sbin_intervals[d] < 0) return fail(SRWCR_EINVAL, "negative sbin_intervals");
    if ((cfg->dims[d] >> (cfg->pyramid_levels - 1)) < 2)
      return fail(SRWCR_EINVAL, "too many pyramid levels for dims[%d]", d);
  }
  if (cfg->tile[0] < 0 || cfg->tile[1] < 0 || cfg->tile[2] < 0)
    return fail(SRWCR_EINVAL, "negative tile size");
  if (cfg->bins_per_pass < 0) return fail(SRWCR_EINVAL, "negative bins_per_pass");
  if (cfg->role != SRWCR_ROLE_M_AS_B && cfg->role != SRWCR_ROLE_M_AS_A)
    return fail(SRWCR_EINVAL, "unknown role");
  if (cfg->keep_warp < -1 || cfg->keep_warp > 1) return fail(SRWCR_EINVAL, "keep_warp must be -1, 0 or 1");
  if (cfg->finalize_lanes != 0 && cfg->finalize_lanes != 1 && cfg->finalize_lanes != 2 &&
      cfg->finalize_lanes != 4 && cfg->finalize_lanes != 8 && cfg->finalize_lanes != 16 &&
      cfg->finalize_lanes != 32)
    return fail(SRWCR_EINVAL, "finalize_lanes must be 0, 1, 2, 4, 8, 16 or 32");
  if (cfg->spatial != SRWCR_SPATIAL_BSPLINE && cfg->spatial != SRWCR_SPATIAL_BOXCAR)
    return fail(SRWCR_EINVAL, "unknown spatial distribution");
  for (int d = 0; d < cfg->ndim && cfg->spatial == SRWCR_SPATIAL_BOXCAR; ++d)
    if (cfg->sbin_intervals[d] < 1)
      return fail(SRWCR_EINVAL, "boxcar patches need sbin_intervals > 0 on axis %d", d);
  srwcr_ctx* ctx = new (std::nothrow) srwcr_ctx();
  if (!ctx) return fail(SRWCR_ENOMEM, "host allocation failed");
  srwcr_status st = create_impl(cfg, fixed, moving, images_on_device, stream, ctx);
  if (st != SRWCR_OK) {
    std::string keep = g_err;
    srwcr_destroy(ctx);
    g_err = keep;
    return st;
  }
  *out = ctx;
  return SRWCR_OK;
}

srwcr_status srwcr_level_info(const srwcr_ctx* ctx, int level, srwcr_level_desc* out) {
  RET_IF(check_level(ctx, level));
  if (!out) return fail(SRWCR_EINVAL, "out is NULL");
  const Geo& g = ctx->lev[level].g;
  for (int d = 0; d < 3; ++d) {
    out->dims[d] = g.n[d];
    out->ffd_nodes[d] = g.nf[d];
    out->sbins[d] = g.nsb[d];
    out->tile[d] = g.tile[d];
  }
  out->n_voxels = g.nvox;
  out->n_params = g.ncoef * ctx->cfg.ndim;
  out->n_regions = g.R;
  out->kernel_path = ctx->lev[level].rows ? 1 : 0;
  out->finalize_lanes = ctx->lev[level].fin_lanes;
  return SRWCR_OK;
}

srwcr_status srwcr_value(srwcr_ctx* ctx, int level, const float* c_dev, double* D_host) {
  RET_IF(check_level(ctx, level));
  if (!c_dev) return fail(SRWCR_EINVAL, "c_dev is NULL");
  Level& lv = ctx->lev[level];
  RET_IF(check_finite_async(ctx, c_dev, lv.g.ncoef * ctx->cfg.ndim));
  RET_IF(run_value(ctx, lv, c_dev, false));
  return finish_sync(ctx, lv, D_host);
}

srwcr_status srwcr_value_and_grad(srwcr_ctx* ctx, int level, const float* c_dev, double* D_host,
                                  float* g_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !g_dev) return fail(SRWCR_EINVAL, "null device pointer");
  Level& lv = ctx->lev[level];
  RET_IF(check_finite_async(ctx, c_dev, lv.g.ncoef * ctx->cfg.ndim));
  RET_IF(run_value_and_grad(ctx, lv, c_dev, g_dev));
  return finish_sync(ctx, lv, D_host);
}

namespace {

// One device-buffer call on ctx->stream: value (keeping the warp), gradient,
// and D, which the value's final sum also stores into D_dev.
srwcr_status queue_async_call(srwcr_ctx* ctx, Level& lv, const float* c_dev, double* D_dev,
                              float* g_dev) {
  RET_IF(run_value_and_grad(ctx, lv, c_dev, g_dev, D_dev));
  return SRWCR_OK;
}

// Captures queue_async_call into ctx->async_graph on the private capture
// stream (nothing runs); on failure the graph stays empty.
void capture_async_call(srwcr_ctx* ctx, int level, const float* c_dev, double* D_dev,
                        float* g_dev) {
  if (!ctx->capture_stream &&
      cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->capture_stream = nullptr;
    return;
  }
  cudaStream_t user = ctx->stream;
  const long long launches = ctx->launches;
  ctx->stream = ctx->capture_stream;
  cudaGraph_t graph = nullptr;
  srwcr_status st = SRWCR_ECUDA;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    st = queue_async_call(ctx, ctx->lev[level], c_dev, D_dev, g_dev);
    if (cudaStreamEndCapture(ctx->stream, &graph) != cudaSuccess) st = SRWCR_ECUDA;
  }
  ctx->stream = user;
  ctx->async_graph_launches = ctx->launches - launches;
  ctx->launches = launches;
  cudaGraphExec_t exec = nullptr;
  if (st == SRWCR_OK && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
    ctx->async_graph = exec;
  else
    ctx->async_repeats = -1;  // no further attempt for these arguments
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

}  // namespace

srwcr_status srwcr_value_and_grad_async(srwcr_ctx* ctx, int level, const float* c_dev,
                                        double* D_dev, float* g_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !g_dev || !D_dev) return fail(SRWCR_EINVAL, "null device pointer");
  Level& lv = ctx->lev[level];
  // Repeated calls with the same buffers (an optimiser's loop) replay one
  // graph: fewer launch gaps.  Not while the caller's stream is being
  // captured (the call then becomes part of the caller's graph as it is) or
  // while the per-kernel profiling events are on.
  if (!(ctx->async_level == level && ctx->async_c == c_dev && ctx->async_D == D_dev &&
        ctx->async_g == g_dev)) {
    drop_async_graph(ctx);
    ctx->async_level = level;
    ctx->async_c = c_dev;
    ctx->async_D = D_dev;
    ctx->async_g = g_dev;
  }
  if (ctx->async_repeats >= 0 && ctx->async_repeats < 2) ++ctx->async_repeats;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess ||
                         cap != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();
  if (!capturing && !ctx->profiling && ctx->async_repeats >= 2) {
    if (!ctx->async_graph) capture_async_call(ctx, level, c_dev, D_dev, g_dev);
    if (ctx->async_graph) {
      CK(cudaGraphLaunch(ctx->async_graph, ctx->stream));
      ctx->launches += ctx->async_graph_launches;
      lv.tables = true;
      return SRWCR_OK;
    }
  }
  return queue_async_call(ctx, lv, c_dev, D_dev, g_dev);
}

namespace {

// The device address through which the page-locked host byte at p is
// reached (null if p is not page-locked).
void* host_byte_alias(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The device address of the n bytes at p (n > 0), or null unless both ends
// lie in page-locked memory mapped at one contiguous device range: a buffer
// that ends in pageable memory (shorter than the caller claims, or running
// past its registration) is never read or written through the mapping or by
// a direct copy, but takes the copy path through pageable memory.
void* host_device_alias(const void* p, size_t n) {
  char* a0 = static_cast<char*>(host_byte_alias(p));
  if (!a0) return nullptr;
  const char* a1 = static_cast<const char*>(host_byte_alias(static_cast<const char*>(p) + (n - 1)));
  return a1 == a0 + (n - 1) ? a0 : nullptr;
}

bool host_page_locked(const void* p, size_t n) { return host_device_alias(p, n) != nullptr; }

// One host-buffer call on ctx->stream: copy c in, check it, value and
// gradient, copy g and D out (the caller synchronises).
// With c_host and the context's flag and D words device-mapped (page-locked
// buffers), one kernel uploads and checks c and the value's sum stores D
// into host memory itself, and with g_host page-locked too a kernel writes g
// through its mapping: no copy-engine transfer and no memset instead of
// four copies and a memset; the host clears the flag before each launch.
srwcr_status queue_host_call(srwcr_ctx* ctx, Level& lv, int64_t np, const float* c_host,
                             float* g_host) {
  const float* c_map = static_cast<const float*>(host_device_alias(c_host, sizeof(float) * np));
  int* flag_map = static_cast<int*>(host_device_alias(ctx->flag_host, sizeof(int)));
  double* D_map = static_cast<double*>(host_device_alias(ctx->D_host, sizeof(double)));
  if (c_map && flag_map && D_map) {
    const int blocks = (int)std::min<int64_t>(4 * 148, (np + 255) / 256);
    k_stage_checked<<<blocks, 256, 0, ctx->stream>>>(c_map, ctx->c_stage, np, flag_map);
    CKL();
    ctx->launches += 1;
    RET_IF(run_value_and_grad(ctx, lv, ctx->c_stage, ctx->g_stage, D_map));
    // A page-locked g_host is written by a kernel through its mapping too
    // (about 2.5 us per call less than a copy-engine transfer of 220 KB).
    float* g_map = static_cast<float*>(host_device_alias(g_host, sizeof(float) * np));
    if (g_map) {
      k_copy_to_mapped<<<blocks, 256, 0, ctx->stream>>>(ctx->g_stage, g_map, np);
      CKL();
      ctx->launches += 1;
    } else {
      CK(cudaMemcpyAsync(g_host, ctx->g_stage, sizeof(float) * np, cudaMemcpyDeviceToHost, ctx->stream));
    }
    return SRWCR_OK;
  }
  CK(cudaMemcpyAsync(ctx->c_stage, c_host, sizeof(float) * np, cudaMemcpyHostToDevice, ctx->stream));
  RET_IF(check_finite_async(ctx, ctx->c_stage, np));
  RET_IF(run_value_and_grad(ctx, lv, ctx->c_stage, ctx->g_stage));
  CK(cudaMemcpyAsync(g_host, ctx->g_stage, sizeof(float) * np, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->D_host, lv.D, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return SRWCR_OK;
}

// Captures queue_host_call into ctx->host_graph (on a private stream).  On
// failure the graph stays empty and the caller queues the call directly.
void capture_host_call(srwcr_ctx* ctx, int level, int64_t np, const float* c_host, float* g_host) {
  drop_host_graph(ctx);
  if (!ctx->capture_stream &&
      cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->capture_stream = nullptr;
    return;
  }
  cudaStream_t user = ctx->stream;
  const long long launches = ctx->launches;
  ctx->stream = ctx->capture_stream;
  cudaGraph_t graph = nullptr;
  srwcr_status st = SRWCR_ECUDA;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    st = queue_host_call(ctx, ctx->lev[level], np, c_host, g_host);
    if (cudaStreamEndCapture(ctx->stream, &graph) != cudaSuccess) st = SRWCR_ECUDA;
  }
  ctx->stream = user;
  ctx->host_graph_launches = ctx->launches - launches;
  ctx->launches = launches;  // nothing ran during the capture
  cudaGraphExec_t exec = nullptr;
  if (st == SRWCR_OK && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    ctx->host_graph = exec;
    ctx->host_graph_level = level;
    ctx->host_graph_c = c_host;
    ctx->host_graph_g = g_host;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

}  // namespace

srwcr_status srwcr_value_and_grad_host(srwcr_ctx* ctx, int level, const float* c_host,
                                       double* D_host, float* g_host) {
  RET_IF(check_level(ctx, level));
  if (!c_host || !g_host) return fail(SRWCR_EINVAL, "null host pointer");
  Level& lv = ctx->lev[level];
  const int64_t np = lv.g.ncoef * ctx->cfg.ndim;
  if (ctx->stage_len < np) {
    drop_host_graph(ctx);
    if (ctx->c_stage) cudaFree(ctx->c_stage);
    if (ctx->g_stage) cudaFree(ctx->g_stage);
    ctx->c_stage = ctx->g_stage = nullptr;
    CK(cudaMalloc((void**)&ctx->c_stage, sizeof(float) * np));
    CK(cudaMalloc((void**)&ctx->g_stage, sizeof(float) * np));
    ctx->stage_len = np;
  }
  // Page-locked host buffers: replay the call from a CUDA graph (captured on
  // first use for this level and these buffers); otherwise queue it.
  const size_t bytes = sizeof(float) * (size_t)np;
  const bool graph_ok = !ctx->profiling && host_page_locked(c_host, bytes) &&
                        host_page_locked(g_host, bytes);
  if (graph_ok && !(ctx->host_graph && ctx->host_graph_level == level &&
                    ctx->host_graph_c == c_host && ctx->host_graph_g == g_host))
    capture_host_call(ctx, level, np, c_host, g_host);
  ctx->flag_host[0] = 0;   // set by the check if c holds a non-finite value
  if (graph_ok && ctx->host_graph) {
    CK(cudaGraphLaunch(ctx->host_graph, ctx->stream));
    ctx->launches += ctx->host_graph_launches;
  } else {
    RET_IF(queue_host_call(ctx, lv, np, c_host, g_host));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->flag_host[0]) return fail(SRWCR_ENUMERIC, "non-finite FFD coefficients");
  if (!std::isfinite(ctx->D_host[0])) return fail(SRWCR_ENUMERIC, "non-finite SRWCR value");
  if (D_host) *D_host = ctx->D_host[0];
  lv.tables = true;
  return SRWCR_OK;
}

srwcr_status srwcr_forward(srwcr_ctx* ctx, int level, const float* c_dev, double* D_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !D_dev) return fail(SRWCR_EINVAL, "null device pointer");
  Level& lv = ctx->lev[level];
  RET_IF(run_value(ctx, lv, c_dev, false));
  CK(cudaMemcpyAsync(D_dev, lv.D, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return SRWCR_OK;
}

srwcr_status srwcr_backward(srwcr_ctx* ctx, int level, const float* c_dev, const float* gD_dev,
                            float* g_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !g_dev) return fail(SRWCR_EINVAL, "null device pointer");
  Level& lv = ctx->lev[level];
  if (!lv.tables) return fail(SRWCR_EINVAL, "srwcr_backward before srwcr_forward at level %d", level);
  return run_grad(ctx, lv, c_dev, gD_dev, g_dev, false);  // warp recomputed
}

srwcr_status srwcr_region_stats(srwcr_ctx* ctx, int level, double* out, int64_t* n_degenerate) {
  RET_IF(check_level(ctx, level));
  Level& lv = ctx->lev[level];
  if (!lv.tables) return fail(SRWCR_EINVAL, "no evaluation at level %d yet", level);
  if (out) CK(cudaMemcpyAsync(out, lv.stats, sizeof(double) * 4 * lv.g.R, cudaMemcpyDeviceToHost, ctx->stream));
  int nd = 0;
  CK(cudaMemcpyAsync(ctx->flag_host, lv.ndeg, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  nd = ctx->flag_host[0];
  ctx->flag_host[0] = 0;
  if (n_degenerate) *n_degenerate = nd;
  return SRWCR_OK;
}

srwcr_status srwcr_debug_bins(srwcr_ctx* ctx, int level, int32_t* out_dev) {
  RET_IF(check_level(ctx, level));
  if (!out_dev) return fail(SRWCR_EINVAL, "out_dev is NULL");
  Level& lv = ctx->lev[level];
  if (ctx->cfg.ndim == 3) {
    if (is_bf16(ctx)) k_debug_bins<3, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>(lv.g, (const __nv_bfloat16*)lv.A, out_dev);
    else k_debug_bins<3, float><<<1024, 256, 0, ctx->stream>>>(lv.g, (const float*)lv.A, out_dev);
  } else {
    if (is_bf16(ctx)) k_debug_bins<2, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>(lv.g, (const __nv_bfloat16*)lv.A, out_dev);
    else k_debug_bins<2, float><<<1024, 256, 0, ctx->stream>>>(lv.g, (const float*)lv.A, out_dev);
  }
  CKL();
  CK(cudaStreamSynchronize(ctx->stream));
  return SRWCR_OK;
}

}  // extern "C"

namespace {

srwcr_status debug_warp(srwcr_ctx* ctx, int level, const float* c_dev, float* out, float4* out4) {
  Level& lv = ctx->lev[level];
  if (ctx->cfg.ndim == 3) {
    if (is_bf16(ctx)) k_debug_warp<3, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>(lv.g, (const __nv_bfloat16*)lv.M, c_dev, out, out4);
    else k_debug_warp<3, float><<<1024, 256, 0, ctx->stream>>>(lv.g, (const float*)lv.M, c_dev, out, out4);
  } else {
    if (is_bf16(ctx)) k_debug_warp<2, __nv_bfloat16><<<1024, 256, 0, ctx->stream>>>(lv.g, (const __nv_bfloat16*)lv.M, c_dev, out, out4);
    else k_debug_warp<2, float><<<1024, 256, 0, ctx->stream>>>(lv.g, (const float*)lv.M, c_dev, out, out4);
  }
  CKL();
  CK(cudaStreamSynchronize(ctx->stream));
  return SRWCR_OK;
}

}  // namespace

extern "C" {

srwcr_status srwcr_debug_warp(srwcr_ctx* ctx, int level, const float* c_dev, float* out_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !out_dev) return fail(SRWCR_EINVAL, "null device pointer");
  return debug_warp(ctx, level, c_dev, out_dev, nullptr);
}

srwcr_status srwcr_debug_warp_grad(srwcr_ctx* ctx, int level, const float* c_dev, float* out_dev) {
  RET_IF(check_level(ctx, level));
  if (!c_dev || !out_dev) return fail(SRWCR_EINVAL, "null device pointer");
  if (reinterpret_cast<uintptr_t>(out_dev) % 16) return fail(SRWCR_EINVAL, "out_dev must be 16-byte aligned");
  return debug_warp(ctx, level, c_dev, nullptr, reinterpret_cast<float4*>(out_dev));
}

srwcr_status srwcr_level_images(srwcr_ctx* ctx, int level, float* fixed_dev, float* moving_dev) {
  RET_IF(check_level(ctx, level));
  Level& lv = ctx->lev[level];
  float* out[2] = {fixed_dev, moving_dev};
  const void* in[2] = {lv.A, lv.M};
  for (int i = 0; i < 2; ++i) {
    if (!out[i]) continue;
    if (is_bf16(ctx))
      k_to_float<__nv_bfloat16><<<1024, 256, 0, ctx->stream>>>((const __nv_bfloat16*)in[i], lv.g.nvox, out[i]);
    else
      k_to_float<float><<<1024, 256, 0, ctx->stream>>>((const float*)in[i], lv.g.nvox, out[i]);
    CKL();
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SRWCR_OK;
}

srwcr_status srwcr_debug_fixed_point(const float* v_dev, int64_t n, const uint32_t* hi_dev,
                                     const uint32_t* lo_dev, int64_t m, uint64_t* fixed_dev,
                                     float* float_dev, int reference) {
  if (n < 0 || m < 0) return fail(SRWCR_EINVAL, "negative count");
  if (n > 0 && (!v_dev || !fixed_dev)) return fail(SRWCR_EINVAL, "null device pointer");
  if (m > 0 && (!hi_dev || !lo_dev || !float_dev)) return fail(SRWCR_EINVAL, "null device pointer");
  if (n == 0 && m == 0) return SRWCR_OK;
  k_debug_fixed<<<256, 256>>>(v_dev, n, hi_dev, lo_dev, m,
                              reinterpret_cast<unsigned long long*>(fixed_dev), float_dev, reference);
  CKL();
  CK(cudaDeviceSynchronize());
  return SRWCR_OK;
}

srwcr_status srwcr_tile_order(const unsigned char* rowdist_host, const int* dims, const int* tile,
                              int* order_out, int* cost_out) {
  if (!rowdist_host || !dims || !tile || !order_out) return fail(SRWCR_EINVAL, "null host pointer");
  for (int d = 0; d < 3; ++d)
    if (dims[d] < 1 || dims[d] > 65535 || tile[d] < 1) return fail(SRWCR_EINVAL, "dims or tile out of range");
  if (tile[0] != 32) return fail(SRWCR_EINVAL, "tile[0] must be 32");
  if ((long long)((dims[0] + 31) / 32) * dims[1] * dims[2] > INT32_MAX)
    return fail(SRWCR_EINVAL, "more than 2^31 - 1 row segments");
  std::vector<int> order, cost;
  tile_order_host(rowdist_host, dims, tile, &order, &cost);
  std::copy(order.begin(), order.end(), order_out);
  if (cost_out) std::copy(cost.begin(), cost.end(), cost_out);
  return SRWCR_OK;
}

srwcr_status srwcr_set_profiling(srwcr_ctx* ctx, int enable) {
  if (!ctx) return fail(SRWCR_EINVAL, "null context");
  ctx->profiling = enable != 0;
  return SRWCR_OK;
}

srwcr_status srwcr_profile_read(srwcr_ctx* ctx, double* ms, int64_t* counts, int64_t* launches,
                                int reset) {
  if (!ctx) return fail(SRWCR_EINVAL, "null context");
  CK(cudaStreamSynchronize(ctx->stream));
  double acc[kProfKinds] = {0, 0, 0};
  int64_t cnt[kProfKinds] = {0, 0, 0};
  for (auto& p : ctx->prof) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.second.first, p.second.second));
    acc[p.first] += t;
    cnt[p.first] += 1;
  }
  for (int k = 0; k < kProfKinds; ++k) {
    if (ms) ms[k] = acc[k];
    if (counts) counts[k] = cnt[k];
  }
  if (launches) *launches = ctx->launches;
  if (reset) {
    for (auto& p : ctx->prof) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    ctx->prof.clear();
    ctx->launches = 0;
  }
  return SRWCR_OK;
}

void srwcr_lbfgs_default_opts(srwcr_lbfgs_opts* o) {
  if (!o) return;
  o->m = 5;
  o->max_iter[0] = 120; o->max_iter[1] = 200; o->max_iter[2] = 200; o->max_iter[3] = 200;
  o->stable_window = 20;
  o->stable_rtol = 1e-5;
  o->max_ls = 20;
  o->c1 = 1e-4;
  o->c2 = 0.9;
  o->penalty_weight = 0.0;
  o->start_jitter = 0.0;
  o->seed = 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free value entry point (srwcr_value_noalloc).
//
// For callers that cannot allocate device memory: code running inside a
// CUDA-graph capture or a stream-ordered allocator's callback, plugins of a
// host application that owns every cudaMalloc, or real-time loops that must
// not touch the allocator.  All scratch (fixed-point accumulators, region
// statistics and tables) lives in one file-scope device array of
// kNoAllocScratchBytes, which every device that loads this library keeps
// until the process exits.  Host code only sees that array's name as a
// host-side stand-in, never as a device address, so the device address is
// obtained once per device with cudaGetSymbolAddress and cached.  The cache
// assumes that each device keeps one primary context for the life of the
// process: after cudaDeviceReset (a new context, the array at a new address)
// the cached address is stale, so a process that resets a device must not
// call this entry point on it again.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" srwcr_status srwcr_value_noalloc(const srwcr_config* cfg, const float* fixed_dev,
                                            const float* moving_dev, const float* c_dev,
                                            double* D_dev, void* stream) {
  if (!cfg || !fixed_dev || !moving_dev || !c_dev || !D_dev)
    return fail(SRWCR_EINVAL, "null argument");
  if (cfg->role != SRWCR_ROLE_M_AS_B)
    return fail(SRWCR_EINVAL, "the allocation-free value takes the moving image as B only");
  if (cfg->ndim != 2 && cfg->ndim != 3) return fail(SRWCR_EINVAL, "ndim must be 2 or 3");
  if (cfg->n_intensity_bins < 2 || cfg->n_intensity_bins > 256)
    return fail(SRWCR_EINVAL, "n_intensity_bins must be in [2, 256]");
  for (int d = 0; d < cfg->ndim; ++d) {
    if (cfg->dims[d] < 2 || cfg->dims[d] > 65535) return fail(SRWCR_EINVAL, "dims[%d] out of range", d);
    if (cfg->ffd_spacing[d] < 1 || cfg->ffd_spacing[d] > cfg->dims[d])
      return fail(SRWCR_EINVAL, "ffd_spacing[%d] out of range", d);
    if (cfg->sbin_intervals[d] < 0) return fail(SRWCR_EINVAL, "negative sbin_intervals");
  }
  if (cfg->tile[0] < 0 || cfg->tile[1] < 0 || cfg->tile[2] < 0)
    return fail(SRWCR_EINVAL, "negative tile size");
  if (cfg->bins_per_pass < 0) return fail(SRWCR_EINVAL, "negative bins_per_pass");
  cudaStream_t st = (cudaStream_t)stream;

  // Device address of the scratch array, looked up once per device.
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(SRWCR_EINVAL, "device %d beyond the %d devices this entry point serves", dev,
                kNoAllocMaxDevices);
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(SRWCR_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
      g_noalloc_ptr[dev] = p;
    }
    scratch = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }

  Geo g;
  const int dims[3] = {cfg->dims[0], cfg->dims[1], cfg->ndim == 3 ? cfg->dims[2] : 1};
  RET_IF(make_geo(*cfg, dims, g));
  // Scratch layout (28 bytes per spatial bin x intensity bin, 48 per spatial
  // bin): S holds first the fixed-image statistics (R*nb u64), converted to P
  // in FP64, and then, cleared again, the two moving-image moments.
  const size_t R = (size_t)g.R, nb = (size_t)g.nbins;
  const size_t offS = 0;
  const size_t offP = align256(offS + sizeof(unsigned long long) * R * nb * 2);
  const size_t offX = align256(offP + sizeof(double) * R * nb);
  const size_t offU = align256(offX + sizeof(float) * R * nb);
  const size_t offV = align256(offU + sizeof(float) * R);
  const size_t offDr = align256(offV + sizeof(float) * R);
  const size_t offSt = align256(offDr + sizeof(double) * R);
  const size_t offNd = align256(offSt + sizeof(double) * R * 4);
  const size_t need = offNd + sizeof(int);
  if (need > kNoAllocScratchBytes)
    return fail(SRWCR_EINVAL,
                "problem needs %zu bytes of scratch (%zu spatial bins x %zu intensity bins); "
                "the allocation-free entry point holds %zu bytes",
                need, R, nb, kNoAllocScratchBytes);
  unsigned long long* S = reinterpret_cast<unsigned long long*>(scratch + offS);
  double* P = reinterpret_cast<double*>(scratch + offP);
  float* X = reinterpret_cast<float*>(scratch + offX);
  float* U = reinterpret_cast<float*>(scratch + offU);
  float* V = reinterpret_cast<float*>(scratch + offV);
  double* Dr = reinterpret_cast<double*>(scratch + offDr);
  double* stats = reinterpret_cast<double*>(scratch + offSt);
  int* ndeg = reinterpret_cast<int*>(scratch + offNd);

  RET_IF(set_smem_limits<float>());
  double sP, s1, s2;
  fixed_scales(g, cfg->ndim, &sP, &s1, &s2);
  const int nblk = g.ntile[0] * g.ntile[1] * g.ntile[2];
  // Everything the kernels accumulate into starts at zero on every call; the
  // steps are ordered on `st`, so S can serve both accumulations in turn.
  CK(cudaMemsetAsync(S, 0, sizeof(unsigned long long) * R * nb, st));
  if (cfg->ndim == 3)
    k_accumulate<3, float, true><<<nblk, kBlock, acc_smem(g, 1), st>>>(
        g, fixed_dev, moving_dev, nullptr, S, (float)sP, 0.f);
  else
    k_accumulate<2, float, true><<<nblk, kBlock, acc_smem(g, 1), st>>>(
        g, fixed_dev, moving_dev, nullptr, S, (float)sP, 0.f);
  CKL();
  k_fixed_to_double<<<256, 256, 0, st>>>(S, 1.0 / sP, P, (long long)(R * nb));
  CKL();
  CK(cudaMemsetAsync(S, 0, sizeof(unsigned long long) * R * nb * 2, st));
  if (cfg->ndim == 3)
    k_accumulate<3, float, false><<<nblk, kBlock, acc_smem(g, 2), st>>>(
        g, fixed_dev, moving_dev, c_dev, S, (float)s1, (float)s2);
  else
    k_accumulate<2, float, false><<<nblk, kBlock, acc_smem(g, 2), st>>>(
        g, fixed_dev, moving_dev, c_dev, S, (float)s1, (float)s2);
  CKL();
  // Z = N: the spatial weights and Parzen weights each sum to one per voxel.
  const double invZ = 1.0 / (double)g.nvox;
  const int fblk = (int)((R * 32 + kBlock - 1) / kBlock);
  k_finalize<<<fblk, kBlock, 0, st>>>(g, P, S, 1.0 / s1, 1.0 / s2, invZ, U, V, X, Dr, stats);
  CKL();
  k_reduce_D<<<1, 1024, 0, st>>>(Dr, stats, g.R, D_dev, ndeg);
  CKL();
  return SRWCR_OK;
}

// ---------------------------------------------------------------------------
// Tile autotuner.  Times value+gradient for each 32-wide tile that fits the
// row kernels and keeps the fastest; the choice is cached per problem
// signature in memory and, when SRWCR_AUTOTUNE_CACHE names a file, in that
// file (one "signature tile_x tile_y tile_z" line per problem).
// ---------------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;
std::vector<std::pair<std::string, std::array<int, 3>>> g_tune_cache;

std::string tune_key(const srwcr_ctx* ctx, const Geo& g) {
  char buf[256];
  snprintf(buf, sizeof buf, "d%d_n%dx%dx%d_f%dx%dx%d_s%d/%d,%d/%d,%d/%d_b%d_t%d_p%d_r%d_w%d", ctx->cfg.ndim,
           g.n[0], g.n[1], g.n[2], g.fsp[0], g.fsp[1], g.fsp[2], g.sbn[0], g.sbd[0], g.sbn[1],
           g.sbd[1], g.sbn[2], g.sbd[2], g.nbins, ctx->cfg.storage, ctx->cfg.bins_per_pass,
           ctx->cfg.role, ctx->cfg.spatial);
  return buf;
}

bool tune_lookup(const std::string& key, std::array<int, 3>* t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tune_cache)
    if (e.first == key) { *t = e.second; return true; }
  const char* path = getenv("SRWCR_AUTOTUNE_CACHE");
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char k[256];
  int a, b, c;
  bool found = false;
  while (fscanf(f, "%255s %d %d %d", k, &a, &b, &c) == 4)
    if (key == k) { *t = {a, b, c}; found = true; }
  fclose(f);
  if (found) g_tune_cache.push_back({key, *t});
  return found;
}

void tune_store(const std::string& key, const std::array<int, 3>& t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.push_back({key, t});
  const char* path = getenv("SRWCR_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", key.c_str(), t[0], t[1], t[2]);
  fclose(f);
}

void release_rows(Level& lv) {
  if (lv.perm) cudaFree(lv.perm);
  if (lv.binmask) cudaFree(lv.binmask);
  if (lv.order) cudaFree(lv.order);
  lv.perm = nullptr;
  lv.binmask = nullptr;
  lv.order = nullptr;
  lv.order_len = 0;
  lv.rows = false;
  lv.g = lv.gv;
}

}  // namespace

extern "C" srwcr_status srwcr_autotune(srwcr_ctx* ctx, int level, const float* c_dev, int reps,
                                       int* tile_out) {
  RET_IF(check_level(ctx, level));
  if (!c_dev) return fail(SRWCR_EINVAL, "c_dev is NULL");
  if (reps < 1) reps = 3;
  Level& lv = ctx->lev[level];
  drop_host_graph(ctx);  // the level's kernels may change
  if (!rows_allowed(ctx->cfg)) {
    // Only the row-parallel tiles are tuned; this level runs the general kernels.
    for (int d = 0; d < 3 && tile_out; ++d) tile_out[d] = lv.g.tile[d];
    return SRWCR_OK;
  }
  const std::string key = tune_key(ctx, lv.gv);
  std::array<int, 3> best{0, 0, 0};
  if (tune_lookup(key, &best)) {
    release_rows(lv);
    RET_IF(select_rows_path(ctx, lv, best.data()));
    if (!lv.rows) RET_IF(select_rows_path(ctx, lv));
  } else {
    static const int cand3[][3] = {{32, 32, 8}, {32, 32, 4}, {32, 16, 8}, {32, 16, 4},
                                   {32, 8, 8},  {32, 8, 4},  {32, 32, 2}, {32, 16, 2},
                                   {32, 64, 4}, {32, 64, 2}, {32, 128, 2}, {32, 64, 1},
                                   {32, 128, 1}, {32, 256, 1}};
    static const int cand2[][3] = {{32, 64, 1}, {32, 32, 1}, {32, 16, 1}, {32, 8, 1},
                                   {32, 128, 1}, {32, 256, 1}};
    const int nc = ctx->cfg.ndim == 3 ? (int)(sizeof cand3 / sizeof cand3[0])
                                      : (int)(sizeof cand2 / sizeof cand2[0]);
    const int (*cand)[3] = ctx->cfg.ndim == 3 ? cand3 : cand2;
    float* g = nullptr;
    double* D = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t np = (size_t)lv.gv.ncoef * ctx->cfg.ndim;
    CK(cudaMalloc((void**)&g, sizeof(float) * np));
    cudaError_t ce = cudaMalloc((void**)&D, sizeof(double));
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    float best_ms = INFINITY;
    srwcr_status st = ce == cudaSuccess ? SRWCR_OK : fail(SRWCR_ECUDA, "autotune set-up failed");
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    for (int i = 0; i < nc && st == SRWCR_OK; ++i) {
      release_rows(lv);
      st = select_rows_path(ctx, lv, cand[i]);
      if (st != SRWCR_OK || !lv.rows) continue;
      for (int w = 0; w < 2 && st == SRWCR_OK; ++w) {
        st = run_value_and_grad(ctx, lv, c_dev, g);
      }
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < reps && st == SRWCR_OK; ++r) {
        st = run_value_and_grad(ctx, lv, c_dev, g);
      }
      cudaEventRecord(e1, ctx->stream);
      if (st != SRWCR_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(SRWCR_ECUDA, "autotune timing failed"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = {cand[i][0], cand[i][1], cand[i][2]};
      }
    }
    ctx->profiling = prof;
    cudaFree(g);
    cudaFree(D);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    RET_IF(st);
    release_rows(lv);
    if (best[0]) {
      RET_IF(select_rows_path(ctx, lv, best.data()));
      tune_store(key, best);
    } else {
      RET_IF(select_rows_path(ctx, lv));
    }
  }
  lv.tables = false;
  if (tile_out) {
    tile_out[0] = lv.g.tile[0];
    tile_out[1] = lv.g.tile[1];
    tile_out[2] = lv.g.tile[2];
  }
  return SRWCR_OK;
}

#include "lbfgs.cuh"
#include "rigid.cuh"
#include "bending.cuh"
#include "batch.cuh"
