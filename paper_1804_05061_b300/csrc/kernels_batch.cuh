// Batched form of the per-evaluation kernels: many registration pairs of
// uneven sizes in one launch per phase.  Each pair keeps its own buffers; a
// table of descriptors gives every CTA (or finalisation warp) its pair by a
// binary search over the prefix sums of the work items, so one launch
// covers every (pair, tile) item.  A per-pair active flag,
// indexed by the caller's pair index (the table itself is in launch order),
// lets an L-BFGS driver drop converged pairs without rebuilding the table.
#pragma once

#include "kernels.cuh"
#include "kernels_rows.cuh"

namespace srwcr {

struct BatchPair {
  Geo g;                         // row-path geometry of this pair
  AccArgs acc;
  AdjArgs adj;
  int id;                        // caller's index of the pair (active flags, D)
  int group;                     // launch group (x-bins per row, 4, 8 or 12)
  long long region_begin;        // first finalisation warp of this pair
  RegionStatic rs;               // static per-region data of the fixed image
  double inv_s1, inv_s2, invZ;
  float *U, *V, *X;              // gradient tables written by the finalisation
  float* uvxz;                   // their per-plane z-contraction (k_zcontract)
  const int* ubins;              // fixed-image bins present in the image
  int nu;
  double* Dr;                    // [R] shares of D
  double* stats;                 // [R][4]
  double* D;                     // this pair's value
  int* ndeg;
  long long acc_len;             // u64 words of acc to clear
  long long grad_len;            // floats of grad to clear
};

// Largest i with key(i) <= idx over a non-decreasing key.
template <typename KeyFn>
__device__ __forceinline__ int batch_find(int lo, int hi, long long idx, KeyFn key) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(mid) <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool batch_active(const int* active, int p) {
  return active == nullptr || active[p] != 0;
}

// Clears each active pair's accumulators and gradient; blockIdx.y = table slot.
__global__ void __launch_bounds__(256)
k_zero_batch(const BatchPair* __restrict__ pairs, const int* __restrict__ active) {
  const BatchPair& bp = pairs[blockIdx.y];
  if (!batch_active(active, bp.id)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long i = t0; i < bp.acc_len; i += stride) bp.acc.acc[i] = 0ull;
  for (long long i = t0; i < bp.grad_len; i += stride) bp.adj.grad[i] = 0.f;
}

// Row kernels take their pair table as one kernel parameter (constant
// bank), as the single-problem kernels take their geometry, so the body's
// geometry reads stay constant-bank operands.  A launch covers at most
// kBatchChunk pairs; larger batches take several launches per phase.
constexpr int kBatchChunk = 112;

struct AccItem {
  Geo g;
  AccArgs a;
  int id;            // caller's pair index
  int tile_begin;    // first CTA of this pair in the launch
};

struct AdjItem {
  Geo g;
  AdjArgs a;
  int id;
  int tile_begin;
};

struct AccTable {
  int n;
  AccItem it[kBatchChunk];
};

struct AdjTable {
  int n;
  AdjItem it[kBatchChunk];
};

// Both tables travel as one kernel parameter each (at most 32764 bytes).
static_assert(sizeof(AccTable) <= 32764, "AccTable exceeds the kernel parameter limit");
static_assert(sizeof(AdjTable) <= 32764, "AdjTable exceeds the kernel parameter limit");

template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(kAccWarps * 32, 2)
k_accumulate_rows_batch(const __grid_constant__ AccTable tab, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned long long smem_acc[];
  const int p = batch_find(0, tab.n - 1, blockIdx.x,
                           [&](int i) { return (long long)tab.it[i].tile_begin; });
  const AccItem& it = tab.it[p];
  const int tile = blockIdx.x - it.tile_begin;
  if (!batch_active(active, it.id) || tile >= it.g.ntile[0] * it.g.ntile[1] * it.g.ntile[2])
    return;  // CTA-uniform
  acc_rows_body<DIM, T, NXB>(it.g, it.a, tile, smem_acc);
}

template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(kAdjWarps * 32, 4)
k_adjoint_rows_batch(const __grid_constant__ AdjTable tab, const int* __restrict__ active) {
  extern __shared__ __align__(16) float smem_adj[];
  const int p = batch_find(0, tab.n - 1, blockIdx.x,
                           [&](int i) { return (long long)tab.it[i].tile_begin; });
  const AdjItem& it = tab.it[p];
  const int tile = blockIdx.x - it.tile_begin;
  if (!batch_active(active, it.id) || tile >= it.g.ntile[0] * it.g.ntile[1] * it.g.ntile[2])
    return;  // CTA-uniform
  adj_rows_body<DIM, T, NXB>(it.g, it.a, tile, smem_adj);
}

// G lanes per (pair, spatial bin) over all pairs' regions.
template <int G>
__global__ void __launch_bounds__(256)
k_finalize_batch(const BatchPair* __restrict__ pairs, int n, long long total,
                 const int* __restrict__ active) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  if ((w - (threadIdx.x & 31) / G) >= total) return;  // the warp's first region: warp-uniform
  bool live = w < total;
  const int p = live ? batch_find(0, n - 1, w, [&](int i) { return pairs[i].region_begin; }) : 0;
  const BatchPair& bp = pairs[p];
  live = live && batch_active(active, bp.id);
  finalize_region_sparse<G>(w - bp.region_begin, live, threadIdx.x & (G - 1), bp.g.nbins, bp.rs,
                            bp.acc.acc, bp.inv_s1, bp.inv_s2, bp.invZ, bp.U, bp.V, bp.X, bp.Dr,
                            bp.stats);
}

// Per-plane z-contraction of every active pair's tables; blockIdx.y = slot.
template <int DIM>
__global__ void __launch_bounds__(256)
k_zcontract_batch(const BatchPair* __restrict__ pairs, const int* __restrict__ active) {
  const BatchPair& bp = pairs[blockIdx.y];
  if (!batch_active(active, bp.id)) return;
  const long long n = zcontract_items(bp.g, bp.nu);
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    zcontract_item<DIM>(bp.g, i, bp.ubins, bp.nu, bp.U, bp.V, bp.X, bp.uvxz);
}

// One block per table slot: D = sum of the region shares in a fixed order.
__global__ void __launch_bounds__(1024)
k_reduce_D_batch(const BatchPair* __restrict__ pairs, const int* __restrict__ active) {
  const BatchPair& bp = pairs[blockIdx.x];
  if (!batch_active(active, bp.id)) return;
  reduce_D_block(bp.Dr, bp.stats, bp.g.R, bp.D, bp.ndeg);
}

}  // namespace srwcr
