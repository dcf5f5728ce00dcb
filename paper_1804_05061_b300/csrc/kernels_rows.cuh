// Row-parallel SRWCR kernels for sm_103a (the fast path).
//
// A CTA owns a voxel tile 32 x TY x TZ; each warp walks x-rows of 32 voxels.
// Along a row y and z are fixed, so the y/z factors of every tensor-product
// B-spline (FFD nodes, Eq. 17; spatial bins, Eq. 7) are row constants:
//
//   * FFD: per row, the warp contracts the staged coefficient tile over the
//     16 (m, n) y/z nodes once per x-node; each voxel then needs 4 FMAs per
//     component.
//   * Joint statistics (value pass): lanes are ordered by their fixed-image
//     bin a0 with a static per-row permutation (A does not change between
//     evaluations), so voxels sharing a0 are adjacent.  A segmented warp
//     reduction forms, per segment, the FP32 sums over <= 32 voxels of
//     beta_x(i) h(a - A) {m1, m2}; each sum is then spread over the 16
//     row-constant y/z weights and added in 64-bit fixed point to the CTA
//     histogram.  Only short FP32 sums are ever formed, so the
//     E[b^2] - mu^2 cancellation of Eq. (10) keeps full accuracy.
//   * Adjoint: per row the warp contracts the region tables U, V and X over
//     the y/z bins; each voxel forms dD/dB (Eq. 19), and the row's
//     contributions to its control points are combined by a reduce-scatter
//     butterfly before one shared-memory add per (node, component, y/z node).
//
// Rows in which every warped intensity is exactly 0 (m1 = m2 = 0) add nothing
// to the statistics, and rows in which the moving-image gradient vanishes at
// every voxel add nothing to the gradient; both are skipped.
#pragma once

#include "device_math.cuh"

namespace srwcr {

constexpr int kRowWarps = 8;            // warps per CTA (256 threads)
constexpr int kMaxRowNodes = 16;        // FFD x-nodes a row may touch
constexpr int kSentinel = 0x7fffffff;   // key of lanes past the image edge

// Stage the tile's control coefficients (all components) into shared memory.
template <int DIM>
__device__ __forceinline__ void stage_coef_tile(const Geo& g, const float* __restrict__ c,
                                                int f0, int f1, int f2, float* ctile) {
  const int nt = g.hf[0] * g.hf[1] * g.hf[2];
  for (int t = threadIdx.x; t < DIM * nt; t += blockDim.x) {
    const int k = t / nt, r = t % nt;
    const int l0 = r % g.hf[0], l1 = (r / g.hf[0]) % g.hf[1], l2 = r / (g.hf[0] * g.hf[1]);
    const int n0 = f0 + l0, n1 = f1 + l1, n2 = f2 + l2;
    float v = 0.f;
    if (n0 < g.nf[0] && n1 < g.nf[1] && n2 < g.nf[2])
      v = __ldg(c + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0);
    ctile[t] = v;
  }
}

// Per-row FFD contraction over the y/z nodes: cyz[k][l] for the row's x-nodes.
template <int DIM>
__device__ __forceinline__ void row_ffd_contract(const Geo& g, const float* ctile, int ly, int lz,
                                                 const float by[4], const float bz[4], int nxn,
                                                 float* cyz, int lane) {
  const int nt = g.hf[0] * g.hf[1] * g.hf[2];
  for (int t = lane; t < DIM * nxn; t += 32) {
    const int k = t / nxn, l = t % nxn;
    float s = 0.f;
    const int NZ = DIM == 3 ? 4 : 1;
    for (int n = 0; n < NZ; ++n)
      for (int m = 0; m < 4; ++m)
        s += by[m] * bz[n] * ctile[k * nt + ((lz + n) * g.hf[1] + (ly + m)) * g.hf[0] + l];
    cyz[k * kMaxRowNodes + l] = s;
  }
}

// The lane's voxel: FFD displacement from the row table, warped intensity
// and (optionally) its gradient.
template <int DIM, typename T>
__device__ __forceinline__ float row_voxel_warp(const Geo& g, const T* __restrict__ M,
                                                const float* cyz, int x, int y, int z, int fx0,
                                                float bx[4], int* fxrel, float gm[3]) {
  float t;
  const int fx = ffd_cell(g, 0, x, &t);
  bspline4(t, bx);
  const int rel = fx - fx0;
  *fxrel = rel;
  float u[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float* cr = cyz + k * kMaxRowNodes + rel;
    u[k] = bx[0] * cr[0] + bx[1] * cr[1] + bx[2] * cr[2] + bx[3] * cr[3];
  }
  return sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
}

// Select beta[i] for a dynamic i in [0, 4); 0 outside.
__device__ __forceinline__ float pick4(const float b[4], int i) {
  return i == 0 ? b[0] : (i == 1 ? b[1] : (i == 2 ? b[2] : (i == 3 ? b[3] : 0.f)));
}

// ---------------------------------------------------------------------------
// (a) value pass: fused FFD + warp + joint statistics, row-parallel.
//
// Dynamic shared memory: hist [hb2][hb1][hb0][nb][2] u64 | segS [warps][32][NXB*4] f32
//   | segA [warps][32] i32 | cyz [warps][DIM][16] f32 | ctile [DIM][hf] f32
// ---------------------------------------------------------------------------
template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(256)
k_accumulate_rows(const Geo g, const T* __restrict__ A, const T* __restrict__ M,
                  const float* __restrict__ c, const unsigned char* __restrict__ perm,
                  unsigned long long* __restrict__ acc, float s1, float s2) {
  extern __shared__ unsigned long long smem_u64[];
  constexpr int NV = NXB * 4;  // (x-bin, {h0 m1, h0 m2, h1 m1, h1 m2})
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int hsz = g.hb[0] * g.hb[1] * g.hb[2] * nb * 2;
  unsigned long long* hist = smem_u64;
  float* segS = reinterpret_cast<float*>(hist + hsz);
  int* segA = reinterpret_cast<int*>(segS + kRowWarps * 32 * NV);
  float* cyz_all = reinterpret_cast<float*>(segA + kRowWarps * 32);
  float* ctile = cyz_all + kRowWarps * DIM * kMaxRowNodes;
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;
  float* mysegS = segS + warp * 32 * NV;
  int* mysegA = segA + warp * 32;

  int o[3];
  {
    const int b = blockIdx.x;
    o[0] = (b % g.ntile[0]) * g.tile[0];
    o[1] = ((b / g.ntile[0]) % g.ntile[1]) * g.tile[1];
    o[2] = (b / (g.ntile[0] * g.ntile[1])) * g.tile[2];
  }
  float tdum;
  const int cb0 = sb_cell(g, 0, o[0], &tdum);
  const int cb1 = sb_cell(g, 1, o[1], &tdum);
  const int cb2 = DIM == 3 ? sb_cell(g, 2, o[2], &tdum) : 0;
  const int f0 = o[0] / g.fsp[0], f1 = o[1] / g.fsp[1], f2 = DIM == 3 ? o[2] / g.fsp[2] : 0;
  for (int i = threadIdx.x; i < hsz; i += blockDim.x) hist[i] = 0ull;
  stage_coef_tile<DIM>(g, c, f0, f1, f2, ctile);
  __syncthreads();

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - f0 + 4;          // FFD x-nodes of this row
  const int nrows = g.tile[1] * g.tile[2];
  for (int row = warp; row < nrows; row += kRowWarps) {
    const int y = o[1] + row % g.tile[1];
    const int z = o[2] + row / g.tile[1];
    if (y >= g.n[1] || z >= g.n[2]) continue;  // warp-uniform
    // Row constants: FFD and spatial y/z weights.
    float by[4], bz[4], sy[4], sz[4], t;
    const int fy = ffd_cell(g, 1, y, &t); bspline4(t, by);
    const int scy = sb_cell(g, 1, y, &t); bspline4(t, sy);
    int fz = 0, scz = 0;
    if (DIM == 3) {
      fz = ffd_cell(g, 2, z, &t); bspline4(t, bz);
      scz = sb_cell(g, 2, z, &t); bspline4(t, sz);
    } else {
      bz[0] = sz[0] = 1.f; bz[1] = bz[2] = bz[3] = sz[1] = sz[2] = sz[3] = 0.f;
    }
    row_ffd_contract<DIM>(g, ctile, fy - f1, fz - f2, by, bz, nxn, cyz, lane);
    __syncwarp();

    const long long rowid = ((long long)z * g.n[1] + y) * nxb + (o[0] >> 5);
    const int x = o[0] + perm[rowid * 32 + lane];
    const bool act = x < g.n[0];
    float m1 = 0.f, m2 = 0.f, h0 = 0.f, h1 = 0.f;
    int key = kSentinel;
    float bsx[4] = {0.f, 0.f, 0.f, 0.f};
    int srel = 0;
    if (act) {
      const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
      float fa;
      const int a0 = bin_split(fminf(fmaxf(ldval(A + idx), 0.f), L), nb, &fa);
      key = a0;
      h1 = parzen_upper(fa);
      h0 = 1.f - h1;
      float bx[4], gm[3];
      int fxrel;
      float B = row_voxel_warp<DIM, T>(g, M, cyz, x, y, z, f0, bx, &fxrel, gm);
      B = fminf(fmaxf(B, 0.f), L);
      float fb;
      const int kb = bin_split(B, nb, &fb);
      const float w1 = parzen_upper(fb), kf = (float)kb;
      m1 = kf + w1;
      m2 = kf * kf + (2.f * kf + 1.f) * w1;
      const int scx = sb_cell(g, 0, x, &t);
      bspline4(t, bsx);
      srel = scx - cb0;
    }
    const bool live = act && (m1 != 0.f || m2 != 0.f);
    __syncwarp();
    if (!__any_sync(0xffffffffu, live)) continue;  // B == 0 everywhere: nothing to add

    // Per-lane contributions over the row's NXB spatial x-bins.
    float v[NV];
#pragma unroll
    for (int b = 0; b < NXB; ++b) {
      const float w = live ? pick4(bsx, b - srel) : 0.f;
      v[4 * b + 0] = w * h0 * m1;
      v[4 * b + 1] = w * h0 * m2;
      v[4 * b + 2] = w * h1 * m1;
      v[4 * b + 3] = w * h1 * m2;
    }
    // Segments of equal a0 (lanes are sorted by a0).
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || key != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned above = lane == 31 ? 0u : (heads & (0xffffffffu << (lane + 1)));
    const int seg_end = above ? __ffs(above) - 1 : 32;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const bool ok = lane + off < seg_end;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float ov = __shfl_down_sync(0xffffffffu, v[q], off);
        if (ok) v[q] += ov;
      }
    }
    const int nseg = __popc(heads);
    if (head) {
      const int sidx = __popc(heads & ((1u << lane) - 1u));
      mysegA[sidx] = key;
#pragma unroll
      for (int q = 0; q < NV; ++q) mysegS[sidx * NV + q] = v[q];
    }
    __syncwarp();
    // Fold each (segment, x-bin, moment) sum over the 16 y/z bins.
    const int lb1 = scy - cb1, lb2 = scz - cb2;
    const int NJK = DIM == 3 ? 16 : 4;
    for (int it = lane; it < nseg * NV; it += 32) {
      const int s = it / NV, q = it % NV;
      const int a = mysegA[s];
      const float val = mysegS[s * NV + q];
      const int b = q >> 2, slot = (q >> 1) & 1, ch = q & 1;
      if (a == kSentinel || val == 0.f || b >= g.hb[0]) continue;
      const float vs = val * (ch ? s2 : s1);
      const int abin = a + slot;
      for (int jk = 0; jk < NJK; ++jk) {
        const int j = jk & 3, k = jk >> 2;
        const float w = sy[j] * sz[k];
        if (w == 0.f) continue;
        const int hb = ((lb2 + k) * g.hb[1] + (lb1 + j)) * g.hb[0] + b;
        atomicAdd(hist + ((size_t)hb * nb + abin) * 2 + ch, __float2ull_rn(vs * w));
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < hsz; i += blockDim.x) {
    const unsigned long long val = hist[i];
    if (!val) continue;
    const int ch = i & 1;
    const int a = (i >> 1) % nb;
    const int hbin = (i >> 1) / nb;
    const int l0 = hbin % g.hb[0];
    const int l1 = (hbin / g.hb[0]) % g.hb[1];
    const int l2 = hbin / (g.hb[0] * g.hb[1]);
    if (cb0 + l0 >= g.nsb[0] || cb1 + l1 >= g.nsb[1] || cb2 + l2 >= g.nsb[2]) continue;
    const long long r = ((long long)(cb2 + l2) * g.nsb[1] + (cb1 + l1)) * g.nsb[0] + (cb0 + l0);
    atomicAdd(acc + ((size_t)r * nb + a) * 2 + ch, val);
  }
}

// Reduce-scatter over the 32 lanes of a warp: on entry each lane holds 32
// values; on exit lane l holds the sum over all lanes of value l.
__device__ __forceinline__ float warp_reduce_scatter32(float v[32], int lane) {
#pragma unroll
  for (int m = 16, n = 32; m >= 1; m >>= 1, n >>= 1) {
    const bool upper = lane & m;
    const int half = n >> 1;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[half + i];
      const float keep = upper ? v[half + i] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return v[0];
}

// ---------------------------------------------------------------------------
// (c) adjoint, row-parallel.
//
// Dynamic shared memory: gt [DIM][hf2][hf1][hf0] f32 | U, V [hb] f32 | X [hb][nb] f32
//   | rowt [warps][2*NXB] f32 | xy [warps][32][NXB][2] f32 | segA [warps][32] i32
//   | cyz [warps][DIM][16] f32 | ctile [DIM][hf] f32
// ---------------------------------------------------------------------------
template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(256)
k_adjoint_rows(const Geo g, const T* __restrict__ A, const T* __restrict__ M,
               const float* __restrict__ c, const unsigned char* __restrict__ perm,
               const float* __restrict__ U, const float* __restrict__ V,
               const float* __restrict__ X, const float* __restrict__ gscale, float invZ,
               float* __restrict__ grad) {
  extern __shared__ float smem_f32[];
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nodes_tile = g.hf[0] * g.hf[1] * g.hf[2];
  const int nbt = g.hb[0] * g.hb[1] * g.hb[2];
  float* gt = smem_f32;
  float* Ut = gt + DIM * nodes_tile;
  float* Vt = Ut + nbt;
  float* Xt = Vt + nbt;
  float* rowt_all = Xt + (size_t)nbt * nb;
  float* xy_all = rowt_all + kRowWarps * 2 * NXB;
  int* segA_all = reinterpret_cast<int*>(xy_all + kRowWarps * 32 * NXB * 2);
  float* cyz_all = reinterpret_cast<float*>(segA_all + kRowWarps * 32);
  float* ctile = cyz_all + kRowWarps * DIM * kMaxRowNodes;
  float* rowt = rowt_all + warp * 2 * NXB;
  float* xy = xy_all + warp * 32 * NXB * 2;
  int* mysegA = segA_all + warp * 32;
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;

  int o[3];
  {
    const int b = blockIdx.x;
    o[0] = (b % g.ntile[0]) * g.tile[0];
    o[1] = ((b / g.ntile[0]) % g.ntile[1]) * g.tile[1];
    o[2] = (b / (g.ntile[0] * g.ntile[1])) * g.tile[2];
  }
  float tdum;
  const int cb0 = sb_cell(g, 0, o[0], &tdum);
  const int cb1 = sb_cell(g, 1, o[1], &tdum);
  const int cb2 = DIM == 3 ? sb_cell(g, 2, o[2], &tdum) : 0;
  const int f0 = o[0] / g.fsp[0], f1 = o[1] / g.fsp[1], f2 = DIM == 3 ? o[2] / g.fsp[2] : 0;
  for (int i = threadIdx.x; i < DIM * nodes_tile; i += blockDim.x) gt[i] = 0.f;
  // Region tables of the tile's spatial bins.
  for (int i = threadIdx.x; i < nbt; i += blockDim.x) {
    const int l0 = i % g.hb[0], l1 = (i / g.hb[0]) % g.hb[1], l2 = i / (g.hb[0] * g.hb[1]);
    const int r0 = cb0 + l0, r1 = cb1 + l1, r2 = cb2 + l2;
    const bool in = r0 < g.nsb[0] && r1 < g.nsb[1] && r2 < g.nsb[2];
    const long long r = in ? ((long long)r2 * g.nsb[1] + r1) * g.nsb[0] + r0 : 0;
    Ut[i] = in ? __ldg(U + r) : 0.f;
    Vt[i] = in ? __ldg(V + r) : 0.f;
  }
  for (int i = threadIdx.x; i < nbt * nb; i += blockDim.x) {
    const int hbin = i / nb, a = i % nb;
    const int l0 = hbin % g.hb[0], l1 = (hbin / g.hb[0]) % g.hb[1], l2 = hbin / (g.hb[0] * g.hb[1]);
    const int r0 = cb0 + l0, r1 = cb1 + l1, r2 = cb2 + l2;
    const bool in = r0 < g.nsb[0] && r1 < g.nsb[1] && r2 < g.nsb[2];
    Xt[i] = in ? __ldg(X + (((long long)r2 * g.nsb[1] + r1) * g.nsb[0] + r0) * nb + a) : 0.f;
  }
  stage_coef_tile<DIM>(g, c, f0, f1, f2, ctile);
  __syncthreads();
  const float scale = (gscale ? __ldg(gscale) : 1.f) * invZ;

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - f0 + 4;
  const int nrows = g.tile[1] * g.tile[2];
  const int NJK = DIM == 3 ? 16 : 4;
  for (int row = warp; row < nrows; row += kRowWarps) {
    const int y = o[1] + row % g.tile[1];
    const int z = o[2] + row / g.tile[1];
    if (y >= g.n[1] || z >= g.n[2]) continue;
    float by[4], bz[4], sy[4], sz[4], t;
    const int fy = ffd_cell(g, 1, y, &t); bspline4(t, by);
    const int scy = sb_cell(g, 1, y, &t); bspline4(t, sy);
    int fz = 0, scz = 0;
    if (DIM == 3) {
      fz = ffd_cell(g, 2, z, &t); bspline4(t, bz);
      scz = sb_cell(g, 2, z, &t); bspline4(t, sz);
    } else {
      bz[0] = sz[0] = 1.f; bz[1] = bz[2] = bz[3] = sz[1] = sz[2] = sz[3] = 0.f;
    }
    row_ffd_contract<DIM>(g, ctile, fy - f1, fz - f2, by, bz, nxn, cyz, lane);
    __syncwarp();

    const long long rowid = ((long long)z * g.n[1] + y) * nxb + (o[0] >> 5);
    const int x = o[0] + perm[rowid * 32 + lane];
    const bool act = x < g.n[0];
    float gm[3] = {0.f, 0.f, 0.f}, bx[4] = {0.f, 0.f, 0.f, 0.f}, bsx[4] = {0.f, 0.f, 0.f, 0.f};
    float dm1 = 0.f, dm2 = 0.f, h0 = 0.f, h1 = 0.f;
    int key = kSentinel, fxrel = 0, srel = 0;
    if (act) {
      const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
      float fa;
      key = bin_split(fminf(fmaxf(ldval(A + idx), 0.f), L), nb, &fa);
      h1 = parzen_upper(fa);
      h0 = 1.f - h1;
      float B = row_voxel_warp<DIM, T>(g, M, cyz, x, y, z, f0, bx, &fxrel, gm);
      B = fminf(fmaxf(B, 0.f), L);
      float fb;
      const int kb = bin_split(B, nb, &fb);
      dm1 = parzen_upper_deriv(fb);
      dm2 = (2.f * (float)kb + 1.f) * dm1;
      const int scx = sb_cell(g, 0, x, &t);
      bspline4(t, bsx);
      srel = scx - cb0;
    }
    const bool live = act && (gm[0] != 0.f || gm[1] != 0.f || (DIM == 3 && gm[2] != 0.f));
    __syncwarp();
    if (!__any_sync(0xffffffffu, live)) continue;  // grad M == 0 on the whole row

    // Row tables: U, V contracted over the y/z bins for the row's x-bins.
    const int lb1 = scy - cb1, lb2 = scz - cb2;
    for (int tt = lane; tt < 2 * NXB; tt += 32) {
      const int b = tt % NXB;
      const float* tab = tt < NXB ? Ut : Vt;
      float s = 0.f;
      for (int jk = 0; jk < (b < g.hb[0] ? NJK : 0); ++jk) {
        const int j = jk & 3, k = jk >> 2;
        s += sy[j] * sz[k] * tab[((lb2 + k) * g.hb[1] + (lb1 + j)) * g.hb[0] + b];
      }
      rowt[tt] = s;
    }
    // Segments of equal a0; X contracted over y/z for each segment's two bins.
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || key != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int nseg = __popc(heads);
    if (head) mysegA[__popc(heads & ((1u << lane) - 1u))] = key;
    __syncwarp();
    for (int it = lane; it < nseg * NXB * 2; it += 32) {
      const int s = it / (NXB * 2), rem = it % (NXB * 2), b = rem >> 1, slot = rem & 1;
      const int a = mysegA[s];
      float acc_x = 0.f;
      if (a != kSentinel && b < g.hb[0]) {
        const int abin = a + slot;
        for (int jk = 0; jk < NJK; ++jk) {
          const int j = jk & 3, k = jk >> 2;
          acc_x += sy[j] * sz[k] * Xt[(size_t)(((lb2 + k) * g.hb[1] + (lb1 + j)) * g.hb[0] + b) * nb + abin];
        }
      }
      xy[(s * NXB + b) * 2 + slot] = acc_x;
    }
    __syncwarp();
    float G = 0.f;
    if (live) {
      const int sidx = __popc(heads & ((2u << lane) - 1u)) - 1;
      float su = 0.f, sv = 0.f, sxr = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = srel + i;
        su += bsx[i] * rowt[b];
        sv += bsx[i] * rowt[NXB + b];
        sxr += bsx[i] * (h0 * xy[(sidx * NXB + b) * 2] + h1 * xy[(sidx * NXB + b) * 2 + 1]);
      }
      G = scale * (dm2 * su + 2.f * dm1 * (sv - sxr));
    }
    // Contributions to the row's control points (nxn x-nodes, DIM components).
    // Value q = 10 k + p: component k, row x-node p (fxrel + l < nxn <= 10).
    float vals[32];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float gk = (live && k < DIM) ? G * gm[k] : 0.f;
#pragma unroll
      for (int p = 0; p < 10; ++p) vals[k * 10 + p] = gk * pick4(bx, p - fxrel);
    }
    vals[30] = vals[31] = 0.f;
    const float tot = warp_reduce_scatter32(vals, lane);
    // Lane q holds component q/10, x-node q%10: spread over the 16 y/z nodes.
    const int kq = lane / 10, lq = lane % 10;
    if (lane < DIM * 10 && lq < nxn && tot != 0.f) {
      const int lyf = fy - f1, lzf = fz - f2;
      for (int mn = 0; mn < NJK; ++mn) {
        const int m = mn & 3, n = mn >> 2;
        const float w = by[m] * bz[n];
        if (w == 0.f) continue;
        atomicAdd(gt + kq * nodes_tile + ((lzf + n) * g.hf[1] + (lyf + m)) * g.hf[0] + lq, tot * w);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < DIM * nodes_tile; i += blockDim.x) {
    const float val = gt[i];
    if (val == 0.f) continue;
    const int k = i / nodes_tile, nl = i % nodes_tile;
    const int n0 = f0 + nl % g.hf[0], n1 = f1 + (nl / g.hf[0]) % g.hf[1],
              n2 = f2 + nl / (g.hf[0] * g.hf[1]);
    if (n0 >= g.nf[0] || n1 >= g.nf[1] || n2 >= g.nf[2]) continue;
    atomicAdd(grad + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0, val);
  }
}

// Static per-row permutation: lanes of each 32-voxel x-row ordered by the
// fixed-image bin a0 (stable); lanes past the image edge go last.
template <typename T>
__global__ void k_row_perm(const Geo g, const T* __restrict__ A, unsigned char* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int nxb = (g.n[0] + 31) >> 5;
  const long long nrows = (long long)nxb * g.n[1] * g.n[2];
  const float L = (float)(g.nbins - 1);
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < nrows;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int xb = (int)(row % nxb);
    const long long yz = row / nxb;
    const int x = xb * 32 + lane;
    int key = kSentinel;
    if (x < g.n[0]) {
      float fa;
      key = bin_split(fminf(fmaxf(ldval(A + yz * g.n[0] + x), 0.f), L), g.nbins, &fa);
    }
    int rank = 0;
    for (int j = 0; j < 32; ++j) {
      const int kj = __shfl_sync(0xffffffffu, key, j);
      rank += (kj < key) || (kj == key && j < lane);
    }
    perm[row * 32 + rank] = (unsigned char)lane;
  }
}

}  // namespace srwcr
