// Row-parallel kernels with the moving image as the model image A (Sec. II-E,
// Eqs. 20, 21) for sm_103a.
//
// The CTA, row and table structure is that of the M-as-B row kernels
// (kernels_rows.cuh): a CTA owns a 32 x TY x TZ voxel tile, each warp walks
// 32-voxel x-rows, per-axis B-spline tables and the z-contracted FFD
// coefficients are built once per tile.  What differs is that the binned
// image A(x) = M(T(x)) moves: the lanes of a row are not reordered; instead
// the lanes whose warped intensity falls in the same bin a0 are grouped at
// every evaluation (a warp match on a0), and each group's sums
//   sum_x beta_x(i) h_slot(A) {1, m1(F), m2(F)}
// over 4 x-bins, 2 Parzen slots (a0, a0+1) and 3 channels (P, S1, S2) are
// formed by a transpose through shared memory: every lane stores its 24
// products as one row, then lane q sums column q over the group's rows and
// adds the total, weighted by the row's 4 y B-spline weights, to the
// per-z-plane fixed-point histogram H[plane][y bin][bin][channel][x bin]
// (two 24-bit fields per entry, as in the M-as-B value kernel).  The flush
// combines the planes of a z cell with their z weights and adds the three
// channels to the global accumulators [R][nbins][3].  The histogram holds
// every intensity bin (the binned image changes every evaluation), so tiles
// are chosen small enough for it to fit in shared memory.
//
// The adjoint forms Eq. (21) per voxel from the bin-to-bin differences of the
// finalisation's tables, contracted over z per image plane (k_zcontract_dy)
// and over y per row, and scatters G(x) dM/dy(T(x)) to the control points
// with the reduce-scatter of the M-as-B adjoint.  Rows whose moving-image
// gradient vanishes at every voxel add nothing and are not visited.
#pragma once

#include "kernels_rows.cuh"

namespace srwcr {

struct AccArgsA {
  const void* F;                 // normalised fixed image (the estimated image B)
  const void* M;                 // normalised moving image (warped: the model image A)
  const float* c;
  unsigned long long* acc;       // [R][nbins][3] fixed-point P, S1, S2
  float4* bg;                    // per voxel (A, dM/dy) for the adjoint, or NULL
  const unsigned char* rowdist;  // per row: distance to the nearest nonzero M voxel, or NULL
  unsigned char* rowlive;        // per row: nonzero dM/dy somewhere, or NULL
  float s0, s1, s2;              // fixed-point scales of P, S1, S2
};

struct AdjArgsA {
  const void* F;
  const void* M;
  const float* c;
  const float2* dyz;             // bin-to-bin table differences contracted over z per plane
  const float* gscale;           // device scalar or NULL (1)
  const float4* bg;              // (A, dM/dy) stored by the value pass, or NULL: recompute
  const unsigned char* rowlive;  // rows with nonzero dM/dy, or NULL: all
  float invZ;
  float* grad;
};

constexpr int kMasARowStride = 28;   // floats per lane row of the transpose (24 used)

// Words per y/z row of the histogram: 3 * nbins * hb0 columns and at least
// 8 spare words (the fold's lanes without a column add zeros there),
// rounded to 8 mod 32 as in the M-as-B kernel.
__host__ __device__ inline int mas_a_yz_stride(const Geo& g) {
  const int w = 3 * g.nbins * g.hb[0];
  return ((w + 31) / 32) * 32 + 8;
}

__host__ __device__ inline size_t acc_rows_mas_a_smem_bytes(const Geo& g, int dim, int nxb) {
  const size_t npy = (size_t)g.tile[2] * g.hb[1];
  size_t b = 2 * npy * mas_a_yz_stride(g) * sizeof(unsigned);          // histogram words
  b += sizeof(float) * kAccWarps * 32 * kMasARowStride;               // transposes
  b += sizeof(float) * kAccWarps * dim * kMaxRowNodes;                 // cyz
  b += sizeof(float) * xtab_words(nxb);                                // x tables
  b += sizeof(AxisEntry) * (g.tile[1] + g.tile[2]);                    // y, z tables
  b += sizeof(float) * g.tile[2] * dim * g.hf[1] * g.hf[0];            // CZ
  return b;
}

// Parzen moments m1 = sum_b b h(b - v), m2 = sum_b b^2 h(b - v) (Eq. 5).
__device__ __forceinline__ void row_parzen_moments(float v, int nb, float* m1, float* m2) {
  float f;
  const int k = bin_split(v, nb, &f);
  const float w1 = parzen_upper(f), kf = (float)k;
  *m1 = kf + w1;
  *m2 = kf * kf + (2.f * kf + 1.f) * w1;
}

template <int DIM, typename T, int NXB>
__device__ __forceinline__ void acc_rows_mas_a_body(const Geo& g, const AccArgsA& args, int tile,
                                                    unsigned long long* smem_u64) {
  const T* __restrict__ F = static_cast<const T*>(args.F);
  const T* __restrict__ M = static_cast<const T*>(args.M);
  const float* __restrict__ c = args.c;
  unsigned long long* __restrict__ acc = args.acc;
  const unsigned char* __restrict__ rowdist = args.rowdist;
  unsigned char* __restrict__ rowlive = args.rowlive;
  constexpr int XC = 4;                       // x-bins per chunk
  constexpr int NK = DIM == 3 ? 4 : 1;
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S = mas_a_yz_stride(g);
  const int NPY = g.tile[2] * g.hb[1];
  unsigned* hlo = reinterpret_cast<unsigned*>(smem_u64);
  unsigned* hhi = hlo + (size_t)NPY * S;
  float* tr_all = reinterpret_cast<float*>(hhi + (size_t)NPY * S);
  float* cyz_all = tr_all + kAccWarps * 32 * kMasARowStride;
  const XTab xt = xtab_carve(cyz_all + kAccWarps * DIM * kMaxRowNodes, NXB);
  AxisEntry* yt = reinterpret_cast<AxisEntry*>(reinterpret_cast<float*>(xt.frel) + xtab_words(NXB));
  AxisEntry* zt = yt + g.tile[1];
  float* CZ = reinterpret_cast<float*>(zt + g.tile[2]);
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;
  float* tr = tr_all + warp * 32 * kMasARowStride;

  const TileOrigin TO = tile_setup<DIM>(g, tile);
  build_axis_tables<DIM>(g, TO, yt, zt);
  __syncthreads();
  build_cz<DIM>(g, TO, c, zt, CZ);
  build_xtab<NXB>(g, TO, xt, (int)blockDim.x - 32);
  const int hwords4 = (2 * NPY * S) >> 2;
  uint4* h4 = reinterpret_cast<uint4*>(hlo);
  for (int i = threadIdx.x; i < hwords4; i += blockDim.x) h4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(TO.o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - TO.f[0] + 4;
  const int nrows = g.tile[1] * g.tile[2];
  const CyzSlots cslots = cyz_slots<DIM>(nxn, lane);
  // Column q < 24 of the transpose: x-bin q / 6 of the chunk, Parzen slot
  // (q / 3) & 1, channel q % 3 (P, S1, S2).
  const int qb = lane / 6, qslot = (lane / 3) & 1, qch = lane % 3;
  const float qscale = qch == 0 ? args.s0 : (qch == 1 ? args.s1 : args.s2);
  // The fixed image's value of the lane's voxel and the row's distance are
  // loaded one row ahead.
  auto fetch = [&](int yr, int zr, float* ff, int* dd) {
    *ff = 0.f;
    *dd = 0;
    if (zr >= g.tile[2]) return false;
    const int y = TO.o[1] + yr, z = TO.o[2] + zr;
    if (y >= g.n[1] || z >= g.n[2]) return false;
    if (rowdist) *dd = rowdist[((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5)];
    const int xn = TO.o[0] + lane;
    if (xn < g.n[0]) *ff = ldval(F + ((long long)z * g.n[1] + y) * g.n[0] + xn);
    return true;
  };
  float f_next;
  int d_next;
  int yn = 0, zn = 0;
  row_step(warp, g.tile[1], &yn, &zn);
  bool ok_next = fetch(yn, zn, &f_next, &d_next);
  for (int row = warp; row < nrows; row += kAccWarps) {
    const float f_lane = f_next;
    const int rdist = d_next;
    const bool ok = ok_next;
    const int yl = yn, zl = zn;
    row_step(kAccWarps, g.tile[1], &yn, &zn);
    ok_next = fetch(yn, zn, &f_next, &d_next);
    if (!ok) continue;  // warp-uniform
    const int y = TO.o[1] + yl, z = TO.o[2] + zl;
    const long long rowid = ((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5);
    const int x = TO.o[0] + lane;
    const bool act = x < g.n[0];
    const AxisEntry ye = yt[yl];
    const float umax = row_cyz<DIM>(g, CZ, zl, ye, cslots, cyz);
    // A row that provably reads only zeros of M has A = 0 and dM/dy = 0 at
    // every voxel: no warp to compute (the row still adds its fixed-image
    // moments to bin 0).
    bool dead = false;
    if (rowdist) {
      const float U = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(umax)));
      dead = (float)rdist > U + kDeadRowMargin;
    }
    __syncwarp();
    float Av = 0.f;
    bool glive = false;
    if (act && !dead) {
      const float bx[4] = {xt.bf[lane], xt.bf[32 + lane], xt.bf[64 + lane], xt.bf[96 + lane]};
      float gm[3];
      Av = row_warp<DIM, T>(g, M, cyz, xt.frel[lane], bx, x, y, z, gm);
      Av = fminf(fmaxf(Av, 0.f), L);
      if (args.bg) args.bg[((long long)z * g.n[1] + y) * g.n[0] + x] = make_float4(Av, gm[0], gm[1], gm[2]);
      glive = gm[0] != 0.f || gm[1] != 0.f || gm[2] != 0.f;
    }
    if (rowlive) {
      const bool any_g = __any_sync(0xffffffffu, glive);
      if (lane == 0) rowlive[rowid] = any_g ? 1 : 0;
    }
    int key = kSentinel;
    float h1 = 0.f, m1 = 0.f, m2 = 0.f;
    if (act) {
      float fa;
      key = bin_split(Av, nb, &fa);
      h1 = parzen_upper(fa);
      row_parzen_moments(fminf(fmaxf(f_lane, 0.f), L), nb, &m1, &m2);
    }
    const float h0 = act ? 1.f - h1 : 0.f;
    // Groups of lanes with the same bin a0 (inactive lanes excluded).
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const unsigned leaders =
        __ballot_sync(0xffffffffu, key != kSentinel && lane == __ffs(peers) - 1);
    const int prow = (zl * g.hb[1] + ye.srel) * S;
    for (int q0 = 0; q0 < NXB && q0 < g.hb[0]; q0 += XC) {
      // This lane's 24 products, stored as its row of the transpose.
      float v[24];
#pragma unroll
      for (int b = 0; b < XC; ++b) {
        const float w = xt.bsp[(q0 + b) * 32 + lane];
        const float e0 = w * h0, e1 = w * h1;
        v[6 * b + 0] = e0;
        v[6 * b + 1] = e0 * m1;
        v[6 * b + 2] = e0 * m2;
        v[6 * b + 3] = e1;
        v[6 * b + 4] = e1 * m1;
        v[6 * b + 5] = e1 * m2;
      }
      float4* rowp = reinterpret_cast<float4*>(tr + lane * kMasARowStride);
#pragma unroll
      for (int k = 0; k < 6; ++k) rowp[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
      __syncwarp();
      // Each group: lane q sums column q over the group's rows and adds the
      // total (bin a0 + slot, channel, x-bin) to the row's 4 y bins.
      for (unsigned gl = leaders; gl; gl &= gl - 1) {
        const int ld = __ffs(gl) - 1;
        const unsigned members = __shfl_sync(0xffffffffu, peers, ld);
        const int a0 = __shfl_sync(0xffffffffu, key, ld);
        float sum = 0.f;
        for (unsigned mm = members; mm; mm &= mm - 1)
          if (lane < 24) sum += tr[(__ffs(mm) - 1) * kMasARowStride + lane];
        // No branch, as in the M-as-B value kernel: lanes without a column
        // (lane >= 24, or an x-bin past the row's) add zeros to a spare
        // word of their own past the row's columns, zero sums add zeros.
        const int bx_ = q0 + qb;
        const bool inq = lane < 24 && bx_ < g.hb[0];
        const float uv = inq ? sum * qscale : 0.f;
        const int col = prow + (inq ? ((a0 + qslot) * 3 + qch) * g.hb[0] + bx_
                                    : 3 * g.nbins * g.hb[0] + (lane & 7));
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float u = uv * ye.bs[m];
          // Two 24-bit fields of u (< 2^48), as in the M-as-B value kernel.
          const float hf = floorf(u * 0x1p-24f);
          const unsigned lo = __float2uint_rn(fmaf(hf, -0x1p24f, u));
          const unsigned hi = __float2uint_rz(hf);
          const int at = col + m * S;
          atomicAdd(hlo + at, lo);
          atomicAdd(hhi + at, hi);
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // Flush: per (column, first plane of a z cell, y bin): combine the cell's
  // planes with their z weights, then add the NK z bins to the global
  // accumulators.
  const int wcols = 3 * nb * g.hb[0];
  const int tpc = wcols < (int)blockDim.x ? min((int)blockDim.x / wcols, g.hb[1]) : 1;
  for (int t = threadIdx.x; t < wcols * tpc; t += blockDim.x) {
    const int sub = t / wcols, col = t - sub * wcols;
    const int ach = col / g.hb[0], b = col - ach * g.hb[0];
    const int r0 = TO.cb[0] + b;
    if (r0 >= g.nsb[0]) continue;
    const int a = ach / 3, ch = ach - 3 * a;
    for (int zl = 0; zl < g.tile[2]; ++zl) {
      const int cz = zt[zl].srel;
      if (zl > 0 && zt[zl - 1].srel == cz) continue;
      for (int l1 = sub; l1 < g.hb[1]; l1 += tpc) {
        const int r1 = TO.cb[1] + l1;
        if (r1 >= g.nsb[1]) break;
        float u[NK];
#pragma unroll
        for (int m = 0; m < NK; ++m) u[m] = 0.f;
        bool any = false;
        for (int pl = zl; pl < g.tile[2] && zt[pl].srel == cz; ++pl) {
          const int j = (pl * g.hb[1] + l1) * S + col;
          const unsigned lo = hlo[j], hi = hhi[j];
          if (!(lo | hi)) continue;
          any = true;
          const float hv = fields_to_float(hi, lo);
#pragma unroll
          for (int m = 0; m < NK; ++m) u[m] = fmaf(zt[pl].bs[m], hv, u[m]);
        }
        if (!any) continue;
#pragma unroll
        for (int m = 0; m < NK; ++m) {
          const int r2 = TO.cb[2] + cz + m;
          if (u[m] == 0.f || r2 >= g.nsb[2]) continue;
          const long long r = ((long long)r2 * g.nsb[1] + r1) * g.nsb[0] + r0;
          atomicAdd(acc + ((size_t)r * nb + a) * 3 + ch, fixed_from_float(u[m]));
        }
      }
    }
  }
}

// Per-plane z-contraction of the finalisation's bin-to-bin differences:
// out[z][r1][r0][a] = sum_q beta_q(z) DY[(cell(z) + q, r1, r0)][a] (Eq. 7
// weights along z), for every bin a.
template <int DIM>
__global__ void __launch_bounds__(256)
k_zcontract_dy(const Geo g, const float2* __restrict__ DY, float2* __restrict__ out) {
  const int nb = g.nbins;
  const long long P1 = (long long)g.nsb[1] * g.nsb[0];
  const long long n = (long long)g.n[2] * P1 * nb;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const long long zr = i / nb;
    const int a = (int)(i - zr * nb);
    const int z = (int)(zr / P1);
    const long long rr = zr - (long long)z * P1;
    AxisEntry e;
    if (DIM == 3) axis_entry(g, 2, z, 0, 0, &e);
    else axis_unit(&e);
    const int NZ = DIM == 3 ? 4 : 1;
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NZ; ++q) {
      const int r2 = e.srel + q;
      if (r2 >= g.nsb[2] || e.bs[q] == 0.f) continue;
      const float2 d = __ldg(DY + (r2 * P1 + rr) * nb + a);
      s.x += e.bs[q] * d.x;
      s.y += e.bs[q] * d.y;
    }
    out[i] = s;
  }
}

__host__ __device__ inline long long zcontract_dy_len(const Geo& g) {
  return (long long)g.n[2] * g.nsb[1] * g.nsb[0] * g.nbins;
}

// Floats of the adjoint's control-point accumulators, rounded up to a
// multiple of 4 so that the float2 table after them starts on 16 bytes.
__host__ __device__ inline size_t adj_mas_a_gt_words(const Geo& g, int dim) {
  return (((size_t)dim * g.hf[0] * g.hf[1] * g.tile[2]) + 3) & ~(size_t)3;
}

__host__ __device__ inline size_t adj_rows_mas_a_smem_bytes(const Geo& g, int dim, int nxb) {
  size_t b = sizeof(float) * adj_mas_a_gt_words(g, dim);                  // gt
  b += sizeof(float2) * g.tile[2] * g.hb[1] * g.hb[0] * g.nbins;          // DYZ tile
  b += sizeof(float) * kAdjWarps * dim * kMaxRowNodes;                    // cyz
  b += sizeof(float) * xtab_words(nxb);                                   // x tables
  b += sizeof(AxisEntry) * (g.tile[1] + g.tile[2]);                       // y, z tables
  b += sizeof(float) * g.tile[2] * dim * g.hf[1] * g.hf[0];               // CZ
  return b;
}

template <int DIM, typename T, int NXB>
__device__ __forceinline__ void adj_rows_mas_a_body(const Geo& g, const AdjArgsA& args, int tile,
                                                    float* smem_f32) {
  const T* __restrict__ F = static_cast<const T*>(args.F);
  const T* __restrict__ M = static_cast<const T*>(args.M);
  const float* __restrict__ c = args.c;
  const float4* __restrict__ bg = args.bg;
  const unsigned char* __restrict__ rowlive = args.rowlive;
  float* __restrict__ grad = args.grad;
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nodes_tile = g.hf[0] * g.hf[1] * g.tile[2];
  const int p01 = g.hb[0] * g.hb[1];
  float* gt = smem_f32;
  float2* DYZ = reinterpret_cast<float2*>(gt + adj_mas_a_gt_words(g, DIM));   // [TZ][hb1][hb0][nb]
  float* cyz_all = reinterpret_cast<float*>(DYZ + (size_t)g.tile[2] * p01 * nb);
  const XTab xt = xtab_carve(cyz_all + kAdjWarps * DIM * kMaxRowNodes, NXB);
  AxisEntry* yt = reinterpret_cast<AxisEntry*>(reinterpret_cast<float*>(xt.frel) + xtab_words(NXB));
  AxisEntry* zt = yt + g.tile[1];
  float* CZ = reinterpret_cast<float*>(zt + g.tile[2]);
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;

  const TileOrigin TO = tile_setup<DIM>(g, tile);
  for (int i = threadIdx.x; i < DIM * nodes_tile; i += blockDim.x) gt[i] = 0.f;
  build_xtab<NXB>(g, TO, xt, (int)blockDim.x - 32);
  build_axis_tables<DIM>(g, TO, yt, zt);
  {
    // The tile's planes of the z-contracted table differences, every bin.
    const float2* __restrict__ dyz = args.dyz;
    const long long n = (long long)g.tile[2] * p01 * nb;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
      const long long e = t / nb;
      const int a = (int)(t - e * nb);
      const int zl = (int)(e / p01), hb01 = (int)(e - (long long)zl * p01);
      const int l1 = hb01 / g.hb[0], l0 = hb01 - l1 * g.hb[0];
      const int r0 = TO.cb[0] + l0, r1 = TO.cb[1] + l1, z = TO.o[2] + zl;
      float2 v = make_float2(0.f, 0.f);
      if (r0 < g.nsb[0] && r1 < g.nsb[1] && z < g.n[2])
        v = __ldg(dyz + (((long long)z * g.nsb[1] + r1) * g.nsb[0] + r0) * nb + a);
      DYZ[t] = v;
    }
  }
  __syncthreads();
  if (!bg) {
    build_cz<DIM>(g, TO, c, zt, CZ);
    __syncthreads();
  }
  const float scale = (args.gscale ? __ldg(args.gscale) : 1.f) * args.invZ;

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(TO.o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - TO.f[0] + 4;
  const int nrows = g.tile[1] * g.tile[2];
  const CyzSlots cslots = cyz_slots<DIM>(nxn, lane);
  // Live rows of this warp (rows with a nonzero moving-image gradient), as in
  // the M-as-B adjoint; loads in lane (x) order one live row ahead.
  struct RowLoad {
    float f;
    float4 b;
    int yl, zl;
    bool ok;
  };
  unsigned cand = 0;
  int kb = -32;
  int cyl = 0, czl = 0;
  auto refill = [&]() {
    kb += 32;
    const int row = warp + (kb + lane) * kAdjWarps;
    bool live = false;
    cyl = 0;
    czl = 0;
    if (row < nrows) {
      czl = row / g.tile[1];
      cyl = row - czl * g.tile[1];
      const int y = TO.o[1] + cyl, z = TO.o[2] + czl;
      live = y < g.n[1] && z < g.n[2];
      if (live && rowlive) live = rowlive[((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5)] != 0;
    }
    cand = __ballot_sync(0xffffffffu, live);
  };
  auto fetch_next = [&]() {
    RowLoad f{0.f, make_float4(0.f, 0.f, 0.f, 0.f), 0, 0, false};
    while (cand == 0) {
      if (warp + (kb + 32) * kAdjWarps >= nrows) return f;   // warp-uniform
      refill();
    }
    const int b = __ffs(cand) - 1;
    cand &= cand - 1;
    f.yl = __shfl_sync(0xffffffffu, cyl, b);
    f.zl = __shfl_sync(0xffffffffu, czl, b);
    f.ok = true;
    const int xn = TO.o[0] + lane;
    if (xn < g.n[0]) {
      const long long idx = ((long long)(TO.o[2] + f.zl) * g.n[1] + (TO.o[1] + f.yl)) * g.n[0] + xn;
      f.f = ldval(F + idx);
      if (bg) f.b = __ldg(bg + idx);
    }
    return f;
  };
  RowLoad nxt = fetch_next();
  while (nxt.ok) {
    const RowLoad cur = nxt;
    const int yl = cur.yl, zl = cur.zl;
    nxt = fetch_next();
    const int y = TO.o[1] + yl, z = TO.o[2] + zl;
    const AxisEntry ye = yt[yl];
    if (!bg) {
      row_cyz<DIM>(g, CZ, zl, ye, cslots, cyz);
      __syncwarp();
    }
    const int x = TO.o[0] + lane;
    const bool act = x < g.n[0];
    float gm[3] = {0.f, 0.f, 0.f};
    float Av = 0.f;
    if (act) {
      if (bg) {
        Av = cur.b.x;
        gm[0] = cur.b.y;
        gm[1] = cur.b.z;
        gm[2] = cur.b.w;
      } else {
        const float bx[4] = {xt.bf[lane], xt.bf[32 + lane], xt.bf[64 + lane], xt.bf[96 + lane]};
        Av = row_warp<DIM, T>(g, M, cyz, xt.frel[lane], bx, x, y, z, gm);
        Av = fminf(fmaxf(Av, 0.f), L);
      }
    }
    const bool live = act && (gm[0] != 0.f || gm[1] != 0.f || (DIM == 3 && gm[2] != 0.f));
    if (!__any_sync(0xffffffffu, live)) continue;  // dM/dy == 0 on the whole row
    float G = 0.f;
    if (live) {
      // Eq. (21): G = (h1'(f) / Z) sum_r w_r [DY2[r][a0] - 2 m1(F) DY1[r][a0]]
      // with w_r separable: x-bins of the lane, y-bins of the row, z done
      // per plane.
      float fa;
      const int a0 = bin_split(Av, nb, &fa);
      float m1, m2;
      row_parzen_moments(fminf(fmaxf(cur.f, 0.f), L), nb, &m1, &m2);
      const int sp = xt.srel[lane];
      const float2* base = DYZ + ((size_t)zl * g.hb[1] + ye.srel) * g.hb[0] * nb + a0;
      const size_t ystep = (size_t)g.hb[0] * nb;
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float w = xt.bs[i * 32 + lane];
        if (w == 0.f || sp + i >= g.hb[0]) continue;
        const float2* col = base + (size_t)(sp + i) * nb;
        float tx = 0.f, ty = 0.f;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const float2 d = col[jj * ystep];
          tx = fmaf(ye.bs[jj], d.x, tx);
          ty = fmaf(ye.bs[jj], d.y, ty);
        }
        s = fmaf(w, tx - 2.f * m1 * ty, s);
      }
      G = scale * parzen_upper_deriv(fa) * s;
    }
    // Scatter G dM/dy_k beta(node) to the row's control points (lanes are in
    // x order: lane = voxel).
    constexpr int NN = kMaxRowNodes;
    float vals[32];
    float bn[NN];
#pragma unroll
    for (int nn = 0; nn < NN; ++nn) bn[nn] = xt.bfp[nn * 32 + lane];
    float gk[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) gk[kk] = (live && kk < DIM) ? G * gm[kk] : 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) vals[q] = (q / NN < DIM) ? gk[q / NN] * bn[q % NN] : 0.f;
    const float tot = warp_reduce_scatter32(vals, lane);
    const int kq = lane / NN, lq = lane % NN;
    float* gpl = gt + (zl * g.hf[1] + ye.frel) * g.hf[0];
    if (lane < DIM * NN && lq < nxn && tot != 0.f) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float w = ye.bf[m];
        if (w == 0.f) continue;
        atomicAdd(gpl + kq * nodes_tile + m * g.hf[0] + lq, tot * w);
      }
    }
    if (DIM == 3 && nxn > 32 - 2 * NN) {
      float e = gk[2] * bn[32 - 2 * NN];
#pragma unroll
      for (int off = 16; off; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
      if (lane == 0 && e != 0.f) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float w = ye.bf[m];
          if (w == 0.f) continue;
          atomicAdd(gpl + 2 * nodes_tile + m * g.hf[0] + (32 - 2 * NN), e * w);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  constexpr int NJZ = DIM == 3 ? 4 : 1;
  const int per_plane = g.hf[1] * g.hf[0];
  for (int i = threadIdx.x; i < DIM * nodes_tile; i += blockDim.x) {
    const int k = i / nodes_tile, rem = i - k * nodes_tile;
    const int zl = rem / per_plane, myx = rem - zl * per_plane;
    const int fz = zt[zl].frel;
    if (zl > 0 && zt[zl - 1].frel == fz) continue;
    float u[NJZ];
#pragma unroll
    for (int n = 0; n < NJZ; ++n) u[n] = 0.f;
    bool any = false;
    for (int pl = zl; pl < g.tile[2] && zt[pl].frel == fz; ++pl) {
      const float v = gt[k * nodes_tile + pl * per_plane + myx];
      if (v == 0.f) continue;
      any = true;
#pragma unroll
      for (int n = 0; n < NJZ; ++n) u[n] = fmaf(zt[pl].bf[n], v, u[n]);
    }
    if (!any) continue;
    const int n0 = TO.f[0] + myx % g.hf[0], n1 = TO.f[1] + myx / g.hf[0];
    if (n0 >= g.nf[0] || n1 >= g.nf[1]) continue;
#pragma unroll
    for (int n = 0; n < NJZ; ++n) {
      const int n2 = TO.f[2] + fz + n;
      if (u[n] == 0.f || n2 >= g.nf[2]) continue;
      atomicAdd(grad + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0, u[n]);
    }
  }
}

template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(kAccWarps * 32, 2)
k_accumulate_rows_mas_a(const Geo g, const AccArgsA args, const int* __restrict__ order) {
  extern __shared__ __align__(16) unsigned long long smem_acc_a[];
  const int tile = order ? __ldg(order + blockIdx.x) : (int)blockIdx.x;   // as k_accumulate_rows
  acc_rows_mas_a_body<DIM, T, NXB>(g, args, tile, smem_acc_a);
}

template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(kAdjWarps * 32, 4)
k_adjoint_rows_mas_a(const Geo g, const AdjArgsA args, const int* __restrict__ order) {
  extern __shared__ __align__(16) float smem_adj_a[];
  const int tile = order ? __ldg(order + blockIdx.x) : (int)blockIdx.x;
  adj_rows_mas_a_body<DIM, T, NXB>(g, args, tile, smem_adj_a);
}

}  // namespace srwcr
