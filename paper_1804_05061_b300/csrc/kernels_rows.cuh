// Row-parallel SRWCR kernels for sm_103a (the fast path).
//
// A CTA owns a voxel tile 32 x TY x TZ; each warp walks x-rows of 32 voxels.
// Along a row y and z are fixed, so the y/z factors of every tensor-product
// B-spline (FFD nodes, Eq. 17; spatial bins, Eq. 7) are row constants.  All
// per-axis geometry (cells, B-spline weights) is computed once per CTA into
// shared-memory tables for the tile's 32 x-positions, TY y-rows and TZ
// z-planes, and everything that only depends on z is contracted once per
// z-plane in the CTA prologue:
//
//   * FFD: CZ[z][k][m][l] = sum_n beta_n(z) c_k[.., m, l]; per row the warp
//     finishes the y-contraction (4 FMAs per x-node), each voxel then needs
//     4 FMAs per component.
//   * Joint statistics (value pass): lanes are ordered by their fixed-image
//     bin a0 with a static per-row permutation (A does not change between
//     evaluations), so voxels sharing a0 are adjacent.  A segmented warp
//     reduction forms, per segment, the FP32 sums over <= 32 voxels of
//     beta_x(i) h(a - A) {m1, m2}; each sum is then spread over the
//     row-constant y/z weights (one lane per y/z bin) and added in 48-bit
//     fixed point to the CTA histogram, whose per-bin stride is odd so those
//     adds hit distinct banks.  Only short FP32 sums are ever formed, so the
//     E[b^2] - mu^2 cancellation of Eq. (10) keeps full accuracy.
//   * Adjoint: the region tables U, V, X are contracted over z per plane in
//     the prologue and over y per row; each voxel forms dD/dB (Eq. 19), and
//     the row's contributions to its control points are combined by a
//     reduce-scatter butterfly before one shared-memory add per (node,
//     component, y/z node).
//
// Rows in which every warped intensity is exactly 0 (m1 = m2 = 0) add nothing
// to the statistics, and rows in which the moving-image gradient vanishes at
// every voxel add nothing to the gradient; both are skipped.  A row whose
// static distance to the nearest nonzero moving-image voxel (L-infinity,
// voxels) exceeds its largest displacement bound by more than the trilinear
// stencil's reach reads only zeros: the value pass skips its warp, and it
// records for the adjoint which rows have a nonzero moving-image gradient,
// so that the adjoint visits only those.
#pragma once

#include "device_math.cuh"

namespace srwcr {

constexpr int kAccWarps = 16;           // value pass: 512 threads per CTA
constexpr int kAdjWarps = 8;            // adjoint: 256 threads per CTA
constexpr int kMaxRowNodes = 11;        // FFD x-nodes a 32-voxel row may touch
constexpr int kSentinel = 0x7fffffff;   // key of lanes past the image edge
// Adjoint: rows whose per-segment X table (segments x x-bins x 2 entries)
// would exceed this form X per lane instead.
constexpr int kAdjLaneXMin = 64;

// Per-axis geometry of one coordinate: FFD cell (relative to the tile's
// first node), its 4 weights, spatial-bin cell (relative to the tile's first
// bin) and its 4 weights (cubic B-spline, Eq. 7, or the boxcar patch of
// Eq. 6 with weights 1, 0, 0, 0).
struct AxisEntry {
  int frel;
  float bf[4];
  int srel;
  float bs[4];
};

__device__ __forceinline__ void axis_entry(const Geo& g, int d, int v, int f0, int c0,
                                           AxisEntry* e) {
  float t;
  e->frel = ffd_cell(g, d, v, &t) - f0;
  bspline4(t, e->bf);
  int sc;
  axis_weights(g, d, v, &sc, e->bs);
  e->srel = sc - c0;
}

// Trivial axis (2-D problems have no z).
__device__ __forceinline__ void axis_unit(AxisEntry* e) {
  e->frel = 0;
  e->srel = 0;
  e->bf[0] = e->bs[0] = 1.f;
  e->bf[1] = e->bf[2] = e->bf[3] = e->bs[1] = e->bs[2] = e->bs[3] = 0.f;
}

struct TileOrigin {
  int o[3];     // first voxel
  int f[3];     // first FFD node
  int cb[3];    // first spatial bin (cell)
};

template <int DIM>
__device__ __forceinline__ TileOrigin tile_setup(const Geo& g, int b) {
  TileOrigin T;
  T.o[0] = (b % g.ntile[0]) * g.tile[0];
  T.o[1] = ((b / g.ntile[0]) % g.ntile[1]) * g.tile[1];
  T.o[2] = (b / (g.ntile[0] * g.ntile[1])) * g.tile[2];
  float t;
  for (int d = 0; d < 3; ++d) {
    const bool on = d < DIM;
    T.f[d] = on ? T.o[d] / g.fsp[d] : 0;
    T.cb[d] = on ? sb_cell(g, d, T.o[d], &t) : 0;
  }
  return T;
}

// Lane-major x tables for the tile's 32 x-positions p (arrays [.][32], so a
// warp reading entry p per lane touches 32 consecutive words):
//   frel[p]            FFD cell relative to the tile's first node
//   bf[l][p]           FFD weights beta_l
//   bfp[n][p]          the same, placed at the row's x-node n (0 elsewhere)
//   srel[p], bs[i][p]  spatial-bin cell and weights
//   bsp[b][p]          spatial weights placed at the row's x-bin b
struct XTab {
  int* frel;
  float* bf;
  float* bfp;
  int* srel;
  float* bs;
  float* bsp;
};

__host__ __device__ inline size_t xtab_words(int nxb) { return 32 * (1 + 4 + kMaxRowNodes + 1 + 4 + nxb); }

__device__ __forceinline__ XTab xtab_carve(float* base, int nxb) {
  XTab t;
  t.frel = reinterpret_cast<int*>(base);
  t.bf = base + 32;
  t.bfp = t.bf + 4 * 32;
  t.srel = reinterpret_cast<int*>(t.bfp + kMaxRowNodes * 32);
  t.bs = reinterpret_cast<float*>(t.srel + 32);
  t.bsp = t.bs + 4 * 32;
  (void)nxb;
  return t;
}

// Built by the 32 threads from `first` on (the callers pass the last warp,
// whose share of the other prologue work is the smallest).
template <int NXB>
__device__ __forceinline__ void build_xtab(const Geo& g, const TileOrigin& T, XTab xt, int first) {
  const int p = (int)threadIdx.x - first;
  if (p >= 0 && p < 32) {
    AxisEntry e;
    axis_entry(g, 0, min(T.o[0] + p, g.n[0] - 1), T.f[0], T.cb[0], &e);
    xt.frel[p] = e.frel;
    xt.srel[p] = e.srel;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      xt.bf[l * 32 + p] = e.bf[l];
      xt.bs[l * 32 + p] = e.bs[l];
    }
    for (int n = 0; n < kMaxRowNodes; ++n) {
      const int l = n - e.frel;
      xt.bfp[n * 32 + p] = (l >= 0 && l < 4) ? e.bf[l] : 0.f;
    }
    for (int b = 0; b < NXB; ++b) {
      const int i = b - e.srel;
      xt.bsp[b * 32 + p] = (i >= 0 && i < 4) ? e.bs[i] : 0.f;
    }
  }
}

// Fill the y-table (tile[1]) and z-table (tile[2]).
template <int DIM>
__device__ __forceinline__ void build_axis_tables(const Geo& g, const TileOrigin& T,
                                                  AxisEntry* yt, AxisEntry* zt) {
  const int n = g.tile[1] + g.tile[2];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i < g.tile[1]) {
      const int y = min(T.o[1] + i, g.n[1] - 1);
      axis_entry(g, 1, y, T.f[1], T.cb[1], yt + i);
    } else {
      const int k = i - g.tile[1];
      if (DIM == 3) {
        const int z = min(T.o[2] + k, g.n[2] - 1);
        axis_entry(g, 2, z, T.f[2], T.cb[2], zt + k);
      } else {
        axis_unit(zt + k);
      }
    }
  }
}

// z-contracted FFD coefficients: CZ[z][k][m][l] for the tile's z-planes,
// components k, y-nodes m < hf1, x-nodes l < hf0 (read through L1/L2).
// Returns the bit pattern of the largest |entry| this thread wrote (as an
// unsigned, so a NaN entry makes it NaN; 0 if none).
template <int DIM>
__device__ __forceinline__ unsigned build_cz(const Geo& g, const TileOrigin& T, const float* __restrict__ c,
                                             const AxisEntry* zt, float* CZ) {
  // Threads are spread over the (y-node m, x-node l) pairs and, when there
  // are fewer pairs than threads, over the (plane, component) entries of a
  // pair; the index divisions are done once per thread.
  const int per_k = g.hf[1] * g.hf[0];
  const int per_z = DIM * per_k;
  const int nzk = g.tile[2] * DIM;
  const int tpp = per_k < (int)blockDim.x ? min((int)blockDim.x / per_k, nzk) : 1;
  unsigned mx = 0u;
  for (int t = threadIdx.x; t < per_k * tpp; t += blockDim.x) {
    const int sub = t / per_k, i = t - sub * per_k;
    const int m = i / g.hf[0], l = i - m * g.hf[0];
    const int n0 = T.f[0] + l, n1 = T.f[1] + m;
    const bool in = n0 < g.nf[0] && n1 < g.nf[1];
    for (int zk = sub; zk < nzk; zk += tpp) {
      const int zl = zk / DIM, k = zk - zl * DIM;
      const AxisEntry& e = zt[zl];
      float s = 0.f;
      if (in) {
        const int NZ = DIM == 3 ? 4 : 1;
        for (int q = 0; q < NZ; ++q) {
          const int n2 = T.f[2] + e.frel + q;
          if (n2 < g.nf[2])
            s += e.bf[q] * __ldg(c + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0);
        }
      }
      CZ[zl * per_z + k * per_k + i] = s;
      mx = max(mx, __float_as_uint(fabsf(s)));
    }
  }
  return mx;
}

// Per-row FFD table: cyz[k][l] = sum_m beta_m(y) CZ[z][k][ly + m][l].
// The lane's entries (component k, x-node l) of that table: t = lane and
// t = lane + 32, t < DIM * nxn (fixed for a tile, so decoded once).
struct CyzSlots {
  int n;        // entries of this lane (0, 1 or 2)
  int k[2], l[2];
};

template <int DIM>
__device__ __forceinline__ CyzSlots cyz_slots(int nxn, int lane) {
  CyzSlots s;
  s.n = (lane < DIM * nxn) + (lane + 32 < DIM * nxn);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int t = lane + 32 * j;
    s.k[j] = t / nxn;
    s.l[j] = t - s.k[j] * nxn;
  }
  return s;
}

// Returns the largest magnitude among the lane's entries: every voxel of the
// row is displaced by at most the warp-wide maximum along each axis (the
// x-weights of Eq. 17 are non-negative and sum to one).
template <int DIM>
__device__ __forceinline__ float row_cyz(const Geo& g, const float* CZ, int zl, const AxisEntry& ye,
                                         const CyzSlots& cs, float* cyz) {
  const int per_z = DIM * g.hf[1] * g.hf[0];
  float mx = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (j >= cs.n) break;
    const int k = cs.k[j], l = cs.l[j];
    const float* base = CZ + zl * per_z + (k * g.hf[1] + ye.frel) * g.hf[0] + l;
    const float v = ye.bf[0] * base[0] + ye.bf[1] * base[g.hf[0]] + ye.bf[2] * base[2 * g.hf[0]] +
                    ye.bf[3] * base[3 * g.hf[0]];
    cyz[k * kMaxRowNodes + l] = v;
    mx = fmaxf(mx, fabsf(v));
  }
  return mx;
}

// Reach of a row's trilinear stencil beyond its largest displacement bound
// U: reads lie within ceil(|u|) + 1 voxels of the voxel (L-infinity), and |u|
// exceeds U only by FP32 rounding, so a row with static distance d > U + 3 to
// the nearest nonzero moving-image voxel reads only zeros.
constexpr float kDeadRowMargin = 3.f;
// Cap of the static row distance (rows farther from any nonzero voxel store
// the cap, a lower bound).
constexpr int kRowDistCap = 64;

// A warp's next row (y, z within the tile), advanced by the number of warps
// without a division.
__device__ __forceinline__ void row_step(int step, int ty, int* yl, int* zl) {
  *yl += step;
  while (*yl >= ty) {
    *yl -= ty;
    ++*zl;
  }
}

// Warp the lane's voxel: displacement from the row table, trilinear sample.
template <int DIM, typename T>
__device__ __forceinline__ float row_warp(const Geo& g, const T* __restrict__ M, const float* cyz,
                                          int frel, const float bx[4], int x, int y, int z,
                                          float gm[3]) {
  float u[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float* cr = cyz + k * kMaxRowNodes + frel;
    u[k] = bx[0] * cr[0] + bx[1] * cr[1] + bx[2] * cr[2] + bx[3] * cr[3];
  }
  return sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
}

__device__ __forceinline__ float pick4(const float b[4], int i) {
  return i == 0 ? b[0] : (i == 1 ? b[1] : (i == 2 ? b[2] : (i == 3 ? b[3] : 0.f)));
}

// Per-problem arguments of the row kernels (also the batch descriptors).
struct AccArgs {
  const void* A;                 // normalised fixed image (storage type)
  const void* M;                 // normalised moving image (storage type)
  const float* c;                // FFD coefficients
  const unsigned char* perm;     // per-row lane permutation
  const unsigned* binmask;       // per-tile fixed-image bins present
  unsigned long long* acc;       // [R][nbins][2] fixed-point sums
  float4* bg;                    // per voxel (B, dM/dy) for the adjoint, or NULL
  const unsigned char* rowdist;  // per row: distance to the nearest nonzero M voxel, or NULL
  unsigned char* rowlive;        // per row: nonzero dM/dy somewhere (written with bg), or NULL
  float s1, s2;                  // fixed-point scales of the two moments
};

struct AdjArgs {
  const void* A;
  const void* M;
  const float* c;
  const unsigned char* perm;
  const unsigned* binmask;
  const float* U;
  const float* V;
  const float* X;
  const float* gscale;           // device scalar or NULL (1)
  const float4* bg;              // (B, dM/dy) stored by the value pass, or NULL: recompute
  const unsigned char* rowlive;  // rows with nonzero dM/dy (value pass, with bg), or NULL: all
  const float* uvxz;             // U, V, X contracted over z per image plane (k_zcontract)
  float invZ;
  float* grad;
};

// Bytes of the value kernel's shared memory (must match the carve-up below).
// Words per y/z bin of the split histogram: 2 * nabin * hb0 rounded up to
// 8 (mod 32), so the 4 y/z groups of a fold pass fall on disjoint banks.
// The intensity axis holds only the fixed-image bins the tile uses (a static
// per-tile mask), in compact order.
__host__ __device__ inline int hist_yz_stride(const Geo& g) {
  // At least 4 words past the row's last column (the value kernel's fold
  // adds zeros up to 3 words past it); 8 modulo 32.
  const int w = 2 * g.cbin * g.hb[0];
  return ((w + 27) / 32) * 32 + 8;
}

__host__ __device__ inline size_t acc_rows_smem_bytes(const Geo& g, int dim, int nxb) {
  const size_t npy = (size_t)g.tile[2] * g.hb[1];          // (z-plane, y-bin) rows
  const size_t nv = (size_t)(nxb == 12 ? 4 : nxb) * 4;   // segment values per chunk
  size_t b = 2 * npy * hist_yz_stride(g) * sizeof(unsigned);  // plane words (2 per entry)
  b += sizeof(float) * kAccWarps * 32 * nv;                 // segS
  b += sizeof(int) * kAccWarps * 32;                        // segA
  b += sizeof(int) * kAccWarps * 64 * 2;                    // bin list
  b += sizeof(int) * ((size_t)g.nbins + g.nabin);           // bin <-> compact index
  b += sizeof(float) * kAccWarps * dim * kMaxRowNodes;      // cyz
  b += sizeof(float) * xtab_words(nxb);                     // x tables
  b += sizeof(AxisEntry) * (g.tile[1] + g.tile[2]);         // y, z tables
  b += sizeof(float) * g.tile[2] * dim * g.hf[1] * g.hf[0]; // CZ
  b += sizeof(unsigned);                                    // tile displacement bound
  return b;
}

// ---------------------------------------------------------------------------
// (a) value pass: fused FFD + warp + joint statistics, row-parallel.
// ---------------------------------------------------------------------------

// Position of value q of row l in a warp's segment buffer of NV floats per
// row (a segment's totals sit in the row of its last lane).  With 8 x-bins
// per chunk (NV = 32, the transpose) 16-byte chunks are XOR-swizzled by the
// row index, so the row stores and the column reads are free of bank
// conflicts; with 4 the layout is plain.
template <int NV>
__device__ __forceinline__ int seg_at(int l, int q) {
  static_assert(NV == 16 || NV == 32, "4 or 8 x-bins per chunk");
  return NV == 32 ? l * 32 + (((q >> 2) ^ (l & 7)) << 2) + (q & 3) : l * 16 + q;
}

// SKIP: the level keeps the per-row records (static distance to nonzero M,
// nonzero-gradient flag); without them every row is processed and the
// per-row tests are compiled out.
template <int DIM, typename T, int NXB, bool SKIP = true>
__device__ __forceinline__ void acc_rows_body(const Geo& g, const AccArgs& args, int tile,
                                              unsigned long long* smem_u64) {
  const T* __restrict__ A = static_cast<const T*>(args.A);
  const T* __restrict__ M = static_cast<const T*>(args.M);
  const float* __restrict__ c = args.c;
  const unsigned char* __restrict__ perm = args.perm;
  const unsigned* __restrict__ binmask = args.binmask;
  unsigned long long* __restrict__ acc = args.acc;
  const unsigned char* __restrict__ rowdist = SKIP ? args.rowdist : nullptr;
  unsigned char* __restrict__ rowlive = SKIP ? args.rowlive : nullptr;
  const float s1 = args.s1, s2 = args.s2;
  // x-bins per chunk of a row (a row with 12 takes three chunks of 4) and
  // segment-buffer values per chunk: v[4b + 2 slot + ch].
  constexpr int XC = NXB == 12 ? 4 : NXB;
  constexpr int NV = XC * 4;
  constexpr int NK = DIM == 3 ? 4 : 1;        // z bins of a row
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Per-plane fixed-point accumulators H[z-plane][y bin][bin][moment][x-bin]:
  // a row's sums are weighted by its y B-spline only (4 updates per item);
  // the z weights are applied once per plane at the flush.  Each entry is
  // held as two 32-bit words (bits 0-23 and 24-47 of each update, which is
  // < 2^48) and receives at most one update per row of its plane (<= 256),
  // so neither word overflows (256 * (2^24 - 1) < 2^32).  The flush
  // recombines a plane's words exactly, combines the planes of one z cell in
  // FP32 in plane order with their z weights and adds the results to the
  // global accumulators.
  // The bin axis holds g.cbin of the tile's compacted bins; a tile that uses
  // more takes several passes over its rows, each folding one chunk of bins
  // and skipping rows with no voxel in that chunk.
  const int S = hist_yz_stride(g);
  const int NPY = g.tile[2] * g.hb[1];
  unsigned* hlo = reinterpret_cast<unsigned*>(smem_u64);
  unsigned* hhi = hlo + (size_t)NPY * S;
  float* segS = reinterpret_cast<float*>(hhi + (size_t)NPY * S);
  int* segA = reinterpret_cast<int*>(segS + kAccWarps * 32 * NV);
  int* binl = segA + kAccWarps * 32;          // [warp][64][2]: a, (row | slot<<8 | merge<<9 | prev row<<10)
  int* a2c = binl + kAccWarps * 64 * 2;       // fixed-image bin -> compact index (-1: unused)
  int* c2a = a2c + nb;                        // compact index -> bin
  float* cyz_all = reinterpret_cast<float*>(c2a + g.nabin);
  const XTab xt = xtab_carve(cyz_all + kAccWarps * DIM * kMaxRowNodes, NXB);
  AxisEntry* yt = reinterpret_cast<AxisEntry*>(reinterpret_cast<float*>(xt.frel) + xtab_words(NXB));
  AxisEntry* zt = yt + g.tile[1];
  float* CZ = reinterpret_cast<float*>(zt + g.tile[2]);
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;
  float* mysegS = segS + warp * 32 * NV;
  int* mybins = binl + warp * 64 * 2;

  const TileOrigin TO = tile_setup<DIM>(g, tile);
  const int cb = g.cbin;
  // Prologue in two phases: the y/z tables, then (independent of each other)
  // the z-contraction of the coefficients (global loads issued first), the
  // bin maps, the x table and the clearing of the first pass's accumulators
  // (16-byte stores; 2 * NPY * S is a multiple of 4 words).
  // The tile's displacement bound: the largest |entry| of CZ bounds every
  // row's coefficient table (non-negative y weights summing to one).
  unsigned* tile_u = reinterpret_cast<unsigned*>(CZ + g.tile[2] * DIM * g.hf[1] * g.hf[0]);
  if (threadIdx.x == 0) *tile_u = 0u;
  build_axis_tables<DIM>(g, TO, yt, zt);
  __syncthreads();
  {
    const unsigned mx = build_cz<DIM>(g, TO, c, zt, CZ);
    if (SKIP && rowdist) {
      const unsigned wmx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) atomicMax(tile_u, wmx);
    }
  }
  int cnt = 0;                                // compacted bins of this tile
  {
    const int words = (nb + 31) >> 5;
    const unsigned* tmask = binmask + (size_t)tile * words;
    for (int k = 0; k < words; ++k) cnt += __popc(__ldg(tmask + k));
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      const int w = a >> 5;
      const unsigned mw = __ldg(tmask + w);
      int before = __popc(mw & ((1u << (a & 31)) - 1u));
      for (int k = 0; k < w; ++k) before += __popc(__ldg(tmask + k));
      const bool used = (mw >> (a & 31)) & 1u;
      a2c[a] = used ? before : -1;
      if (used) c2a[before] = a;
    }
  }
  build_xtab<NXB>(g, TO, xt, (int)blockDim.x - 32);
  const int hwords4 = (2 * NPY * S) >> 2;
  uint4* h4 = reinterpret_cast<uint4*>(hlo);
  for (int i = threadIdx.x; i < hwords4; i += blockDim.x) h4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(TO.o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - TO.f[0] + 4;   // FFD x-nodes of the row
  const int nrows = g.tile[1] * g.tile[2];
  const CyzSlots cslots = cyz_slots<DIM>(nxn, lane);
  for (int c0 = 0; c0 < cnt; c0 += cb) {
    const bool multi = cnt > cb;                // CTA-uniform
    if (c0 > 0) {                               // the first pass was cleared above
      for (int i = threadIdx.x; i < hwords4; i += blockDim.x) h4[i] = make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();
    }
    // A row's permutation and fixed-image values are loaded in lane order
    // (independent of each other) one row ahead; the value lane l needs,
    // that of voxel o + perm[l], comes by shuffle.
    auto fetch = [&](int yr, int zr, int* pp, float* aa, int* dd) {
      *pp = 0;
      *aa = 0.f;
      *dd = 0;
      if (zr >= g.tile[2]) return false;          // past the tile's last row
      const int y = TO.o[1] + yr, z = TO.o[2] + zr;
      if (y >= g.n[1] || z >= g.n[2]) return false;
      const long long rowid = ((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5);
      *pp = perm[rowid * 32 + lane];
      if (SKIP && rowdist) *dd = rowdist[rowid];
      const int xn = TO.o[0] + lane;
      if (xn < g.n[0]) *aa = ldval(A + ((long long)z * g.n[1] + y) * g.n[0] + xn);
      return true;
    };
    // The warp's rows are row = warp + k * kAccWarps.  On levels with the
    // per-row distances, a row farther than the tile's displacement bound
    // + 3 from the nonzero moving image is empty whatever its own bound (it
    // is at most the tile's): the warp reads the distances of 32 of its
    // rows at a time, records those rows as having no moving-image
    // gradient and visits only the others (each then takes the exact
    // per-row test below).
    const bool scan = SKIP && rowdist != nullptr;   // CTA-uniform
    const float Ut = __uint_as_float(*tile_u);
    unsigned cand = 0;                          // candidates kb .. kb + 31 not yet visited
    int kb = -32;
    auto refill = [&]() {
      kb += 32;
      const int r = warp + (kb + lane) * kAccWarps;
      bool cnd = false;
      if (r < nrows) {
        const int zr = r / g.tile[1], yr = r - zr * g.tile[1];
        const int y = TO.o[1] + yr, z = TO.o[2] + zr;
        if (y < g.n[1] && z < g.n[2]) {
          const long long rowid = ((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5);
          cnd = !((float)rowdist[rowid] > Ut + kDeadRowMargin);   // NaN bound: kept
          if (!cnd && rowlive) rowlive[rowid] = 0;
        }
      }
      cand = __ballot_sync(0xffffffffu, cnd);
    };
    auto next_candidate = [&]() {
      while (cand == 0) {
        if (warp + (kb + 32) * kAccWarps >= nrows) return nrows;   // warp-uniform
        refill();
      }
      const int b = __ffs(cand) - 1;
      cand &= cand - 1;
      return warp + (kb + b) * kAccWarps;
    };
    int p_next, d_next;
    float a_next;
    int row = scan ? next_candidate() : warp;   // row = zn * tile[1] + yn
    int zn = row / g.tile[1], yn = row - zn * g.tile[1];
    bool ok_next = fetch(yn, zn, &p_next, &a_next, &d_next);
    while (row < nrows) {
      const int p = p_next;
      const float a_lane = a_next;
      const int rdist = d_next;
      const bool ok = ok_next;
      const int yl = yn, zl = zn;
      if (scan) {
        row = next_candidate();
        zn = row / g.tile[1];
        yn = row - zn * g.tile[1];
      } else {
        row += kAccWarps;
        row_step(kAccWarps, g.tile[1], &yn, &zn);
      }
      ok_next = fetch(yn, zn, &p_next, &a_next, &d_next);
      if (!ok) continue;  // warp-uniform
      const int y = TO.o[1] + yl, z = TO.o[2] + zl;
      const long long rowid = ((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5);

      const int x = TO.o[0] + p;
      const bool act = x < g.n[0];
      const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
      const float av = __shfl_sync(0xffffffffu, a_lane, p);
      float fa = 0.f;
      int key = kSentinel;
      if (act) key = bin_split(fminf(fmaxf(av, 0.f), L), nb, &fa);
      if (multi) {
        // Rows with no voxel whose bins fall in this chunk wait for their pass.
        const bool in = act && ((unsigned)(a2c[key] - c0) < (unsigned)cb ||
                                (unsigned)(a2c[key + 1] - c0) < (unsigned)cb);
        if (!__any_sync(0xffffffffu, in)) continue;
      }
      const AxisEntry ye = yt[yl];
      const float umax = row_cyz<DIM>(g, CZ, zl, ye, cslots, cyz);
      if (SKIP && rowdist) {
        // Row provably reading only zeros of M: B = 0 and dM/dy = 0 at every
        // voxel, nothing to add (warp-uniform; NaN coefficients never pass).
        const float U = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(umax)));
        if ((float)rdist > U + kDeadRowMargin) {
          if (rowlive && lane == 0) rowlive[rowid] = 0;
          continue;
        }
      }
      __syncwarp();
      float m1 = 0.f, m2 = 0.f, h0 = 0.f, h1 = 0.f;
      bool glive = false;
      if (act) {
        h1 = parzen_upper(fa);
        h0 = 1.f - h1;
        const float bx[4] = {xt.bf[p], xt.bf[32 + p], xt.bf[64 + p], xt.bf[96 + p]};
        float gm[3];
        float B = row_warp<DIM, T>(g, M, cyz, xt.frel[p], bx, x, y, z, gm);
        B = fminf(fmaxf(B, 0.f), L);
        if (args.bg) args.bg[idx] = make_float4(B, gm[0], gm[1], gm[2]);
        if (SKIP) glive = gm[0] != 0.f || gm[1] != 0.f || gm[2] != 0.f;
        float fb;
        const int kb = bin_split(B, nb, &fb);
        const float w1 = parzen_upper(fb), kf = (float)kb;
        m1 = kf + w1;                              // sum_b b   h(b - B)
        m2 = kf * kf + (2.f * kf + 1.f) * w1;      // sum_b b^2 h(b - B)
      }
      if (SKIP && rowlive) {
        const bool any_g = __any_sync(0xffffffffu, glive);
        if (lane == 0) rowlive[rowid] = any_g ? 1 : 0;
      }
      const bool live = act && (m1 != 0.f || m2 != 0.f);
      if (!__any_sync(0xffffffffu, live)) continue;  // B == 0 on the whole row

      const float e0 = live ? h0 * m1 : 0.f, e1 = live ? h0 * m2 : 0.f;
      const float e2 = live ? h1 * m1 : 0.f, e3 = live ? h1 * m2 : 0.f;
      // Segments of equal a0 (lanes are sorted by a0).
      const int prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || key != prev;
      const unsigned heads = __ballot_sync(0xffffffffu, head);
      const unsigned above = lane == 31 ? 0u : (heads & (0xffffffffu << (lane + 1)));
      const unsigned ends = (heads >> 1) | 0x80000000u;   // last lane of each segment
      // The row's x-bins in chunks of XC (one chunk unless NXB = 12); the bin
      // list is built after the first chunk's segment sums.
      int nbin = 0;
      for (int q0 = 0; q0 < NXB && q0 < g.hb[0]; q0 += XC) {
        // Per-lane contributions over the chunk's spatial x-bins.
        float v[NV];
  #pragma unroll
        for (int b = 0; b < XC; ++b) {
          const float w = xt.bsp[(q0 + b) * 32 + p];
          v[4 * b + 0] = w * e0;
          v[4 * b + 1] = w * e1;
          v[4 * b + 2] = w * e2;
          v[4 * b + 3] = w * e3;
        }
        // Segment sums; a segment's NV totals end up in the row of its last
        // lane in the warp's segment buffer.
        //  * 8 x-bins per chunk: transpose.  Lane l stores its NV values as
        //    row l, then lane q sums column q down the rows in lane order and,
        //    at the last lane of each segment, writes the running sum (the
        //    segment's total) back into that row (already read): 32 loads and
        //    one store per segment instead of a 5-level shuffle over 32
        //    values, however many segments the row has.
        //  * 4 x-bins: segmented shuffle reduction toward each head, which
        //    stores its segment's totals (with 16 values the shuffle tree
        //    beats a transpose).
        if (NV == 32) {
          float4* rowp = reinterpret_cast<float4*>(mysegS);
  #pragma unroll
          for (int k = 0; k < NV / 4; ++k)
            rowp[seg_at<NV>(lane, 4 * k) >> 2] =
                make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          __syncwarp();
          float sum = 0.f;
  #pragma unroll
          for (int l = 0; l < 32; ++l) {
            const int at = seg_at<NV>(l, lane);
            sum += mysegS[at];
            if ((ends >> l) & 1u) {
              mysegS[at] = sum;
              sum = 0.f;
            }
          }
        } else {
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
          if (head && key != kSentinel) {
            float4* rowp = reinterpret_cast<float4*>(mysegS);
  #pragma unroll
            for (int k = 0; k < NV / 4; ++k)
              rowp[seg_at<NV>(seg_end - 1, 4 * k) >> 2] =
                  make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          }
        }
        __syncwarp();
        if (q0 == 0) {
          // Bin list.  Segment s (key a) adds bin a (slot 0, plus slot 1 of
          // s-1 when that segment's key is a-1) and, unless segment s+1 has
          // key a+1, bin a+1 (slot 1 alone).  An entry names the rows holding
          // the totals: its segment's last lane and, when merged, the last
          // lane of segment s-1 (the head's left neighbour).
          const int next_head = above ? __ffs(above) - 1 : -1;
          const int last = next_head < 0 ? 31 : next_head - 1;
          const int next_key = __shfl_sync(0xffffffffu, key, next_head < 0 ? lane : next_head);
          const bool real = head && key != kSentinel;
          const bool upper = real && (next_head < 0 || next_key != key + 1);
          const unsigned below = heads & ((1u << lane) - 1u);
          const int prev_head = below ? 31 - __clz(below) : lane;
          const int prev_key = __shfl_sync(0xffffffffu, key, prev_head);
          const bool merge = real && below && prev_key + 1 == key;
          // Only bins of the current bin pass are listed.
          const bool in0 = real && (unsigned)(a2c[key] - c0) < (unsigned)cb;
          const bool in1 = upper && (unsigned)(a2c[key + 1] - c0) < (unsigned)cb;
          const unsigned emit0 = __ballot_sync(0xffffffffu, in0);
          const unsigned emit1 = __ballot_sync(0xffffffffu, in1);
          const unsigned lt = (1u << lane) - 1u;
          const int pos = __popc(emit0 & lt) + __popc(emit1 & lt);
          nbin = __popc(emit0) + __popc(emit1);
          if (in0) {
            mybins[2 * pos] = key;
            mybins[2 * pos + 1] = last | (merge ? (1 << 9) | ((lane - 1) << 10) : 0);
          }
          if (in1) {
            const int q = pos + (in0 ? 1 : 0);
            mybins[2 * q] = key + 1;
            mybins[2 * q + 1] = last | (1 << 8);
          }
          __syncwarp();
        }
        // Fold: each lane takes whole (bin, moment, x-bin) items (32 per
        // pass) and adds each to the row's 4 y bins of its z-plane (one item
        // decode per item; all 32 lanes of an update touch one y row,
        // consecutive items consecutive columns).
        const int prow = (zl * g.hb[1] + ye.srel) * S;
        const int per_bin = 2 * XC;
        // The body has no branch: an item past the row's x-bins or with a
        // zero sum carries uv = 0 and adds zeros, which costs fewer
        // instructions than skipping the additions.  Past the x-bins a
        // column lies at most 3 words beyond the last one of its y row
        // (NXB - hb0 <= 3), inside the row's spare words.
        for (int f = lane; f < nbin * per_bin; f += 32) {
          const int e = f / per_bin, r = f % per_bin;
          const int ch = r / XC, b = r % XC;
          const int bx_ = q0 + b;                  // the row's x-bin
          const int a = mybins[2 * e];
          const int info = mybins[2 * e + 1];
          const int sg = info & 0xff, slot = (info >> 8) & 1;
          const float v0 = mysegS[seg_at<NV>(sg, 4 * b + 2 * slot + ch)];
          const float v1 = mysegS[seg_at<NV>((info >> 10) & 31, 4 * b + 2 + ch)];
          const float val = (info & (1 << 9)) ? v0 + v1 : v0;
          const float uv = bx_ < g.hb[0] ? val * (ch ? s2 : s1) : 0.f;
          const int col = prow + ((a2c[a] - c0) * 2 + ch) * g.hb[0] + bx_;
  #pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float u = uv * ye.bs[m];
            // Split of u (< 2^48) into 24-bit fields: the power-of-two
            // scaling, the floor and the fused subtraction are exact; the low
            // field rounds u's fraction (u < 2^24) to the fixed-point unit.
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
    // Flush: one entry per (first plane of a z cell, y bin, column); the
    // planes of that cell are combined with their z weights, then the NK z
    // bins are added to the global accumulators.
    // Threads are spread over the columns (bin, moment, x bin) and, when
    // there are fewer columns than threads, over the y bins of a column; each
    // loops over the first planes of the z cells and its y bins.  Consecutive
    // threads take consecutive (bin, moment) pairs of one x bin, so a warp's
    // global additions fall on consecutive words of one region's record.
    // Their shared-memory stride is then the x-bin count; when that is a
    // multiple of 4, each group of 8 pairs starts at another x bin, which
    // spreads a warp's reads over all 32 banks.
    const int nach = 2 * cb;
    const int wcols = nach * g.hb[0];
    const int tpc = wcols < (int)blockDim.x ? min((int)blockDim.x / wcols, g.hb[1]) : 1;
    const bool rotate = (g.hb[0] & 3) == 0;
    const size_t ystride = (size_t)g.nsb[0] * nb * 2, zstride = ystride * g.nsb[1];
    for (int t = threadIdx.x; t < wcols * tpc; t += blockDim.x) {
      const int sub = t / wcols, i = t - sub * wcols;
      const int bq = i / nach, ach = i - bq * nach;
      if (c0 + (ach >> 1) >= cnt) continue;
      const int b = rotate ? (bq + (ach >> 3)) % g.hb[0] : bq;
      const int r0 = TO.cb[0] + b;
      if (r0 >= g.nsb[0]) continue;
      const int col = ach * g.hb[0] + b;
      const int a = c2a[c0 + (ach >> 1)], ch = ach & 1;
      unsigned long long* accx = acc + ((size_t)r0 * nb + a) * 2 + ch;
      for (int zl = 0; zl < g.tile[2]; ++zl) {
        const int cz = zt[zl].srel;
        if (zl > 0 && zt[zl - 1].srel == cz) continue;
        const int r2b = TO.cb[2] + cz;
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
          unsigned long long* accy = accx + (size_t)r1 * ystride + (size_t)r2b * zstride;
#pragma unroll
          for (int m = 0; m < NK; ++m) {
            if (u[m] == 0.f || r2b + m >= g.nsb[2]) continue;
            atomicAdd(accy + (size_t)m * zstride, fixed_from_float(u[m]));
          }
        }
      }
    }
    __syncthreads();                            // the next pass clears the accumulators
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

// The adjoint's X table is X[plane][y bin][bin a][x bin] with the x-bin
// stride made odd: a warp's reads of one (y bin, x bin) for lanes of
// different bins and neighbouring x bins (a row's bins are few and close)
// then fall in different shared-memory banks unless the bins are about
// 32 / stride apart, and one bin at neighbouring x bins is contiguous.
__host__ __device__ inline int adj_x_stride(const Geo& g) { return g.hb[0] | 1; }

// Bytes of the adjoint's shared memory (must match the carve-up below).
__host__ __device__ inline size_t adj_rows_smem_bytes(const Geo& g, int dim, int nxb) {
  const size_t hf = (size_t)g.hf[0] * g.hf[1] * g.tile[2];         // per-plane nodes
  const size_t p01 = (size_t)g.hb[0] * g.hb[1];
  size_t b = sizeof(float) * dim * hf;                               // gt
  b += sizeof(float) * g.tile[2] * p01 * 2;                          // UZ, VZ
  b += sizeof(float) * g.tile[2] * g.hb[1] * g.nbins * adj_x_stride(g);  // XZ
  b += sizeof(float) * kAdjWarps * (2 * nxb + 32 * nxb * 2);         // rowt, xy
  b += sizeof(int) * kAdjWarps * 32;                                 // segA
  b += sizeof(float) * kAdjWarps * dim * kMaxRowNodes;               // cyz
  b += sizeof(float) * xtab_words(nxb);                              // x tables
  b += sizeof(AxisEntry) * (g.tile[1] + g.tile[2]);                  // y, z tables
  b += sizeof(float) * g.tile[2] * dim * g.hf[1] * g.hf[0];          // CZ
  return b;
}

// ---------------------------------------------------------------------------
// (c) adjoint, row-parallel.
// ---------------------------------------------------------------------------
template <int DIM, typename T, int NXB>
__device__ __forceinline__ void adj_rows_body(const Geo& g, const AdjArgs& args, int tile,
                                              float* smem_f32) {
  const T* __restrict__ A = static_cast<const T*>(args.A);
  const T* __restrict__ M = static_cast<const T*>(args.M);
  const float* __restrict__ c = args.c;
  const unsigned char* __restrict__ perm = args.perm;
  const unsigned* __restrict__ binmask = args.binmask;
  const float* __restrict__ gscale = args.gscale;
  const float invZ = args.invZ;
  float* __restrict__ grad = args.grad;
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Control-point accumulators per z-plane of the tile: gt[k][zl][m][l] over
  // the tile's y/x nodes; the z-node weights are applied once per plane at
  // the flush.
  const int nodes_tile = g.hf[0] * g.hf[1] * g.tile[2];
  const int p01 = g.hb[0] * g.hb[1];
  float* gt = smem_f32;
  float* UZ = gt + DIM * nodes_tile;                 // [TZ][hb1][hb0]
  float* VZ = UZ + g.tile[2] * p01;
  const int hx = adj_x_stride(g);
  const int xzy = nb * hx;                           // words per (plane, y bin) of XZ
  float* XZ = VZ + g.tile[2] * p01;                  // [TZ][hb1][nb][hx]
  float* rowt_all = XZ + (size_t)g.tile[2] * g.hb[1] * xzy;
  float* xy_all = rowt_all + kAdjWarps * 2 * NXB;
  int* segA_all = reinterpret_cast<int*>(xy_all + kAdjWarps * 32 * NXB * 2);
  float* cyz_all = reinterpret_cast<float*>(segA_all + kAdjWarps * 32);
  const XTab xt = xtab_carve(cyz_all + kAdjWarps * DIM * kMaxRowNodes, NXB);
  AxisEntry* yt = reinterpret_cast<AxisEntry*>(reinterpret_cast<float*>(xt.frel) + xtab_words(NXB));
  AxisEntry* zt = yt + g.tile[1];
  float* CZ = reinterpret_cast<float*>(zt + g.tile[2]);
  float* rowt = rowt_all + warp * 2 * NXB;
  float* xy = xy_all + warp * 32 * NXB * 2;
  int* mysegA = segA_all + warp * 32;
  float* cyz = cyz_all + warp * DIM * kMaxRowNodes;

  const float4* __restrict__ bg = args.bg;  // CTA-uniform: stored warp or recompute
  const TileOrigin TO = tile_setup<DIM>(g, tile);
  for (int i = threadIdx.x; i < DIM * nodes_tile; i += blockDim.x) gt[i] = 0.f;
  build_xtab<NXB>(g, TO, xt, (int)blockDim.x - 32);
  build_axis_tables<DIM>(g, TO, yt, zt);
  // Region tables contracted over z for each of the tile's z-planes, read
  // from the per-plane tables of k_zcontract (in the same phase as the axis
  // tables, which this does not read).  X is only needed for the
  // fixed-image bins present in the tile (a0 and a0+1 of its voxels, a static
  // mask); other entries are never read.
  const unsigned* tmask = binmask + (size_t)tile * ((nb + 31) >> 5);
  {
    const long long nzp_g = (long long)g.n[2] * g.nsb[1] * g.nsb[0];
    const float* __restrict__ UZg = args.uvxz;
    const float* __restrict__ VZg = UZg + nzp_g;
    const float* __restrict__ XZg = UZg + 2 * nzp_g;
    // Threads are spread over the (plane, y/x bin) entries and, when there
    // are fewer entries than threads, over the columns (U, V, X[a]) of an
    // entry; the index divisions are done once per thread.
    const int nzp = g.tile[2] * p01;
    const int ncol = 2 + nb;                  // 0 = U, 1 = V, 2 + a = X[a]
    const int tpe = nzp < (int)blockDim.x ? min((int)blockDim.x / nzp, ncol) : 1;
    for (int t = threadIdx.x; t < nzp * tpe; t += blockDim.x) {
      const int sub = t / nzp, e = t - sub * nzp;
      const int zl = e / p01, hb01 = e - zl * p01;
      const int l1 = hb01 / g.hb[0], l0 = hb01 - l1 * g.hb[0];
      const int r0 = TO.cb[0] + l0, r1 = TO.cb[1] + l1;
      const int z = TO.o[2] + zl;
      const bool in = r0 < g.nsb[0] && r1 < g.nsb[1] && z < g.n[2];
      const long long zr = in ? ((long long)z * g.nsb[1] + r1) * g.nsb[0] + r0 : 0;
      for (int col = sub; col < ncol; col += tpe) {
        if (col >= 2) {
          const int a = col - 2;
          if (!((__ldg(tmask + (a >> 5)) >> (a & 31)) & 1u)) continue;
        }
        float s = 0.f;
        if (in) s = col == 0 ? __ldg(UZg + zr) : (col == 1 ? __ldg(VZg + zr) : __ldg(XZg + zr * nb + (col - 2)));
        if (col == 0) UZ[e] = s;
        else if (col == 1) VZ[e] = s;
        else XZ[(size_t)(zl * g.hb[1] + l1) * xzy + (col - 2) * hx + l0] = s;
      }
    }
  }
  __syncthreads();
  if (!bg) {
    build_cz<DIM>(g, TO, c, zt, CZ);
    __syncthreads();
  }
  const float scale = (gscale ? __ldg(gscale) : 1.f) * invZ;

  const int nxb = (g.n[0] + 31) >> 5;
  const int xlast = min(TO.o[0] + 31, g.n[0] - 1);
  const int nxn = xlast / g.fsp[0] - TO.f[0] + 4;
  const int nrows = g.tile[1] * g.tile[2];
  // The warp's rows are row = warp + k * kAdjWarps, k = 0, 1, ...  With the
  // value pass's record of the rows whose moving-image gradient is nonzero
  // somewhere (rowlive), only those are visited: 32 candidates' flags are
  // read at a time and the set ones taken in order.  A row's loads (lane
  // order, lane l reading voxel o + l, so they do not wait for the
  // permutation) are issued one live row ahead of its processing; the
  // permuted values are then exchanged by shuffles.
  const unsigned char* __restrict__ rowlive = args.rowlive;
  struct RowLoad {
    int p;
    float a;
    float4 b;
    int yl, zl;
    bool ok;
  };
  unsigned cand = 0;       // flags of candidates kb .. kb + 31 not yet taken
  int kb = -32;
  int cyl = 0, czl = 0;    // this lane's candidate kb + lane: (y, z) within the tile
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
    RowLoad f{0, 0.f, make_float4(0.f, 0.f, 0.f, 0.f), 0, 0, false};
    while (cand == 0) {
      if (warp + (kb + 32) * kAdjWarps >= nrows) return f;   // warp-uniform
      refill();
    }
    const int b = __ffs(cand) - 1;
    cand &= cand - 1;
    f.yl = __shfl_sync(0xffffffffu, cyl, b);
    f.zl = __shfl_sync(0xffffffffu, czl, b);
    f.ok = true;
    const int y = TO.o[1] + f.yl, z = TO.o[2] + f.zl;
    const long long rowid = ((long long)z * g.n[1] + y) * nxb + (TO.o[0] >> 5);
    f.p = perm[rowid * 32 + lane];
    const int xn = TO.o[0] + lane;
    if (xn < g.n[0]) {
      const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + xn;
      f.a = ldval(A + idx);
      if (bg) f.b = __ldg(bg + idx);
    }
    return f;
  };
  const CyzSlots cslots = cyz_slots<DIM>(nxn, lane);
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

    const int p = cur.p;
    const int x = TO.o[0] + p;
    const bool act = x < g.n[0];
    const float av = __shfl_sync(0xffffffffu, cur.a, p);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (bg) {  // the value pass at the same coefficients stored the warp
      s.x = __shfl_sync(0xffffffffu, cur.b.x, p);
      s.y = __shfl_sync(0xffffffffu, cur.b.y, p);
      s.z = __shfl_sync(0xffffffffu, cur.b.z, p);
      s.w = __shfl_sync(0xffffffffu, cur.b.w, p);
    }
    float gm[3] = {0.f, 0.f, 0.f};
    float dm1 = 0.f, dm2 = 0.f, h0 = 0.f, h1 = 0.f;
    int key = kSentinel;
    if (act) {
      float fa;
      key = bin_split(fminf(fmaxf(av, 0.f), L), nb, &fa);
      h1 = parzen_upper(fa);
      h0 = 1.f - h1;
      float B;
      if (bg) {
        B = s.x;
        gm[0] = s.y;
        gm[1] = s.z;
        gm[2] = s.w;
      } else {
        const float bx[4] = {xt.bf[p], xt.bf[32 + p], xt.bf[64 + p], xt.bf[96 + p]};
        B = row_warp<DIM, T>(g, M, cyz, xt.frel[p], bx, x, y, z, gm);
        B = fminf(fmaxf(B, 0.f), L);
      }
      float fb;
      const int kb = bin_split(B, nb, &fb);
      dm1 = parzen_upper_deriv(fb);
      dm2 = (2.f * (float)kb + 1.f) * dm1;
    }
    const bool live = act && (gm[0] != 0.f || gm[1] != 0.f || (DIM == 3 && gm[2] != 0.f));
    if (!__any_sync(0xffffffffu, live)) continue;  // grad M == 0 on the whole row

    // Row tables: U, V over the y bins (z done per plane) for the row's x-bins.
    const float* UZr = UZ + zl * p01;
    const float* VZr = VZ + zl * p01;
    for (int tt = lane; tt < 2 * NXB; tt += 32) {
      const int b = tt % NXB;
      const float* tab = tt < NXB ? UZr : VZr;
      float s = 0.f;
      if (b < g.hb[0])
        for (int jj = 0; jj < 4; ++jj) s += ye.bs[jj] * tab[(ye.srel + jj) * g.hb[0] + b];
      rowt[tt] = s;
    }
    // Segments of equal a0.  X summed over the row's y bins is formed either
    // once per segment for every x-bin of the row (few segments), or, in rows
    // with many segments (speckled fixed images), by each lane for its own
    // 4 x-bins and 2 a-bins only (warp-uniform choice; the same sums in the
    // same order either way).
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || key != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int nseg = __popc(heads);
    const float* XZr = XZ + (size_t)zl * g.hb[1] * xzy;
    const bool xlane = nseg * NXB * 2 > kAdjLaneXMin;
    if (!xlane) {
      if (head) mysegA[__popc(heads & ((1u << lane) - 1u))] = key;
      __syncwarp();
      for (int it = lane; it < nseg * NXB * 2; it += 32) {
        const int s = it / (NXB * 2), rem = it % (NXB * 2), b = rem >> 1, slot = rem & 1;
        const int a = mysegA[s];
        float acc_x = 0.f;
        if (a != kSentinel && b < g.hb[0]) {
          for (int jj = 0; jj < 4; ++jj)
            acc_x += ye.bs[jj] * XZr[(size_t)(ye.srel + jj) * xzy + (a + slot) * hx + b];
        }
        xy[(s * NXB + b) * 2 + slot] = acc_x;
      }
    }
    __syncwarp();
    float G = 0.f;
    if (live) {
      float su = 0.f, sv = 0.f, sxr = 0.f;
      if (xlane) {
        const int sp = xt.srel[p];
        const int ystep = xzy;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int b = sp + i;
          const float w = xt.bs[i * 32 + p];
          if (w == 0.f || b >= g.hb[0]) continue;
          su += w * rowt[b];
          sv += w * rowt[NXB + b];
          const float* xr = XZr + (size_t)ye.srel * xzy + key * hx + b;
          float x0 = 0.f, x1 = 0.f;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            x0 += ye.bs[jj] * xr[jj * ystep];
            x1 += ye.bs[jj] * xr[jj * ystep + hx];
          }
          sxr += w * (h0 * x0 + h1 * x1);
        }
      } else {
        const int sidx = __popc(heads & ((2u << lane) - 1u)) - 1;
#pragma unroll
        for (int b = 0; b < NXB; ++b) {
          const float w = xt.bsp[b * 32 + p];
          su += w * rowt[b];
          sv += w * rowt[NXB + b];
          sxr += w * (h0 * xy[(sidx * NXB + b) * 2] + h1 * xy[(sidx * NXB + b) * 2 + 1]);
        }
      }
      G = scale * (dm2 * su + 2.f * dm1 * (sv - sxr));
    }
    // Value q = 11 k + n: component k, row x-node n (n < nxn <= 11), for
    // q < 32; in 3-D the 33rd (k = 2, n = 10) is summed on its own.
    constexpr int NN = kMaxRowNodes;
    float vals[32];
    float bn[NN];
#pragma unroll
    for (int nn = 0; nn < NN; ++nn) bn[nn] = xt.bfp[nn * 32 + p];
    float gk[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) gk[kk] = (live && kk < DIM) ? G * gm[kk] : 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) vals[q] = (q / NN < DIM) ? gk[q / NN] * bn[q % NN] : 0.f;
    const float tot = warp_reduce_scatter32(vals, lane);
    // Lane q holds component q/11, x-node q%11: spread over the y/z nodes.
    const int kq = lane / NN, lq = lane % NN;
    float* gpl = gt + (zl * g.hf[1] + ye.frel) * g.hf[0];   // this row's plane, first y node
    if (lane < DIM * NN && lq < nxn && tot != 0.f) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float w = ye.bf[m];
        if (w == 0.f) continue;
        atomicAdd(gpl + kq * nodes_tile + m * g.hf[0] + lq, tot * w);
      }
    }
    if (DIM == 3 && nxn > 32 - 2 * NN) {     // rows touching 11 x-nodes (warp-uniform)
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
  // Flush: per (component, first plane of an FFD z cell, y node, x node),
  // combine that cell's planes with their z-node weights and add the NJZ z
  // nodes to the gradient.
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

// One problem: one CTA per tile.  order[b] (NULL: b) is the tile of CTA b:
// blocks start roughly in index order, so listing the costly tiles first
// leaves the cheap ones for the end of the launch, where they fill the SMs
// that the last costly tiles leave idle.
template <int DIM, typename T, int NXB, bool SKIP>
__global__ void __launch_bounds__(kAccWarps * 32, 2)
k_accumulate_rows(const Geo g, const AccArgs args, const int* __restrict__ order) {
  extern __shared__ __align__(16) unsigned long long smem_acc[];
  const int tile = order ? __ldg(order + blockIdx.x) : (int)blockIdx.x;
  acc_rows_body<DIM, T, NXB, SKIP>(g, args, tile, smem_acc);
}

template <int DIM, typename T, int NXB>
__global__ void __launch_bounds__(kAdjWarps * 32, 4)
k_adjoint_rows(const Geo g, const AdjArgs args, const int* __restrict__ order) {
  extern __shared__ __align__(16) float smem_adj[];
  const int tile = order ? __ldg(order + blockIdx.x) : (int)blockIdx.x;
  adj_rows_body<DIM, T, NXB>(g, args, tile, smem_adj);
}

// Region tables contracted over z for every image plane z.  Output layout:
// [U | V | X], U and V as [z][r1][r0] (P = nz * nsb1 * nsb0 plane-columns),
// X as [z][r1][r0][a]; each entry is sum_q beta_q(z) T[(cell(z) + q, r1, r0)]
// (Eq. 7 weights along z; the same terms and order as a per-tile
// contraction).  Only the X entries of the nu fixed-image bins that occur
// anywhere in the image (ubins) are formed; the adjoint reads no other.
__host__ __device__ inline long long zcontract_len(const Geo& g) {
  return (long long)g.n[2] * g.nsb[1] * g.nsb[0] * (2 + g.nbins);
}

// The batched contraction enumerates entries over all planes at once (item
// i), each item forming its plane's weights: with many pairs of uneven
// plane counts in one launch, that keeps every block's threads on
// independent entries.
__host__ __device__ inline long long zcontract_items(const Geo& g, int nu) {
  return (long long)g.n[2] * g.nsb[1] * g.nsb[0] * (2 + nu);
}

template <int DIM>
__device__ __forceinline__ void zcontract_item(const Geo& g, long long i, const int* __restrict__ ubins,
                                               int nu, const float* __restrict__ U,
                                               const float* __restrict__ V,
                                               const float* __restrict__ X, float* __restrict__ out) {
  const int nb = g.nbins;
  const long long P1 = (long long)g.nsb[1] * g.nsb[0];
  const long long nzp = (long long)g.n[2] * P1;
  long long zr, o;
  int col;
  if (i < 2 * nzp) {
    col = (int)(i / nzp);
    zr = i - col * nzp;
    o = i;
  } else {
    const long long r = i - 2 * nzp;
    zr = r / nu;
    const int a = __ldg(ubins + (r - zr * nu));
    col = 2 + a;
    o = 2 * nzp + zr * nb + a;
  }
  const int z = (int)(zr / P1);
  const long long rr = zr - (long long)z * P1;
  AxisEntry e;
  if (DIM == 3) axis_entry(g, 2, z, 0, 0, &e);
  else axis_unit(&e);
  const int NZ = DIM == 3 ? 4 : 1;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < NZ; ++q) {
    const int r2 = e.srel + q;
    if (r2 >= g.nsb[2]) continue;
    const long long r = r2 * P1 + rr;
    const float tv = col == 0 ? __ldg(U + r) : (col == 1 ? __ldg(V + r) : __ldg(X + r * nb + (col - 2)));
    s += e.bs[q] * tv;
  }
  out[o] = s;
}

// Entry i of image plane z (weights e of that plane): i < 2 P enumerates U
// and V over the plane's P = nsb1 * nsb0 spatial-bin columns, then X for the
// nu bins of ubins per column.
template <int DIM>
__device__ __forceinline__ void zcontract_entry(const Geo& g, const AxisEntry& e, int z, long long i,
                                                const int* __restrict__ ubins, int nu,
                                                const float* __restrict__ U, const float* __restrict__ V,
                                                const float* __restrict__ X, float* __restrict__ out) {
  const int nb = g.nbins;
  const long long P1 = (long long)g.nsb[1] * g.nsb[0];
  const long long nzp = (long long)g.n[2] * P1;
  int col;
  long long rr, o;
  if (i < 2 * P1) {
    col = (int)(i / P1);
    rr = i - col * P1;
    o = col * nzp + (long long)z * P1 + rr;
  } else {
    const long long r = i - 2 * P1;
    rr = r / nu;
    const int a = __ldg(ubins + (r - rr * nu));
    col = 2 + a;
    o = 2 * nzp + ((long long)z * P1 + rr) * nb + a;
  }
  const int NZ = DIM == 3 ? 4 : 1;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < NZ; ++q) {
    const int r2 = e.srel + q;
    if (r2 >= g.nsb[2]) continue;
    const long long r = r2 * P1 + rr;
    const float tv = col == 0 ? __ldg(U + r) : (col == 1 ? __ldg(V + r) : __ldg(X + r * nb + (col - 2)));
    s += e.bs[q] * tv;
  }
  out[o] = s;
}

// The plane's z cell and weights (Eq. 7 weights along z), formed by thread 0
// into shared memory; every thread of the block must call it.
template <int DIM>
__device__ __forceinline__ AxisEntry zcontract_plane(const Geo& g, int z, AxisEntry* ze) {
  __syncthreads();                              // earlier readers of *ze are done
  if (threadIdx.x == 0) {
    if (DIM == 3) axis_entry(g, 2, z, 0, 0, ze);
    else axis_unit(ze);
  }
  __syncthreads();
  return *ze;
}

// Block (x, z) takes a share of image plane z's entries; the plane's z cell
// and weights are formed once per block, the entries summed with the same
// terms in the same order as before.  The blocks also clear the nzero floats
// at `zero` (the gradient the adjoint that follows accumulates into), which
// saves the step a memset.
template <int DIM>
__global__ void __launch_bounds__(256)
k_zcontract(const Geo g, const int* __restrict__ ubins, int nu, const float* __restrict__ U,
            const float* __restrict__ V, const float* __restrict__ X, float* __restrict__ out,
            float* __restrict__ zero, long long nzero) {
  __shared__ AxisEntry ze;
  const int z = blockIdx.y;
  const long long nthr = (long long)gridDim.x * gridDim.y * 256;
  for (long long i = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 256 + threadIdx.x; i < nzero;
       i += nthr)
    zero[i] = 0.f;
  const AxisEntry e = zcontract_plane<DIM>(g, z, &ze);
  const long long per = (2 + nu) * (long long)g.nsb[1] * g.nsb[0];   // entries of one plane
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < per; i += (long long)gridDim.x * 256)
    zcontract_entry<DIM>(g, e, z, i, ubins, nu, U, V, X, out);
}

// Static L-infinity distance (voxels, capped at kRowDistCap) from each voxel
// to the nearest voxel where the moving image is nonzero, by separable
// passes: along x the distance within the x-line, then along y and z
// d(v) = min over offsets t of max(|t|, d_prev(v + t e_axis)) (the L-infinity
// distance is the largest per-axis offset, minimised axis by axis).  Capped
// values are lower bounds of the true distance.
template <typename T>
__global__ void k_mdist_x(const Geo g, const T* __restrict__ M, unsigned char* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n[0]);
    const long long line = i - x;
    int best = kRowDistCap;
    for (int t = 0; t < best; ++t) {
      const bool lo = x - t >= 0 && ldval(M + line + x - t) != 0.f;
      const bool hi = x + t < g.n[0] && ldval(M + line + x + t) != 0.f;
      if (lo || hi) { best = t; break; }
    }
    d[i] = (unsigned char)best;
  }
}

// One separable pass along axis `axis` (1 = y, 2 = z): out(v) = min over t
// of max(|t|, in(v + t e_axis)), |t| < kRowDistCap.
__global__ void k_mdist_pass(const Geo g, int axis, const unsigned char* __restrict__ in,
                             unsigned char* __restrict__ out) {
  const long long stride = axis == 1 ? g.n[0] : (long long)g.n[0] * g.n[1];
  const int n = g.n[axis];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)((i / stride) % n);
    int best = in[i];
    for (int t = 1; t < best; ++t) {
      const int lo = c - t >= 0 ? in[i - t * stride] : kRowDistCap;
      const int hi = c + t < n ? in[i + t * stride] : kRowDistCap;
      best = min(best, max(t, min(lo, hi)));
    }
    out[i] = (unsigned char)best;
  }
}

// Per 32-voxel x-row (row id ((z * ny + y) * nxb + x / 32)): the smallest
// distance over its voxels.
__global__ void k_row_dist(const Geo g, const unsigned char* __restrict__ d,
                           unsigned char* __restrict__ rowdist) {
  const int nxb = (g.n[0] + 31) >> 5;
  const long long nrows = (long long)nxb * g.n[1] * g.n[2];
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    const int xb = (int)(r % nxb);
    const long long yz = r / nxb;
    int best = kRowDistCap;
    for (int x = xb * 32; x < min(xb * 32 + 32, g.n[0]); ++x) best = min(best, (int)d[yz * g.n[0] + x]);
    rowdist[r] = (unsigned char)best;
  }
}

// Static per-tile mask of the fixed-image bins its voxels touch (a0, a0+1).
template <int DIM, typename T>
__global__ void k_tile_binmask(const Geo g, const T* __restrict__ A, unsigned* __restrict__ mask) {
  const float L = (float)(g.nbins - 1);
  const int words = (g.nbins + 31) >> 5;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n[0]), y = (int)((i / g.n[0]) % g.n[1]),
              z = (int)(i / ((long long)g.n[0] * g.n[1]));
    const int t = (x / g.tile[0]) + g.ntile[0] * ((y / g.tile[1]) + g.ntile[1] * (z / g.tile[2]));
    float fa;
    const int a0 = bin_split(fminf(fmaxf(ldval(A + i), 0.f), L), g.nbins, &fa);
    atomicOr(mask + (size_t)t * words + (a0 >> 5), 1u << (a0 & 31));
    atomicOr(mask + (size_t)t * words + ((a0 + 1) >> 5), 1u << ((a0 + 1) & 31));
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
