// SRWCR kernels for sm_103a.
//
//   k_accumulate  (a) fused FFD + warp + joint statistics: per voxel the 4^d
//                 spatial bins x 2 fixed-intensity bins of Eqs. (3)/(7) get
//                 the moving-intensity moments sum_b b h(b-B), sum_b b^2 h(b-B)
//                 (STATIC = false) or the weight w h(a-A) itself
//                 (STATIC = true, computed once per context: p(r), p_r(a)
//                 do not depend on the transform).  Sums are kept in 64-bit
//                 fixed point in a CTA-private shared-memory histogram and
//                 merged once per CTA, so the result does not depend on the
//                 order of the atomic additions.
//   k_finalize    (b) per spatial bin, in FP64: Eqs. (9)/(10)/(12), the
//                 region's share of D and the tables the gradient needs.
//   k_reduce_D    deterministic FP64 sum of the regions' shares.
//   k_adjoint     (c) recomputes the warp, forms dD/dB(x) of Eq. (19) from
//                 the tables and scatters dD/dB * grad M * dT/dc (Eqs. 16-17)
//                 into a CTA-private tile of control points.
#pragma once

#include "device_math.cuh"

namespace srwcr {

// Non-negative float -> 64-bit fixed point (round to nearest).
__device__ __forceinline__ unsigned long long to_fixed(float v) {
  return fixed_from_float(v);
}

// Exact 64-bit add into a shared-memory word with two native 32-bit atomics
// (a 64-bit shared atomic add is not a single instruction): the low word's
// wrap-around, seen in the value the first atomic returns, is carried into
// the high word.  Once all adds are done the word holds the exact sum.
__device__ __forceinline__ void shared_add_u64(unsigned long long* p, unsigned long long v) {
  unsigned* w = reinterpret_cast<unsigned*>(p);       // little-endian: low word first
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  unsigned carry = 0u;
  if (lo) {
    const unsigned old = atomicAdd(w, lo);
    carry = old + lo < old ? 1u : 0u;
  }
  if (hi + carry) atomicAdd(w + 1, hi + carry);
}

template <int DIM>
__device__ __forceinline__ void tile_origin(const Geo& g, int b, int o[3]) {
  const int t0 = b % g.ntile[0];
  const int t1 = (b / g.ntile[0]) % g.ntile[1];
  const int t2 = b / (g.ntile[0] * g.ntile[1]);
  o[0] = t0 * g.tile[0];
  o[1] = t1 * g.tile[1];
  o[2] = t2 * g.tile[2];
}

// Histogram layout in shared memory: [hb2][hb1][hb0][nbins][NCH] uint64.
// Global accumulators: [R][nbins][NCH] uint64 (fixed point).  RIGID: c is
// the rigid table (kRigidTab floats) and T is the rigid model.
template <int DIM, typename T, bool STATIC, bool RIGID = false>
__global__ void __launch_bounds__(256)
k_accumulate(const Geo g, const T* __restrict__ A, const T* __restrict__ M,
             const float* __restrict__ c, unsigned long long* __restrict__ acc, float s0,
             float s1) {
  Rigid rg{};
  if (RIGID) rg = load_rigid(c);
  extern __shared__ __align__(16) unsigned long long hist[];
  constexpr int NCH = STATIC ? 1 : 2;
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  int o[3];
  tile_origin<DIM>(g, blockIdx.x, o);
  float tdum;
  const int cb0 = sb_cell(g, 0, o[0], &tdum);
  const int cb1 = sb_cell(g, 1, o[1], &tdum);
  const int cb2 = DIM == 3 ? sb_cell(g, 2, o[2], &tdum) : 0;
  const int hsz = g.hb[0] * g.hb[1] * g.hb[2] * nb * NCH;
  for (int i = threadIdx.x; i < hsz; i += blockDim.x) hist[i] = 0ull;
  __syncthreads();

  const int tv = g.tile[0] * g.tile[1] * g.tile[2];
  for (int v = threadIdx.x; v < tv; v += blockDim.x) {
    const int x = o[0] + v % g.tile[0];
    const int y = o[1] + (v / g.tile[0]) % g.tile[1];
    const int z = o[2] + v / (g.tile[0] * g.tile[1]);
    if (x >= g.n[0] || y >= g.n[1] || z >= g.n[2]) continue;
    const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
    // Fixed-image bins a0, a0+1 with Parzen weights (Eq. 5).
    float fa;
    const float av = fminf(fmaxf(ldval(A + idx), 0.f), L);
    const int a0 = bin_split(av, nb, &fa);
    const float h1 = parzen_upper(fa), h0 = 1.f - h1;
    float m1 = 0.f, m2 = 0.f;
    if (!STATIC) {
      float u[3], gm[3];
      if (RIGID) {
        rigid_displacement<DIM>(rg, x, y, z, u);
      } else {
        float bw[3][4];
        int fc[3];
        ffd_displacement<DIM>(g, c, x, y, z, u, fc, bw);
      }
      float B = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1],
                                      (float)z + u[2], gm);
      B = fminf(fmaxf(B, 0.f), L);
      float fb;
      const int kb = bin_split(B, nb, &fb);
      const float w1 = parzen_upper(fb);
      const float kf = (float)kb;
      m1 = kf + w1;                              // sum_b b   h(b - B)
      m2 = kf * kf + (2.f * kf + 1.f) * w1;      // sum_b b^2 h(b - B)
    }
    int sc[3];
    float sw[3][4];
    spatial_weights<DIM>(g, x, y, z, sc, sw);
    const int NZ = DIM == 3 ? 4 : 1;
    for (int k = 0; k < NZ; ++k)
      for (int j = 0; j < 4; ++j) {
        const float wjk = sw[1][j] * sw[2][k];
        const int hrow = ((sc[2] - cb2 + k) * g.hb[1] + (sc[1] - cb1 + j)) * g.hb[0] + (sc[0] - cb0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float w = wjk * sw[0][i];
          if (w == 0.f) continue;
          unsigned long long* hp = hist + (size_t)(hrow + i) * nb * NCH;
          const float wa0 = w * h0, wa1 = w * h1;
          if (STATIC) {
            if (wa0 != 0.f) shared_add_u64(hp + a0, to_fixed(wa0 * s0));
            if (wa1 != 0.f) shared_add_u64(hp + a0 + 1, to_fixed(wa1 * s0));
          } else {
            if (wa0 != 0.f) {
              shared_add_u64(hp + 2 * a0, to_fixed(wa0 * m1 * s0));
              shared_add_u64(hp + 2 * a0 + 1, to_fixed(wa0 * m2 * s1));
            }
            if (wa1 != 0.f) {
              shared_add_u64(hp + 2 * a0 + 2, to_fixed(wa1 * m1 * s0));
              shared_add_u64(hp + 2 * a0 + 3, to_fixed(wa1 * m2 * s1));
            }
          }
        }
      }
  }
  __syncthreads();
  // Merge the CTA's nonzero entries into the global accumulators.
  for (int i = threadIdx.x; i < hsz; i += blockDim.x) {
    const unsigned long long val = hist[i];
    if (!val) continue;
    const int ch = i % NCH;
    const int a = (i / NCH) % nb;
    const int hbin = i / (NCH * nb);
    const int l0 = hbin % g.hb[0];
    const int l1 = (hbin / g.hb[0]) % g.hb[1];
    const int l2 = hbin / (g.hb[0] * g.hb[1]);
    if (cb0 + l0 >= g.nsb[0] || cb1 + l1 >= g.nsb[1] || cb2 + l2 >= g.nsb[2]) continue;
    const long long r = ((long long)(cb2 + l2) * g.nsb[1] + (cb1 + l1)) * g.nsb[0] + (cb0 + l0);
    atomicAdd(acc + ((size_t)r * nb + a) * NCH + ch, val);
  }
}

// Fixed point -> FP64 for the static statistics P[r][a].
__global__ void k_fixed_to_double(const unsigned long long* __restrict__ in, double inv_scale,
                                  double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i] * inv_scale;
}

// (b) One warp per spatial bin r, FP64 throughout (Table I):
//   W_r = sum_a P, T1 = sum_a S1, T2 = sum_a S2, mu_r = T1/W, sigma_r^2 = T2/W - mu^2,
//   Q_r = sum_a (S2 - S1^2/P) = W_r sum_a sigma_r^2(a) p_r(a)        (Eqs. 9, 10)
//   1 - CR_r = Q_r/(W_r sigma_r^2),  share of D = Q_r/(Z sigma_r^2)      (Eq. 9)
// and the gradient tables of Eq. (19) with the b-sum done in closed form:
//   U_r = CR_r/sigma_r^2,  V_r = (1-CR_r) mu_r/sigma_r^2,  X_ra = mu_r(a)/sigma_r^2.
__device__ __forceinline__ void finalize_region(const Geo& g, long long r, int lane,
                                                const double* __restrict__ P,
                                                const unsigned long long* __restrict__ S,
                                                double inv_s1, double inv_s2, double invZ,
                                                float* __restrict__ U, float* __restrict__ V,
                                                float* __restrict__ X, double* __restrict__ Dr,
                                                double* __restrict__ stats) {
  const int nb = g.nbins;
  const double* Pr = P + r * nb;
  const unsigned long long* Sr = S + r * nb * 2;
  double W = 0.0, T1 = 0.0, T2 = 0.0;
  for (int a = lane; a < nb; a += 32) {
    W += Pr[a];
    T1 += (double)Sr[2 * a] * inv_s1;
    T2 += (double)Sr[2 * a + 1] * inv_s2;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    W += __shfl_xor_sync(0xffffffffu, W, off);
    T1 += __shfl_xor_sync(0xffffffffu, T1, off);
    T2 += __shfl_xor_sync(0xffffffffu, T2, off);
  }
  bool valid = W > 0.0;
  double mu = 0.0, var = 0.0, ms = 0.0;
  if (valid) {
    mu = T1 / W;
    ms = T2 / W;
    var = ms - mu * mu;
    valid = var > 1e-6 * fmax(1.0, ms);  // degenerate: sigma_r^2 -> 0 (0/0 in Eq. 9)
  }
  double Q = 0.0;
  for (int a = lane; a < nb; a += 32) {
    const double p = Pr[a];
    double x = 0.0;
    if (valid && p > 0.0) {
      const double s1 = (double)Sr[2 * a] * inv_s1, s2 = (double)Sr[2 * a + 1] * inv_s2;
      Q += s2 - s1 * s1 / p;
      x = (s1 / p) / var;
    }
    X[r * nb + a] = (float)x;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) Q += __shfl_xor_sync(0xffffffffu, Q, off);
  if (lane == 0) {
    double omc = 0.0, share = 0.0;
    if (valid) {
      omc = Q / (W * var);
      share = Q * invZ / var;
    }
    U[r] = valid ? (float)((1.0 - omc) / var) : 0.f;
    V[r] = valid ? (float)(omc * mu / var) : 0.f;
    Dr[r] = share;
    stats[4 * r + 0] = W * invZ;
    stats[4 * r + 1] = valid ? var : 0.0;
    stats[4 * r + 2] = valid ? 1.0 - omc : 0.0;
    stats[4 * r + 3] = share;
  }
}

// Static per-region data of the fixed image that the finalisation reuses at
// every evaluation: W_r = sum_a P[r][a] = Z p(r) and its reciprocal, and the
// bins with P[r][a] > 0 (the only ones where S1, S2 can be nonzero) with
// 1/P[r][a], in compressed rows.
struct RegionStatic {
  const double* W;      // [R]
  const double* inv_w;  // [R] 1 / W_r (0 where W_r = 0)
  const int* ptr;       // [R+1] row offsets into bin/inv_p
  const int* bin;       // [nnz] fixed-image bin a
  const double* inv_p;  // [nnz] 1 / P[r][a]
};

// Same quantities as finalize_region, over the static nonzero bins only, by
// a group of G lanes (G divides 32; sub = lane index within the group):
// the moment sums T1 = sum_a S1[r][a], T2 = sum_a S2[r][a] are formed exactly
// in 64-bit integers and rounded once, divisions by P and W become products
// with the stored reciprocals, and one division (1 / sigma_r^2) per region
// remains.  Q_r = sum_a (S2 - S1^2 / P) is taken as T2 - sum_a S1 mu_r(a).
// A group with live == false (past the last region, or an inactive batch
// pair) still takes part in the group shuffles and writes nothing.  X entries
// of bins outside the list stay at the zero they were initialised to.  FP64
// issue is the bound of this step, so small G (several regions per warp)
// pays when the lists are short and regions are many.
template <int G>
__device__ __forceinline__ void finalize_region_sparse(long long r, bool live, int sub, int nb,
                                                       const RegionStatic& rs,
                                                       const unsigned long long* __restrict__ S,
                                                       double inv_s1, double inv_s2, double invZ,
                                                       float* __restrict__ U, float* __restrict__ V,
                                                       float* __restrict__ X, double* __restrict__ Dr,
                                                       double* __restrict__ stats) {
  const unsigned long long* Sr = S + (live ? r : 0) * nb * 2;
  const int beg = live ? rs.ptr[r] : 0, end = live ? rs.ptr[r + 1] : 0;
  unsigned long long t1 = 0ull, t2 = 0ull;
  for (int k = beg + sub; k < end; k += G) {
    const ulonglong2 s = *reinterpret_cast<const ulonglong2*>(Sr + 2 * rs.bin[k]);
    t1 += s.x;
    t2 += s.y;
  }
#pragma unroll
  for (int off = G / 2; off; off >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, off, G);
    t2 += __shfl_xor_sync(0xffffffffu, t2, off, G);
  }
  const double W = live ? rs.W[r] : 0.0, iw = live ? rs.inv_w[r] : 0.0;
  bool valid = W > 0.0;
  double mu = 0.0, var = 0.0, ms = 0.0;
  if (valid) {
    mu = (double)t1 * inv_s1 * iw;
    ms = (double)t2 * inv_s2 * iw;
    var = ms - mu * mu;
    valid = var > 1e-6 * fmax(1.0, ms);  // degenerate: sigma_r^2 -> 0 (0/0 in Eq. 9)
  }
  const double iv = valid ? 1.0 / var : 0.0;
  double q = 0.0;  // this lane's share of sum_a S1 mu_r(a)
  for (int k = beg + sub; k < end; k += G) {
    const int a = rs.bin[k];
    double x = 0.0;
    if (valid) {
      const double s1 = (double)Sr[2 * a] * inv_s1;
      const double m = s1 * rs.inv_p[k];     // mu_r(a) = S1 / P
      q = fma(s1, m, q);
      x = m * iv;
    }
    X[r * nb + a] = (float)x;
  }
#pragma unroll
  for (int off = G / 2; off; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off, G);
  if (live && sub == 0) {
    double omc = 0.0, share = 0.0;
    if (valid) {
      const double Q = (double)t2 * inv_s2 - q;
      omc = Q * iv * iw;
      share = Q * invZ * iv;
    }
    U[r] = valid ? (float)((1.0 - omc) * iv) : 0.f;
    V[r] = valid ? (float)(omc * mu * iv) : 0.f;
    Dr[r] = share;
    stats[4 * r + 0] = W * invZ;
    stats[4 * r + 1] = valid ? var : 0.0;
    stats[4 * r + 2] = valid ? 1.0 - omc : 0.0;
    stats[4 * r + 3] = share;
  }
}

// Lanes per region of the sparse finalisation.
constexpr int kFinLanes[6] = {1, 2, 4, 8, 16, 32};

template <int G>
__global__ void __launch_bounds__(256)
k_finalize_sparse(long long R, int nb, const RegionStatic rs,
                  const unsigned long long* __restrict__ S, double inv_s1, double inv_s2,
                  double invZ, float* __restrict__ U, float* __restrict__ V,
                  float* __restrict__ X, double* __restrict__ Dr, double* __restrict__ stats) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  if ((r - (threadIdx.x & 31) / G) >= R) return;  // the warp's first region: warp-uniform
  finalize_region_sparse<G>(r, r < R, threadIdx.x & (G - 1), nb, rs, S, inv_s1, inv_s2, invZ, U,
                            V, X, Dr, stats);
}

__global__ void k_finalize(const Geo g, const double* __restrict__ P,
                           const unsigned long long* __restrict__ S, double inv_s1,
                           double inv_s2, double invZ, float* __restrict__ U,
                           float* __restrict__ V, float* __restrict__ X, double* __restrict__ Dr,
                           double* __restrict__ stats) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (r >= g.R) return;  // warp-uniform
  finalize_region(g, r, threadIdx.x & 31, P, S, inv_s1, inv_s2, invZ, U, V, X, Dr, stats);
}

// Deterministic sum of the regions' shares (fixed partition, fixed tree).
// D_copy (may be null): a second place for D (the caller's device buffer,
// or device-mapped page-locked host memory), so no copy of D follows.
__device__ __forceinline__ void reduce_D_block(const double* __restrict__ Dr,
                                               const double* __restrict__ stats, long long R,
                                               double* __restrict__ D, int* __restrict__ ndeg,
                                               double* D_copy = nullptr) {
  __shared__ double sh[1024];
  __shared__ int shn[1024];
  double s = 0.0;
  int nd = 0;
  for (long long r = threadIdx.x; r < R; r += blockDim.x) {
    s += Dr[r];
    nd += stats[4 * r + 1] > 0.0 ? 0 : 1;
  }
  sh[threadIdx.x] = s;
  shn[threadIdx.x] = nd;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[threadIdx.x] += sh[threadIdx.x + w];
      shn[threadIdx.x] += shn[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    D[0] = sh[0];
    ndeg[0] = shn[0];
    if (D_copy) *reinterpret_cast<volatile double*>(D_copy) = sh[0];
  }
}

__global__ void __launch_bounds__(1024)
k_reduce_D(const double* __restrict__ Dr, const double* __restrict__ stats, long long R,
           double* __restrict__ D, int* __restrict__ ndeg, double* D_copy = nullptr) {
  reduce_D_block(Dr, stats, R, D, ndeg, D_copy);
}

// (c) Adjoint.  dD/dB(x) of Eq. (19) with the b-sums in closed form:
//   G(x) = (1/Z) [ m2'(B) sum_r w_r U_r + 2 m1'(B) sum_r w_r (V_r - sum_a h(a-A) X_ra) ]
// with m1' = d/dB sum_b b h(b-B), m2' = d/dB sum_b b^2 h(b-B); then
//   g[k][node] += G(x) dM/dy_k(T(x)) beta(node; x)                     (Eqs. 16, 17)
// accumulated in a CTA-private tile [DIM][hf2][hf1][hf0] of control points.
// dD/dB at voxel (x, y, z) (Eq. 19 with the b-sums in closed form, Eq. 27):
// scale * [m2'(B) sum_r w_r U_r + 2 m1'(B) sum_r w_r (V_r - sum_a h X_{r,a})]
// over the voxel's spatial bins, with U = CR/sigma^2, V = (1-CR) mu/sigma^2,
// X_a = mu(a)/sigma^2; a0, h0, h1: the fixed image's Parzen bins.
template <int DIM>
__device__ __forceinline__ float voxel_dDdB(const Geo& g, int x, int y, int z, int a0, float h0,
                                            float h1, float B, const float* __restrict__ U,
                                            const float* __restrict__ V,
                                            const float* __restrict__ X, float scale) {
  const int nb = g.nbins;
  B = fminf(fmaxf(B, 0.f), (float)(nb - 1));
  float fb;
  const int kb = bin_split(B, nb, &fb);
  const float dm1 = parzen_upper_deriv(fb);
  const float dm2 = (2.f * (float)kb + 1.f) * dm1;
  int sc[3];
  float sw[3][4];
  spatial_weights<DIM>(g, x, y, z, sc, sw);
  float su = 0.f, sv = 0.f;
  const int NZ = DIM == 3 ? 4 : 1;
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < 4; ++j) {
      const float wjk = sw[1][j] * sw[2][k];
      const long long rrow = ((long long)(sc[2] + k) * g.nsb[1] + (sc[1] + j)) * g.nsb[0] + sc[0];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float w = wjk * sw[0][i];
        if (w == 0.f) continue;  // also keeps boxcar reads inside the patch grid
        const long long r = rrow + i;
        const float xr = h0 * __ldg(X + r * nb + a0) + h1 * __ldg(X + r * nb + a0 + 1);
        su += w * __ldg(U + r);
        sv += w * (__ldg(V + r) - xr);
      }
    }
  return scale * (dm2 * su + 2.f * dm1 * sv);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256)
k_adjoint(const Geo g, const T* __restrict__ A, const T* __restrict__ M,
          const float* __restrict__ c, const float* __restrict__ U, const float* __restrict__ V,
          const float* __restrict__ X, const float* __restrict__ gscale, float invZ,
          float* __restrict__ grad) {
  extern __shared__ __align__(16) float gt[];
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  int o[3];
  tile_origin<DIM>(g, blockIdx.x, o);
  const int f0 = o[0] / g.fsp[0], f1 = o[1] / g.fsp[1], f2 = DIM == 3 ? o[2] / g.fsp[2] : 0;
  const int nodes_tile = g.hf[0] * g.hf[1] * g.hf[2];
  const int gsz = DIM * nodes_tile;
  for (int i = threadIdx.x; i < gsz; i += blockDim.x) gt[i] = 0.f;
  __syncthreads();
  const float scale = (gscale ? __ldg(gscale) : 1.f) * invZ;

  const int tv = g.tile[0] * g.tile[1] * g.tile[2];
  for (int v = threadIdx.x; v < tv; v += blockDim.x) {
    const int x = o[0] + v % g.tile[0];
    const int y = o[1] + (v / g.tile[0]) % g.tile[1];
    const int z = o[2] + v / (g.tile[0] * g.tile[1]);
    if (x >= g.n[0] || y >= g.n[1] || z >= g.n[2]) continue;
    const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
    float fa;
    const float av = fminf(fmaxf(ldval(A + idx), 0.f), L);
    const int a0 = bin_split(av, nb, &fa);
    const float h1 = parzen_upper(fa), h0 = 1.f - h1;
    float u[3], bw[3][4], gm[3];
    int fc[3];
    ffd_displacement<DIM>(g, c, x, y, z, u, fc, bw);
    float B = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
    const float G = voxel_dDdB<DIM>(g, x, y, z, a0, h0, h1, B, U, V, X, scale);
    if (G == 0.f) continue;
    const int NZ = DIM == 3 ? 4 : 1;
    float gk[3] = {G * gm[0], G * gm[1], DIM == 3 ? G * gm[2] : 0.f};
    for (int nn = 0; nn < NZ; ++nn)
      for (int m = 0; m < 4; ++m) {
        const float wmn = bw[1][m] * bw[2][nn];
        const int lrow = ((fc[2] - f2 + nn) * g.hf[1] + (fc[1] - f1 + m)) * g.hf[0] + (fc[0] - f0);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float b = wmn * bw[0][l];
#pragma unroll
          for (int k = 0; k < DIM; ++k) atomicAdd(gt + k * nodes_tile + lrow + l, gk[k] * b);
        }
      }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < gsz; i += blockDim.x) {
    const float val = gt[i];
    if (val == 0.f) continue;
    const int k = i / nodes_tile;
    const int nl = i % nodes_tile;
    const int l0 = nl % g.hf[0];
    const int l1 = (nl / g.hf[0]) % g.hf[1];
    const int l2 = nl / (g.hf[0] * g.hf[1]);
    const int n0 = f0 + l0, n1 = f1 + l1, n2 = f2 + l2;
    if (n0 >= g.nf[0] || n1 >= g.nf[1] || n2 >= g.nf[2]) continue;
    atomicAdd(grad + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0, val);
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels: normalisation (Sec. II) and the image pyramid (Sec. II-F).
// ---------------------------------------------------------------------------
__global__ void k_minmax_partial(const float* __restrict__ v, long long n, float* __restrict__ part) {
  __shared__ float smin[256], smax[256];
  float mn = INFINITY, mx = -INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float x = v[i];
    mn = fminf(mn, x);
    mx = fmaxf(mx, x);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + w]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = smin[0];
    part[2 * blockIdx.x + 1] = smax[0];
  }
}

__device__ __forceinline__ void store_val(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_val(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// out = L (v - min) / (max - min) in FP64, rounded to float, then to T.
template <typename T>
__global__ void k_normalise(const float* __restrict__ v, long long n, const float* __restrict__ part,
                            int nparts, double L, T* __restrict__ out) {
  float mn = INFINITY, mx = -INFINITY;
  for (int i = 0; i < nparts; ++i) {
    mn = fminf(mn, part[2 * i]);
    mx = fmaxf(mx, part[2 * i + 1]);
  }
  const double dmn = mn, den = (double)mx - dmn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = L * ((double)v[i] - dmn) / den;
    store_val(out + i, __double2float_rn(r));
  }
}

// Coarser pyramid level: mean of the 2^d children (floor sizes).
template <int DIM, typename T>
__global__ void k_downsample(const T* __restrict__ in, int inx, int iny, T* __restrict__ out,
                             int onx, int ony, int onz) {
  const long long n = (long long)onx * ony * onz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % onx), y = (int)((i / onx) % ony), z = (int)(i / ((long long)onx * ony));
    float s = 0.f;
    const int DZ = DIM == 3 ? 2 : 1;
    for (int dz = 0; dz < DZ; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
          s += ldval(in + ((long long)(2 * z + dz) * iny + (2 * y + dy)) * inx + (2 * x + dx));
    store_val(out + i, s * (DIM == 3 ? 0.125f : 0.25f));
  }
}

// Debug views of what the kernels compute.
template <int DIM, typename T>
__global__ void k_debug_bins(const Geo g, const T* __restrict__ A, int* __restrict__ out) {
  const float L = (float)(g.nbins - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n[0]), y = (int)((i / g.n[0]) % g.n[1]),
              z = (int)(i / ((long long)g.n[0] * g.n[1]));
    int sc[3];
    float sw[3][4];
    spatial_weights<DIM>(g, x, y, z, sc, sw);
    float fa;
    const int a0 = bin_split(fminf(fmaxf(ldval(A + i), 0.f), L), g.nbins, &fa);
    out[4 * i + 0] = sc[0];
    out[4 * i + 1] = sc[1];
    out[4 * i + 2] = sc[2];
    out[4 * i + 3] = a0;
  }
}

// B(x) = M(T(x)) per voxel; with out4 != NULL, (B, dM/dy_x, dM/dy_y, dM/dy_z)
// per voxel instead.
template <int DIM, typename T>
__global__ void k_debug_warp(const Geo g, const T* __restrict__ M, const float* __restrict__ c,
                             float* __restrict__ out, float4* __restrict__ out4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n[0]), y = (int)((i / g.n[0]) % g.n[1]),
              z = (int)(i / ((long long)g.n[0] * g.n[1]));
    float u[3], bw[3][4], gm[3];
    int fc[3];
    ffd_displacement<DIM>(g, c, x, y, z, u, fc, bw);
    const float B = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
    if (out4) out4[i] = make_float4(B, gm[0], gm[1], gm[2]);
    else out[i] = B;
  }
}

// Storage-type image to float32.
template <typename T>
__global__ void k_to_float(const T* __restrict__ in, long long n, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ldval(in + i);
}

// The fixed-point conversions of the histogram flushes on n floats v and on
// m word pairs (hi, lo); reference != 0 takes CUDA's 64-bit conversions
// instead, the values the 32-bit forms must reproduce.
__global__ void k_debug_fixed(const float* __restrict__ v, long long n, const unsigned* __restrict__ hi,
                              const unsigned* __restrict__ lo, long long m,
                              unsigned long long* __restrict__ fixed, float* __restrict__ flt,
                              int reference) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    fixed[i] = reference ? __float2ull_rn(v[i]) : fixed_from_float(v[i]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += stride)
    flt[i] = reference ? __ull2float_rn(((unsigned long long)hi[i] << 24) + lo[i])
                       : fields_to_float(hi[i], lo[i]);
}

}  // namespace srwcr
