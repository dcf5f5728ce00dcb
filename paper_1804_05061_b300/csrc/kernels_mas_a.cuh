// Moving image as the model image A (Sec. II-E, Eqs. 20, 21): general
// per-voxel kernels.  The warped moving image A(x) = M(T(x)) is binned by
// the Parzen window of Eq. (5) (bins a0, a0+1, weights h0, h1) and the fixed
// image F is the estimated image B, whose Parzen moments
// m1 = sum_b b h(b - F), m2 = sum_b b^2 h(b - F) do not change.  Because the
// binned image moves, p_r(a) is accumulated at every evaluation: three
// fixed-point channels per (region, bin), P = sum w h, S1 = sum w h m1,
// S2 = sum w h m2.  The value and the per-region finalisation then follow
// Eqs. (9), (10) exactly as with M as B; the gradient is Eq. (21).
#pragma once

#include "kernels.cuh"

namespace srwcr {

// Parzen moments of an intensity v in [0, L] (bins k, k+1; Eq. 5).
__device__ __forceinline__ void parzen_moments(float v, int nb, float* m1, float* m2) {
  float f;
  const int k = bin_split(v, nb, &f);
  const float w1 = parzen_upper(f), kf = (float)k;
  *m1 = kf + w1;
  *m2 = kf * kf + (2.f * kf + 1.f) * w1;
}

// (a) with M as A.  Histogram in shared memory: [hb2][hb1][hb0][nbins][3]
// u64; global accumulators [R][nbins][3] (fixed point, scales s0, s1, s2).
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
k_accumulate_mas_a(const Geo g, const T* __restrict__ F, const T* __restrict__ M,
                   const float* __restrict__ c, unsigned long long* __restrict__ acc, float s0,
                   float s1, float s2) {
  extern __shared__ __align__(16) unsigned long long hist[];
  constexpr int NCH = 3;
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
    float u[3], bw[3][4], gm[3];
    int fc[3];
    ffd_displacement<DIM>(g, c, x, y, z, u, fc, bw);
    float Av = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
    Av = fminf(fmaxf(Av, 0.f), L);
    float fa;
    const int a0 = bin_split(Av, nb, &fa);
    const float h1 = parzen_upper(fa), h0 = 1.f - h1;
    float m1, m2;
    parzen_moments(fminf(fmaxf(ldval(F + idx), 0.f), L), nb, &m1, &m2);
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
          if (wa0 != 0.f) {
            shared_add_u64(hp + 3 * a0, to_fixed(wa0 * s0));
            shared_add_u64(hp + 3 * a0 + 1, to_fixed(wa0 * m1 * s1));
            shared_add_u64(hp + 3 * a0 + 2, to_fixed(wa0 * m2 * s2));
          }
          if (wa1 != 0.f) {
            shared_add_u64(hp + 3 * a0 + 3, to_fixed(wa1 * s0));
            shared_add_u64(hp + 3 * a0 + 4, to_fixed(wa1 * m1 * s1));
            shared_add_u64(hp + 3 * a0 + 5, to_fixed(wa1 * m2 * s2));
          }
        }
      }
  }
  __syncthreads();
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

// (b) with M as A, one warp per region, FP64: W_r = sum_a P, T1, T2 and
// sigma_r^2 of F in the region, Q_r = sum_{a: P > 0} (S2 - S1^2/P), share
// Q_r / (Z sigma_r^2) (Eq. 9), and the gradient tables
// Y1[r][a] = mu_r(a) / sigma_r^2, Y2[r][a] = mu_r(a)^2 / sigma_r^2
// (mu_r(a) = S1/P; 0 for an empty bin or a degenerate region), with their
// bin-to-bin differences DY[r][a] = (Y2[a+1] - Y2[a], Y1[a+1] - Y1[a]) in
// FP32 for the adjoint (one 8-byte load per spatial bin instead of four).
__global__ void __launch_bounds__(256)
k_finalize_mas_a(const Geo g, const unsigned long long* __restrict__ S, double inv_s0,
                 double inv_s1, double inv_s2, double invZ, float* __restrict__ Y1,
                 float* __restrict__ Y2, float2* __restrict__ DY, double* __restrict__ Dr,
                 double* __restrict__ stats) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (r >= g.R) return;  // warp-uniform
  const int lane = threadIdx.x & 31, nb = g.nbins;
  const unsigned long long* Sr = S + r * nb * 3;
  double W = 0.0, T1 = 0.0, T2 = 0.0;
  for (int a = lane; a < nb; a += 32) {
    W += (double)Sr[3 * a] * inv_s0;
    T1 += (double)Sr[3 * a + 1] * inv_s1;
    T2 += (double)Sr[3 * a + 2] * inv_s2;
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
  const double iv = valid ? 1.0 / var : 0.0;
  double Q = 0.0;
  for (int a = lane; a < nb; a += 32) {
    const unsigned long long p = Sr[3 * a];
    double y1 = 0.0, y2 = 0.0;
    if (valid && p != 0ull) {
      const double P = (double)p * inv_s0, s1 = (double)Sr[3 * a + 1] * inv_s1,
                   s2 = (double)Sr[3 * a + 2] * inv_s2;
      const double m = s1 / P;
      Q += s2 - s1 * m;
      y1 = m * iv;
      y2 = m * m * iv;
    }
    Y1[r * nb + a] = (float)y1;
    Y2[r * nb + a] = (float)y2;
  }
  __syncwarp();
  for (int a = lane; a < nb - 1; a += 32)
    DY[r * nb + a] = make_float2(Y2[r * nb + a + 1] - Y2[r * nb + a],
                                 Y1[r * nb + a + 1] - Y1[r * nb + a]);
#pragma unroll
  for (int off = 16; off; off >>= 1) Q += __shfl_xor_sync(0xffffffffu, Q, off);
  if (lane == 0) {
    const double omc = valid ? Q * iv / W : 0.0, share = valid ? Q * invZ * iv : 0.0;
    Dr[r] = share;
    stats[4 * r + 0] = W * invZ;
    stats[4 * r + 1] = valid ? var : 0.0;
    stats[4 * r + 2] = valid ? 1.0 - omc : 0.0;
    stats[4 * r + 3] = share;
  }
}

// (c) with M as A: per voxel, Eq. (21) on the two active bins of A(x):
//   G(x) = (h1'(f)/Z) sum_r w_r [(Y2[r][a0+1] - Y2[r][a0])
//                                - 2 m1(F(x)) (Y1[r][a0+1] - Y1[r][a0])]
// (the differences read from DY),
// h1' = d/df of the upper-bin weight (the in-cell Parzen derivative), then
//   g[k][node] += G(x) dM/dy_k(T(x)) beta(node; x)                 (Eqs. 16, 17)
// through a CTA-private tile of control points.
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
k_adjoint_mas_a(const Geo g, const T* __restrict__ F, const T* __restrict__ M,
                const float* __restrict__ c, const float2* __restrict__ DY,
                const float* __restrict__ gscale, float invZ, float* __restrict__ grad) {
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
    float u[3], bw[3][4], gm[3];
    int fc[3];
    ffd_displacement<DIM>(g, c, x, y, z, u, fc, bw);
    float Av = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1], (float)z + u[2], gm);
    Av = fminf(fmaxf(Av, 0.f), L);
    float fa;
    const int a0 = bin_split(Av, nb, &fa);
    const float dh = parzen_upper_deriv(fa);
    float m1, m2;
    parzen_moments(fminf(fmaxf(ldval(F + idx), 0.f), L), nb, &m1, &m2);
    int sc[3];
    float sw[3][4];
    spatial_weights<DIM>(g, x, y, z, sc, sw);
    float s = 0.f;
    const int NZ = DIM == 3 ? 4 : 1;
    for (int k = 0; k < NZ; ++k)
      for (int j = 0; j < 4; ++j) {
        const float wjk = sw[1][j] * sw[2][k];
        const long long rrow = ((long long)(sc[2] + k) * g.nsb[1] + (sc[1] + j)) * g.nsb[0] + sc[0];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float w = wjk * sw[0][i];
          if (w == 0.f) continue;  // also keeps boxcar reads inside the patch grid
          const float2 d = __ldg(DY + (rrow + i) * nb + a0);   // a0 <= nb - 2
          s += w * (d.x - 2.f * m1 * d.y);
        }
      }
    const float G = scale * dh * s;
    if (G == 0.f) continue;
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
    const int n0 = f0 + nl % g.hf[0], n1 = f1 + (nl / g.hf[0]) % g.hf[1],
              n2 = f2 + nl / (g.hf[0] * g.hf[1]);
    if (n0 >= g.nf[0] || n1 >= g.nf[1] || n2 >= g.nf[2]) continue;
    atomicAdd(grad + k * g.ncoef + ((long long)n2 * g.nf[1] + n1) * g.nf[0] + n0, val);
  }
}

}  // namespace srwcr
