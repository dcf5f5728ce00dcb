// Rigid model (the pre-alignment of Sec. III-D, with the same measure):
//   T(x) = R (x - x_c) + x_c + t,  x_c = (N - 1) / 2 per axis (voxel units),
// 3-D parameters (t_x, t_y, t_z, alpha, beta, gamma), R = Rz(gamma) Ry(beta)
// Rx(alpha); 2-D (t_x, t_y, theta).  The value pass is k_accumulate<RIGID>;
// the gradient is Eq. (16) with dT/dmu in place of the FFD basis:
//   dD/dmu_i = sum_x dD/dB(x) grad M(T(x)) . dT/dmu_i(x),
// dT/dt_k = e_k, dT/d(angle) = (dR/d(angle)) (x - x_c), reduced per CTA and
// added to FP64 accumulators.
#pragma once

#include "kernels.cuh"

namespace srwcr {

__host__ __device__ inline void rot3(int axis, double a, double d, double out[3][3]) {
  // Elementary rotation about `axis` by a (d = 0) or its derivative (d = 1).
  const double c = cos(a), s = sin(a);
  const double cc = d ? -s : c, ss = d ? c : s, one = d ? 0.0 : 1.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[i][j] = 0.0;
  const int i0 = (axis + 1) % 3, i1 = (axis + 2) % 3;
  out[axis][axis] = one;
  out[i0][i0] = cc;
  out[i0][i1] = -ss;
  out[i1][i0] = ss;
  out[i1][i1] = cc;
}

__host__ __device__ inline void mul3(const double a[3][3], const double b[3][3], double o[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      o[i][j] = s;
    }
}

// Builds the rigid table from mu (angles = mu_angle * ang_scale) in FP64.
// One thread.  The rotation about y (axis 1) in the cyclic form above is
// [[c, 0, s], [0, 1, 0], [-s, 0, c]], as are the ones about x and z.
__global__ void k_rigid_setup(const float* __restrict__ mu, int ndim, double cx, double cy,
                              double cz, double ang_scale, float* __restrict__ tab) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[3][3], dR[3][3][3];
  const int na = ndim == 3 ? 3 : 1;
  if (ndim == 3) {
    const double ang[3] = {mu[3] * ang_scale, mu[4] * ang_scale, mu[5] * ang_scale};
    double E[3][3][3], D[3][3][3], t1[3][3];
    for (int a = 0; a < 3; ++a) {
      rot3(a, ang[a], 0.0, E[a]);
      rot3(a, ang[a], 1.0, D[a]);
    }
    mul3(E[1], E[0], t1);
    mul3(E[2], t1, R);                 // Rz Ry Rx
    mul3(E[1], D[0], t1);
    mul3(E[2], t1, dR[0]);             // Rz Ry dRx
    mul3(D[1], E[0], t1);
    mul3(E[2], t1, dR[1]);             // Rz dRy Rx
    mul3(E[1], E[0], t1);
    mul3(D[2], t1, dR[2]);             // dRz Ry Rx
  } else {
    rot3(2, mu[2] * ang_scale, 0.0, R);
    rot3(2, mu[2] * ang_scale, 1.0, dR[0]);
    R[2][2] = 1.0;
    dR[0][2][2] = 0.0;
  }
  for (int i = 0; i < 9; ++i) tab[i] = (float)R[i / 3][i % 3];
  for (int k = 0; k < 3; ++k) tab[9 + k] = k < ndim ? mu[k] : 0.f;
  tab[12] = (float)cx;
  tab[13] = (float)cy;
  tab[14] = (float)cz;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < 9; ++i) tab[15 + 9 * a + i] = a < na ? (float)dR[a][i / 3][i % 3] : 0.f;
}

// dD/dmu summed over the CTA's tile into acc (FP64, NP = 6 or 3 entries).
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
k_adjoint_rigid(const Geo g, const T* __restrict__ A, const T* __restrict__ M,
                const float* __restrict__ tab, const float* __restrict__ U,
                const float* __restrict__ V, const float* __restrict__ X,
                const float* __restrict__ gscale, float invZ, double* __restrict__ acc) {
  constexpr int NA = DIM == 3 ? 3 : 1;  // angles
  constexpr int NP = DIM + NA;
  __shared__ float red[8][NP];
  const Rigid rg = load_rigid(tab);
  float dR[NA][9];
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int i = 0; i < 9; ++i) dR[a][i] = __ldg(tab + 15 + 9 * a + i);
  const int nb = g.nbins;
  const float L = (float)(nb - 1);
  int o[3];
  tile_origin<DIM>(g, blockIdx.x, o);
  const float scale = (gscale ? __ldg(gscale) : 1.f) * invZ;
  float part[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) part[i] = 0.f;

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
    float u[3], gm[3];
    rigid_displacement<DIM>(rg, x, y, z, u);
    const float B = sample_moving<DIM, T>(g, M, (float)x + u[0], (float)y + u[1],
                                          (float)z + u[2], gm);
    const float G = voxel_dDdB<DIM>(g, x, y, z, a0, h0, h1, B, U, V, X, scale);
    if (G == 0.f) continue;
    const float q[3] = {(float)x - rg.ctr[0], (float)y - rg.ctr[1],
                        DIM == 3 ? (float)z - rg.ctr[2] : 0.f};
#pragma unroll
    for (int k = 0; k < DIM; ++k) part[k] = fmaf(G, gm[k], part[k]);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        s = fmaf(gm[k], fmaf(dR[a][3 * k], q[0], fmaf(dR[a][3 * k + 1], q[1], dR[a][3 * k + 2] * q[2])), s);
      part[DIM + a] = fmaf(G, s, part[DIM + a]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float s = part[i];
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)red[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, s);
  }
}

// g_i = acc_i, the angle entries times ang_scale (d/d mu of angle = mu * ang_scale).
__global__ void k_rigid_grad_out(const double* __restrict__ acc, int ndim, double ang_scale,
                                 float* __restrict__ g) {
  const int np = ndim == 3 ? 6 : 3;
  const int i = threadIdx.x;
  if (i < np) g[i] = (float)(i < ndim ? acc[i] : acc[i] * ang_scale);
}

// FFD coefficients equal to the rigid displacement at the control nodes
// (node j of an axis at (j - 1) delta); the cubic B-spline reproduces an
// affine field exactly, so the FFD warp equals the rigid one.
__global__ void k_rigid_to_ffd(const Geo g, int ndim, const float* __restrict__ tab,
                               float* __restrict__ c) {
  const long long n = g.ncoef;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int j0 = (int)(i % g.nf[0]);
    const int j1 = (int)((i / g.nf[0]) % g.nf[1]);
    const int j2 = (int)(i / ((long long)g.nf[0] * g.nf[1]));
    const double p[3] = {(double)(j0 - 1) * g.fsp[0], (double)(j1 - 1) * g.fsp[1],
                         ndim == 3 ? (double)(j2 - 1) * g.fsp[2] : 0.0};
    const double q[3] = {p[0] - tab[12], p[1] - tab[13], ndim == 3 ? p[2] - tab[14] : 0.0};
    for (int k = 0; k < ndim; ++k) {
      const double rq = (double)tab[3 * k] * q[0] + (double)tab[3 * k + 1] * q[1] +
                        (double)tab[3 * k + 2] * q[2];
      c[k * n + i] = (float)(rq + tab[12 + k] + tab[9 + k] - p[k]);
    }
  }
}

// Chain rule through the FFD form of a rigid transform: with c_j =
// R (p_j - x_c) + x_c + t - p_j at node j, dD/dt_k = sum_j g[k][j] and
// dD/d(angle) = sum_j sum_k g[k][j] ((dR/d(angle)) (p_j - x_c))_k, reduced
// per CTA into acc (FP64).  256 threads per CTA.
template <int DIM>
__global__ void __launch_bounds__(256)
k_rigid_chain(const Geo g, const float* __restrict__ tab, const float* __restrict__ grad,
              double* __restrict__ acc) {
  constexpr int NA = DIM == 3 ? 3 : 1;
  constexpr int NP = DIM + NA;
  __shared__ float red[8][NP];
  float part[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) part[i] = 0.f;
  const long long n = g.ncoef;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int j0 = (int)(i % g.nf[0]);
    const int j1 = (int)((i / g.nf[0]) % g.nf[1]);
    const int j2 = (int)(i / ((long long)g.nf[0] * g.nf[1]));
    const float q[3] = {(float)((j0 - 1) * g.fsp[0]) - __ldg(tab + 12),
                        (float)((j1 - 1) * g.fsp[1]) - __ldg(tab + 13),
                        DIM == 3 ? (float)((j2 - 1) * g.fsp[2]) - __ldg(tab + 14) : 0.f};
    float gk[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      gk[k] = __ldg(grad + k * n + i);
      part[k] += gk[k];
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const float* dR = tab + 15 + 9 * a;
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        s = fmaf(gk[k], fmaf(__ldg(dR + 3 * k), q[0], fmaf(__ldg(dR + 3 * k + 1), q[1], __ldg(dR + 3 * k + 2) * q[2])), s);
      part[DIM + a] += s;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float s = part[i];
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += (double)red[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, s);
  }
}

}  // namespace srwcr
