// Device arithmetic shared by the SRWCR kernels (sm_103a).
//
// Each helper restates one definition of Gong et al. (arXiv 1804.05061):
//   bspline4        Eq. (8), the four uniform cubic B-spline pieces
//   parzen_upper    Eq. (5) on its two active bins: for v = k + f the window
//                   puts h(f) on bin k and h(1-f) on bin k+1
//   Grid            the integer cell / fraction arithmetic of Eq. (17) (FFD)
//   SBins           the same for the spatial distribution of Eq. (7), with a
//                   rational spacing num/den so cell indices are exact
//   sample_moving   backward warping (Sec. II-F): trilinear, clamp-to-border,
//                   analytic gradient of the interpolant
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace srwcr {

// Problem geometry of one pyramid level, passed by value to every kernel.
struct Geo {
  int n[3];       // voxels per axis (n[2] = 1 in 2-D)
  int fsp[3];     // FFD control spacing delta (voxels)
  int nf[3];      // FFD nodes per axis (1 for an absent axis)
  int sbn[3];     // spatial-bin spacing numerator   (spacing = sbn/sbd)
  int sbd[3];     // spatial-bin spacing denominator
  int nsb[3];     // spatial bins per axis
  int nbins;      // intensity bins L_eps + 1
  int tile[3];    // voxel tile of one CTA
  int ntile[3];   // tiles per axis
  int hb[3];      // max spatial bins a tile touches, per axis
  int hf[3];      // max FFD nodes a tile touches, per axis
  long long nvox;
  long long ncoef;  // nodes per component = nf[0]*nf[1]*nf[2]
  long long R;      // spatial bins = nsb[0]*nsb[1]*nsb[2]
  int nabin;        // row kernels: most fixed-image bins any one tile uses
  int cbin;         // row kernels: compacted bins per pass of the value kernel
  int boxcar;       // spatial distribution: 0 cubic B-spline (Eq. 7), 1 boxcar (Eq. 6)
};

__device__ __forceinline__ float ldval(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldval(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }

// Fixed-point conversions done with 32-bit operations only: conversions
// between 64-bit integers and floats run on the narrow FP64 unit of this
// GPU, and a histogram flush issues one per entry.
//
// Nearest 64-bit integer to v, 0 <= v < 2^64 (ties to even), the value
// __float2ull_rn returns.  hf = floor(v / 2^32) is exact (power-of-two
// scaling, then floor); v - hf 2^32 is exact in the FMA and lies in
// [0, 2^32); below 2^32 the conversion rounds the fraction of v, from 2^32
// up v is a multiple of 2^9 and the remainder an integer.
__device__ __forceinline__ unsigned long long fixed_from_float(float v) {
  const float hf = floorf(v * 0x1p-32f);
  const unsigned lo = __float2uint_rn(fmaf(hf, -0x1p32f, v));
  return ((unsigned long long)__float2uint_rz(hf) << 32) | lo;
}

// Nearest float to hi 2^24 + lo for hi <= 256 (2^24 - 1) and lo < 2^32 (a
// 48-bit histogram word pair), the value __ull2float_rn returns for that
// sum.  After the carry of lo's top byte into hi the sum is hn 2^24 + l with
// l < 2^24; below 2^48 (hn < 2^24) both halves are exact floats and the FMA
// rounds their exact sum once.  Larger sums take the 64-bit conversion.
__device__ __forceinline__ float fields_to_float(unsigned hi, unsigned lo) {
  const unsigned hn = hi + (lo >> 24);
  if (hn < (1u << 24)) return fmaf((float)hn, 0x1p24f, (float)(lo & 0xffffffu));
  return __ull2float_rn(((unsigned long long)hi << 24) + lo);
}

// Eq. (8): w[l] = beta_l(t), t in [0, 1].
__device__ __forceinline__ void bspline4(float t, float w[4]) {
  const float s = 1.0f / 6.0f;
  const float t2 = t * t, t3 = t2 * t, u = 1.0f - t;
  w[0] = u * u * u * s;
  w[1] = (3.0f * t3 - 6.0f * t2 + 4.0f) * s;
  w[2] = (-3.0f * t3 + 3.0f * t2 + 3.0f * t + 1.0f) * s;
  w[3] = t3 * s;
}

// Eq. (5) at 1 - f: the weight the window gives bin k+1 for v = k + f.
__device__ __forceinline__ float parzen_upper(float f) {
  const float g = 1.0f - f;
  return f < 0.5f ? f * (1.8f * f + 0.1f) : 1.0f - g * (1.8f * g + 0.1f);
}

// d/df of parzen_upper (one-sided inside [0, 1]; Eq. 19's dh/dkappa).
__device__ __forceinline__ float parzen_upper_deriv(float f) {
  return f < 0.5f ? 3.6f * f + 0.1f : 3.6f * (1.0f - f) + 0.1f;
}

// Split v in [0, L] into bin k = min(floor(v), L-1) and f = v - k in [0, 1].
__device__ __forceinline__ int bin_split(float v, int nbins, float* f) {
  int k = (int)floorf(v);
  k = k < 0 ? 0 : (k > nbins - 2 ? nbins - 2 : k);
  *f = v - (float)k;
  return k;
}

// Spatial-bin cell of voxel coordinate x along axis d: floor(x*den/num).
__device__ __forceinline__ int sb_cell(const Geo& g, int d, int x, float* t) {
  const int q = x * g.sbd[d];
  const int c = q / g.sbn[d];
  *t = (float)(q - c * g.sbn[d]) / (float)g.sbn[d];
  return c;
}

// FFD cell of x along axis d: floor(x/delta), eta = (x mod delta)/delta.
__device__ __forceinline__ int ffd_cell(const Geo& g, int d, int x, float* t) {
  const int c = x / g.fsp[d];
  *t = (float)(x - c * g.fsp[d]) / (float)g.fsp[d];
  return c;
}

// FFD displacement u(x) = sum beta_l beta_m beta_n c_k[node] (Eqs. 1, 17);
// coefficients read from global memory through the read-only path.
template <int DIM>
__device__ __forceinline__ void ffd_displacement(const Geo& g, const float* __restrict__ c, int x,
                                                 int y, int z, float u[3], int fc[3],
                                                 float bw[3][4]) {
  float t;
  fc[0] = ffd_cell(g, 0, x, &t); bspline4(t, bw[0]);
  fc[1] = ffd_cell(g, 1, y, &t); bspline4(t, bw[1]);
  if (DIM == 3) { fc[2] = ffd_cell(g, 2, z, &t); bspline4(t, bw[2]); }
  else { fc[2] = 0; bw[2][0] = 1.f; bw[2][1] = bw[2][2] = bw[2][3] = 0.f; }
  u[0] = u[1] = u[2] = 0.f;
  const int NZ = DIM == 3 ? 4 : 1;
  for (int nn = 0; nn < NZ; ++nn) {
    for (int m = 0; m < 4; ++m) {
      const float wyz = bw[1][m] * bw[2][nn];
      const long long row = ((long long)(fc[2] + nn) * g.nf[1] + (fc[1] + m)) * g.nf[0] + fc[0];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const float* cr = c + k * g.ncoef + row;
        const float s = bw[0][0] * __ldg(cr) + bw[0][1] * __ldg(cr + 1) +
                        bw[0][2] * __ldg(cr + 2) + bw[0][3] * __ldg(cr + 3);
        u[k] += wyz * s;
      }
    }
  }
}

// Backward warping (Sec. II-F): B = M(y) by trilinear interpolation with the
// coordinate clamped to [0, N-1] per axis, and the analytic gradient of the
// interpolant (zero along an axis where y left the domain).  The cell is
// [floor(y), floor(y)+1], or [N-2, N-1] at y = N-1.
template <int DIM, typename T>
__device__ __forceinline__ float sample_moving(const Geo& g, const T* __restrict__ M, float yx,
                                               float yy, float yz, float grad[3]) {
  float yv[3] = {yx, yy, yz}, t[3];
  int i0[3];
  bool in[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const float hi = (float)(g.n[d] - 1);
    float v = yv[d];
    in[d] = true;
    if (!(v >= 0.f)) { v = 0.f; in[d] = false; }   // also catches NaN
    if (v > hi) { v = hi; in[d] = false; }
    int f = (int)floorf(v);
    if (f > g.n[d] - 2) f = g.n[d] - 2;
    i0[d] = f;
    t[d] = v - (float)f;
  }
  const long long sx = 1, sy = g.n[0];
  if (DIM == 2) {
    const T* p = M + (long long)i0[1] * sy + i0[0];
    const float m00 = ldval(p), m10 = ldval(p + sx), m01 = ldval(p + sy), m11 = ldval(p + sy + sx);
    const float a0 = m00 + t[0] * (m10 - m00), a1 = m01 + t[0] * (m11 - m01);
    grad[0] = in[0] ? (m10 - m00) * (1.f - t[1]) + (m11 - m01) * t[1] : 0.f;
    grad[1] = in[1] ? a1 - a0 : 0.f;
    grad[2] = 0.f;
    return a0 + t[1] * (a1 - a0);
  }
  const long long sz = (long long)g.n[0] * g.n[1];
  const T* p = M + (long long)i0[2] * sz + (long long)i0[1] * sy + i0[0];
  const float m000 = ldval(p), m100 = ldval(p + sx), m010 = ldval(p + sy), m110 = ldval(p + sy + sx);
  const float m001 = ldval(p + sz), m101 = ldval(p + sz + sx), m011 = ldval(p + sz + sy),
              m111 = ldval(p + sz + sy + sx);
  const float c00 = m000 + t[0] * (m100 - m000), c10 = m010 + t[0] * (m110 - m010);
  const float c01 = m001 + t[0] * (m101 - m001), c11 = m011 + t[0] * (m111 - m011);
  const float e0 = c00 + t[1] * (c10 - c00), e1 = c01 + t[1] * (c11 - c01);
  if (in[0]) {
    const float d0 = (m100 - m000) + t[1] * ((m110 - m010) - (m100 - m000));
    const float d1 = (m101 - m001) + t[1] * ((m111 - m011) - (m101 - m001));
    grad[0] = d0 + t[2] * (d1 - d0);
  } else {
    grad[0] = 0.f;
  }
  grad[1] = in[1] ? (c10 - c00) + t[2] * ((c11 - c01) - (c10 - c00)) : 0.f;
  grad[2] = in[2] ? e1 - e0 : 0.f;
  return e0 + t[2] * (e1 - e0);
}

// Spatial distribution at voxel (x, y, z): cells and per-axis weights; the
// voxel lies in bins cell+i, i = 0..3, per axis.  Eq. (7): cubic B-spline
// weights.  Eq. (6) (g.boxcar): the patch floor(x K / N) with weight 1 and
// zero weight for i > 0 (those bins may lie past the last patch: callers
// skip zero weights before touching a bin).
__device__ __forceinline__ void axis_weights(const Geo& g, int d, int x, int* sc, float w[4]) {
  float t;
  *sc = sb_cell(g, d, x, &t);
  if (g.boxcar) {
    w[0] = 1.f; w[1] = w[2] = w[3] = 0.f;
  } else {
    bspline4(t, w);
  }
}

template <int DIM>
__device__ __forceinline__ void spatial_weights(const Geo& g, int x, int y, int z, int sc[3],
                                                float sw[3][4]) {
  axis_weights(g, 0, x, &sc[0], sw[0]);
  axis_weights(g, 1, y, &sc[1], sw[1]);
  if (DIM == 3) axis_weights(g, 2, z, &sc[2], sw[2]);
  else { sc[2] = 0; sw[2][0] = 1.f; sw[2][1] = sw[2][2] = sw[2][3] = 0.f; }
}

// Rigid model (the pre-alignment of Sec. III-D with the same measure):
// T(x) = R (x - x_c) + x_c + t.  The per-evaluation table (built in FP64 by
// k_rigid_setup from the parameters) holds R row-major [0, 9), t [9, 12),
// x_c [12, 15) and dR/d(angle) for up to three angles [15, 42).
constexpr int kRigidTab = 48;

struct Rigid {
  float R[9];
  float t[3];
  float ctr[3];
};

__device__ __forceinline__ Rigid load_rigid(const float* __restrict__ tab) {
  Rigid r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.R[i] = __ldg(tab + i);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.t[i] = __ldg(tab + 9 + i);
    r.ctr[i] = __ldg(tab + 12 + i);
  }
  return r;
}

// u = T(x) - x for voxel (x, y, z).
template <int DIM>
__device__ __forceinline__ void rigid_displacement(const Rigid& r, int x, int y, int z, float u[3]) {
  const float q0 = (float)x - r.ctr[0], q1 = (float)y - r.ctr[1];
  const float q2 = DIM == 3 ? (float)z - r.ctr[2] : 0.f;
  const float xv[3] = {(float)x, (float)y, (float)z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k >= DIM) { u[k] = 0.f; continue; }
    const float rq = fmaf(r.R[3 * k], q0, fmaf(r.R[3 * k + 1], q1, r.R[3 * k + 2] * q2));
    u[k] = (rq + r.ctr[k] + r.t[k]) - xv[k];
  }
}

}  // namespace srwcr
