// Bending energy C_p of the FFD displacement, the penalty term of Eq. (1)
// (Sec. II-F): the thin-plate bending energy averaged over the image box
// Omega = prod_d [0, N_d - 1] (voxel units),
//
//   C_p = 1/|Omega| * int_Omega sum_k sum_{i,j} (d^2 u_k / dx_i dx_j)^2 dx,
//
// over ordered pairs (i, j).  u is a tensor-product cubic B-spline, so C_p is
// a quadratic form c_k' K c_k with K a sum of Kronecker products of 1-D Gram
// matrices G_a[i][j] = int_0^{N-1} beta_i^(a) beta_j^(a) dx (a = 0, 1, 2
// derivatives; banded, |i - j| <= 3):
//   3-D: K = G2x G0y G0z + G0x G2y G0z + G0x G0y G2z
//            + 2 (G1x G1y G0z + G1x G0y G1z + G0x G1y G1z)
//   2-D: K = G2x G0y + G0x G2y + 2 G1x G1y.
// The Gram entries are integrated exactly on the host (4-point
// Gauss-Legendre per knot interval; the integrands are polynomials of degree
// <= 6); K c is applied on the device as separable 7-tap stencils along z, y
// and x, and C_p = c . K c / |Omega| is summed in FP64; dC_p/dc = 2 K c /
// |Omega|.  Included once, at the end of srwcr.cu (after lbfgs.cuh).
#pragma once

namespace {

// Uniform cubic B-spline piece l (Eq. 8) and its t-derivatives.
double bs_piece(int l, double t, int order) {
  const double u = 1.0 - t;
  switch (order) {
    case 0:
      return l == 0 ? u * u * u / 6.0
           : l == 1 ? (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0
           : l == 2 ? (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0
                    : t * t * t / 6.0;
    case 1:
      return l == 0 ? -0.5 * u * u
           : l == 1 ? 1.5 * t * t - 2.0 * t
           : l == 2 ? -1.5 * t * t + t + 0.5
                    : 0.5 * t * t;
    default:
      return l == 0 ? u : l == 1 ? 3.0 * t - 2.0 : l == 2 ? 1.0 - 3.0 * t : t;
  }
}

// Diagonals of the three Gram matrices of one axis: out[a][i][t + 3] =
// G_a[i][i + t], node j at (j - 1) delta, derivatives in voxel units.
void gram_diagonals(int n, int delta, int nodes, std::vector<float>& out) {
  static const double gx[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563,
                               0.8611363115940526};
  static const double gw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461,
                               0.3478548451374538};
  std::vector<double> G(3 * (size_t)nodes * 7, 0.0);
  for (int p = 0; (long long)p * delta < n - 1; ++p) {
    const double a = (double)p * delta, b = std::min((double)(p + 1) * delta, (double)(n - 1));
    for (int q = 0; q < 4; ++q) {
      const double x = 0.5 * (b - a) * gx[q] + 0.5 * (a + b), w = 0.5 * (b - a) * gw[q];
      const double t = x / delta - p;
      for (int ord = 0; ord < 3; ++ord) {
        const double sc = std::pow((double)delta, -ord);
        for (int l = 0; l < 4; ++l)
          for (int m = 0; m < 4; ++m) {
            const int i = p + l, tt = m - l;
            G[((size_t)ord * nodes + i) * 7 + tt + 3] +=
                w * bs_piece(l, t, ord) * sc * bs_piece(m, t, ord) * sc;
          }
      }
    }
  }
  out.assign(G.begin(), G.end());
}

// out (+)= alpha * (G applied along `axis`) in, for `ncomp` components of an
// (nx, ny, nz) node grid, G given by its 7 diagonals per node.
__global__ void __launch_bounds__(256)
k_band_axis(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ diag,
            int axis, int nx, int ny, int nz, int ncomp, float alpha, int accumulate) {
  const long long per = (long long)nx * ny * nz, total = per * ncomp;
  const int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < total; e += (long long)gridDim.x * 256) {
    const long long r = e % per;
    const int i = (int)((r / stride) % n_axis);
    const float* dg = diag + (size_t)i * 7;
    float s = 0.f;
#pragma unroll
    for (int t = -3; t <= 3; ++t) {
      const int j = i + t;
      if (j < 0 || j >= n_axis) continue;
      s += dg[t + 3] * in[e + t * stride];
    }
    out[e] = accumulate ? out[e] + alpha * s : alpha * s;
  }
}

struct BendWork {
  long long n = 0;
  float* buf = nullptr;    // 7 arrays of n: Z0 Z1 Z2 T1 T2 T3 OUT
  float* diag = nullptr;   // per axis d: [3][nodes_d][7]
  size_t diag_off[3] = {0, 0, 0};
  double* part = nullptr;  // dot partials
  double inv_vol = 0.0;
};

}  // namespace

struct srwcr_bend_levels {
  BendWork w[4];
};

namespace {

srwcr_status bend_setup(srwcr_ctx* ctx, int level, BendWork& bw) {
  if (bw.buf) return SRWCR_OK;
  const Geo& g = ctx->lev[level].g;
  const int nd = ctx->cfg.ndim;
  bw.n = g.ncoef * nd;
  std::vector<float> all;
  double vol = 1.0;
  for (int d = 0; d < nd; ++d) {
    std::vector<float> dg;
    gram_diagonals(g.n[d], g.fsp[d], g.nf[d], dg);
    bw.diag_off[d] = all.size();
    all.insert(all.end(), dg.begin(), dg.end());
    vol *= (double)(g.n[d] - 1);
  }
  bw.inv_vol = 1.0 / vol;
  CK(cudaMalloc((void**)&bw.buf, sizeof(float) * bw.n * 7));
  CK(cudaMalloc((void**)&bw.diag, sizeof(float) * all.size()));
  CK(cudaMalloc((void**)&bw.part, sizeof(double) * kDotBlocks));
  CK(cudaMemcpy(bw.diag, all.data(), sizeof(float) * all.size(), cudaMemcpyHostToDevice));
  return SRWCR_OK;
}

// OUT = K c (all components); returns its device pointer.
srwcr_status bend_apply(srwcr_ctx* ctx, int level, BendWork& bw, const float* c, float** out) {
  const Geo& g = ctx->lev[level].g;
  const int nd = ctx->cfg.ndim;
  const long long n = bw.n;
  float* Z0 = bw.buf;
  float* Z1 = Z0 + n;
  float* Z2 = Z1 + n;
  float* T1 = Z2 + n;
  float* T2 = T1 + n;
  float* T3 = T2 + n;
  float* O = T3 + n;
  const int blocks = (int)std::min<long long>(148 * 8, (n + 255) / 256);
  auto G = [&](int axis, int ord) {
    return bw.diag + bw.diag_off[axis] + (size_t)ord * g.nf[axis] * 7;
  };
  auto band = [&](const float* in, float* o, int axis, int ord, float alpha, int acc) {
    k_band_axis<<<blocks, 256, 0, ctx->stream>>>(in, o, G(axis, ord), axis, g.nf[0], g.nf[1],
                                                 g.nf[2], nd, alpha, acc);
  };
  if (nd == 3) {
    band(c, Z0, 2, 0, 1.f, 0);
    band(c, Z1, 2, 1, 1.f, 0);
    band(c, Z2, 2, 2, 1.f, 0);
    band(Z0, T1, 1, 0, 1.f, 0);                 // y0 z0
    band(Z0, T2, 1, 2, 1.f, 0);                 // y2 z0 + y0 z2 + 2 y1 z1
    band(Z2, T2, 1, 0, 1.f, 1);
    band(Z1, T2, 1, 1, 2.f, 1);
    band(Z0, T3, 1, 1, 1.f, 0);                 // y1 z0 + y0 z1
    band(Z1, T3, 1, 0, 1.f, 1);
    band(T1, O, 0, 2, 1.f, 0);                  // x2 (y0 z0) + x0 (...) + 2 x1 (...)
    band(T2, O, 0, 0, 1.f, 1);
    band(T3, O, 0, 1, 2.f, 1);
    ctx->launches += 12;
  } else {
    band(c, Z0, 1, 0, 1.f, 0);                  // y0
    band(c, Z2, 1, 2, 1.f, 0);                  // y2
    band(c, Z1, 1, 1, 1.f, 0);                  // y1
    band(Z0, O, 0, 2, 1.f, 0);
    band(Z2, O, 0, 0, 1.f, 1);
    band(Z1, O, 0, 1, 2.f, 1);
    ctx->launches += 6;
  }
  CKL();
  *out = O;
  return SRWCR_OK;
}

__global__ void k_scale_scalar(double* __restrict__ v, double s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) v[0] *= s;
}

// E_dev <- C_p(c) (may be NULL); g_dev += weight * dC_p/dc (may be NULL).
srwcr_status bending_energy(srwcr_ctx* ctx, int level, const float* c, double* E_dev, float* g_dev,
                            float weight) {
  BendWork& bw = ctx->bend->w[level];
  RET_IF(bend_setup(ctx, level, bw));
  float* O = nullptr;
  RET_IF(bend_apply(ctx, level, bw, c, &O));
  if (E_dev) {
    k_dot_partial<<<kDotBlocks, 256, 0, ctx->stream>>>(c, O, bw.n, bw.part);
    k_dot_final<<<1, 32, 0, ctx->stream>>>(bw.part, kDotBlocks, E_dev);
    k_scale_scalar<<<1, 32, 0, ctx->stream>>>(E_dev, bw.inv_vol);
    CKL();
    ctx->launches += 3;
  }
  if (g_dev) {
    k_axpby<<<kDotBlocks, 256, 0, ctx->stream>>>((float)(2.0 * weight * bw.inv_vol), O, 1.f, g_dev,
                                                 bw.n);
    CKL();
    ctx->launches += 1;
  }
  return SRWCR_OK;
}

srwcr_status ensure_bend(srwcr_ctx* ctx) {
  if (!ctx->bend) {
    ctx->bend = new (std::nothrow) srwcr_bend_levels();
    if (!ctx->bend) return fail(SRWCR_ENOMEM, "host allocation failed");
  }
  return SRWCR_OK;
}

void free_bend(srwcr_ctx* ctx) {
  if (!ctx->bend) return;
  for (auto& w : ctx->bend->w) {
    if (w.buf) cudaFree(w.buf);
    if (w.diag) cudaFree(w.diag);
    if (w.part) cudaFree(w.part);
  }
  delete ctx->bend;
  ctx->bend = nullptr;
}

}  // namespace

extern "C" srwcr_status srwcr_bending_energy(srwcr_ctx* ctx, int level, const float* c_dev,
                                             double* E_dev, float* g_dev, float weight) {
  RET_IF(check_level(ctx, level));
  if (!c_dev) return fail(SRWCR_EINVAL, "c_dev is NULL");
  RET_IF(ensure_bend(ctx));
  return bending_energy(ctx, level, c_dev, E_dev, g_dev, weight);
}
