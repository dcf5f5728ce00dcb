// L-BFGS registration driver (Sec. II-F): limited-memory BFGS with m
// corrections (two-loop recursion), backtracking line search with the
// Armijo and weak-Wolfe conditions, and the "metric stable over the last w
// steps" stop; coarse-to-fine over the pyramid with cubic B-spline
// subdivision of the coefficients between levels.
//
// Vectors (coefficients, gradients, the m (s, y) pairs) live on the device
// in FP32; every inner product is accumulated in FP64 on the device with a
// fixed reduction order into a device scalar.  The two-loop recursion takes
// its coefficients from those scalars on the device, so the host, which runs
// the control flow, synchronises only for its decisions: once per iteration
// (g.g, g.d, d.d) and once per line-search trial (the cost, g_new.d and, for
// the history, s.y).  Included once, at the end of srwcr.cu.
#pragma once

namespace {

constexpr int kDotBlocks = 148;

// Partial FP64 dot products with a fixed partition; k_dot_final sums them in
// a fixed order, so results do not depend on scheduling.
__global__ void __launch_bounds__(256)
k_dot_partial(const float* __restrict__ a, const float* __restrict__ b, long long n,
              double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    s += (double)a[i] * (double)b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[i];
    out[0] = s;
  }
}

// y = a*x + b*y
__global__ void k_axpby(float a, const float* __restrict__ x, float b, float* __restrict__ y,
                        long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// y = a*x (x and y may alias)
__global__ void k_scal(float a, const float* __restrict__ x, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// Device scalars of one L-BFGS level (FP64): the decision values read by the
// host and the two-loop coefficients.
enum : int {
  kScGG = 0, kScGD, kScDD, kScSYN, kScYY, kScGND, kScSY,
  kScSQ = 8,              // [16] s_i . q of the first loop
  kScYQ = kScSQ + 16,     // [16] y_i . d of the second loop
  kScAlpha = kScYQ + 16,  // [16] alpha_i = rho_i s_i . q
  kScCount = kScAlpha + 16
};

// Two-loop updates with the coefficient formed from device scalars in FP64
// and rounded to FP32 as the host would: mode 0 (first loop) a = -(rho q_i),
// also storing alpha_i = rho q_i; mode 1 (second loop) a = alpha_i - rho q_i.
// y = a*x + b*y.
__global__ void k_axpby_sc(int mode, double rho, int iq, int ialpha, double* __restrict__ sc,
                           const float* __restrict__ x, float b, float* __restrict__ y,
                           long long n) {
  const double t = rho * sc[iq];
  const float a = mode == 0 ? (float)-t : (float)(sc[ialpha] - t);
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) sc[ialpha] = t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// y = (sc[inum] / sc[iden]) * x, the ratio rounded to FP32 (x, y may alias).
__global__ void k_scal_sc(const double* __restrict__ sc, int inum, int iden, const float* x,
                          float* y, long long n) {
  const float a = (float)(sc[inum] / sc[iden]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// z = x + a*y
__global__ void k_xpay(const float* __restrict__ x, float a, const float* __restrict__ y,
                       float* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    z[i] = x[i] + a * y[i];
}

// x[i] += a uniform draw from [-amp, amp]: SplitMix64 (S. Vigna's published
// generator: golden-ratio increment, two xor-shift-multiply rounds and a
// final xor-shift) of seed + (i + 1) steps, its top 24 bits as the fraction.
__global__ void k_jitter(float* __restrict__ x, long long n, float amp, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * 0x1p-24f;    // [0, 1)
    x[i] += amp * (2.f * u - 1.f);
  }
}

// Dyadic refinement of uniform cubic B-spline coefficients (knot doubling):
// fine node j sits at coarse node position (j+1)/2 (offset indices); odd j
// take (c[i-1] + 6c[i] + c[i+1])/8 with i = (j+1)/2, even j take
// (c[i] + c[i+1])/2 with i = j/2; coarse indices are clamped.  Values are
// doubled: displacements are in voxels of the level.
__device__ __forceinline__ int stencil(int j, int nc, int idx[3], float w[3]) {
  auto cl = [nc](int i) { return i < 0 ? 0 : (i >= nc ? nc - 1 : i); };
  if (j & 1) {
    const int i = (j + 1) / 2;
    idx[0] = cl(i - 1); idx[1] = cl(i); idx[2] = cl(i + 1);
    w[0] = 0.125f; w[1] = 0.75f; w[2] = 0.125f;
    return 3;
  }
  const int i = j / 2;
  idx[0] = cl(i); idx[1] = cl(i + 1);
  w[0] = 0.5f; w[1] = 0.5f;
  return 2;
}

__global__ void k_subdivide(const float* __restrict__ cc, int ndim, int cx, int cy, int cz,
                            float* __restrict__ cf, int fx, int fy, int fz) {
  const long long nfine = (long long)fx * fy * fz, ncoarse = (long long)cx * cy * cz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nfine * ndim;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / nfine);
    const long long nidx = i % nfine;
    const int jx = (int)(nidx % fx), jy = (int)((nidx / fx) % fy), jz = (int)(nidx / ((long long)fx * fy));
    int ix[3], iy[3], iz[3] = {0, 0, 0};
    float wx[3], wy[3], wz[3] = {1.f, 0.f, 0.f};
    const int nx = stencil(jx, cx, ix, wx), ny = stencil(jy, cy, iy, wy);
    const int nz = ndim == 3 ? stencil(jz, cz, iz, wz) : 1;
    float s = 0.f;
    for (int c = 0; c < nz; ++c)
      for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a)
          s += wx[a] * wy[b] * wz[c] * cc[k * ncoarse + ((long long)iz[c] * cy + iy[b]) * cx + ix[a]];
    cf[i] = 2.f * s;
  }
}

// bending.cuh: E_dev <- C_p(c), g_dev += weight * dC_p/dc; per-context work.
srwcr_status bending_energy(srwcr_ctx* ctx, int level, const float* c, double* E_dev, float* g_dev,
                            float weight);
srwcr_status ensure_bend(srwcr_ctx* ctx);

struct LbfgsWork {
  long long n = 0;
  int m = 0;
  float *x = nullptr, *g = nullptr, *d = nullptr, *xn = nullptr, *gn = nullptr;
  float* S = nullptr;  // [m][n]
  float* Y = nullptr;  // [m][n]
  double* part = nullptr;
  double* Edev = nullptr;  // device scalar: bending energy at the evaluated point
  double* host = nullptr;  // pinned [3]
  double* sc = nullptr;    // device scalars [kScCount]
  double* hsc = nullptr;   // pinned copies of the decision scalars [8]
  double wp = 0.0;         // penalty weight w_p of Eq. (1)
  bool rigid = false;      // x holds rigid parameters (angles as angle / ang_scale)
  double ang_scale = 1.0;
};

void free_work(LbfgsWork& w) {
  void* p[] = {w.x, w.g, w.d, w.xn, w.gn, w.S, w.Y, w.part, w.Edev, w.sc};
  for (void* q : p)
    if (q) cudaFree(q);
  if (w.host) cudaFreeHost(w.host);
  if (w.hsc) cudaFreeHost(w.hsc);
  w = LbfgsWork();
}

srwcr_status alloc_work(LbfgsWork& w, long long n, int m) {
  w.n = n;
  w.m = m;
  CK(cudaMalloc((void**)&w.x, sizeof(float) * n));
  CK(cudaMalloc((void**)&w.g, sizeof(float) * n));
  CK(cudaMalloc((void**)&w.d, sizeof(float) * n));
  CK(cudaMalloc((void**)&w.xn, sizeof(float) * n));
  CK(cudaMalloc((void**)&w.gn, sizeof(float) * n));
  CK(cudaMalloc((void**)&w.S, sizeof(float) * n * m));
  CK(cudaMalloc((void**)&w.Y, sizeof(float) * n * m));
  CK(cudaMalloc((void**)&w.part, sizeof(double) * kDotBlocks));
  CK(cudaMalloc((void**)&w.Edev, sizeof(double)));
  CK(cudaMallocHost((void**)&w.host, sizeof(double) * 3));
  CK(cudaMalloc((void**)&w.sc, sizeof(double) * kScCount));
  CK(cudaMallocHost((void**)&w.hsc, sizeof(double) * 8));
  return SRWCR_OK;
}

// Queue an FP64 inner product into the device scalar sc[idx].
srwcr_status dot_sc(srwcr_ctx* ctx, LbfgsWork& w, const float* a, const float* b, int idx) {
  k_dot_partial<<<kDotBlocks, 256, 0, ctx->stream>>>(a, b, w.n, w.part);
  CKL();
  k_dot_final<<<1, 32, 0, ctx->stream>>>(w.part, kDotBlocks, w.sc + idx);
  CKL();
  return SRWCR_OK;
}

// Copy sc[first, first + count) to hsc[first ...] and wait.
srwcr_status read_sc(srwcr_ctx* ctx, LbfgsWork& w, int first, int count) {
  CK(cudaMemcpyAsync(w.hsc + first, w.sc + first, sizeof(double) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SRWCR_OK;
}

srwcr_status scal(srwcr_ctx* ctx, LbfgsWork& w, float a, const float* x, float* y) {
  k_scal<<<kDotBlocks, 256, 0, ctx->stream>>>(a, x, y, w.n);
  CKL();
  return SRWCR_OK;
}

// w.d = -H w.g by the two-loop recursion (Nocedal & Wright, Alg. 7.4), all
// on the device: the hist_len newest (s, y) pairs sit in ring slots of w.S /
// w.Y (m slots, the newest at head - 1), rho[slot] = 1 / s.y, and the
// initial matrix is H0 = (s.y / y.y) I from the newest pair.  Queued.
srwcr_status two_loop(srwcr_ctx* ctx, LbfgsWork& w, int m, int hist_len, int head,
                      const double* rho) {
  const long long n = w.n;
  CK(cudaMemcpyAsync(w.d, w.g, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  for (int t = 0; t < hist_len; ++t) {
    const int slot = (head - 1 - t + m) % m;
    RET_IF(dot_sc(ctx, w, w.S + slot * n, w.d, kScSQ + slot));
    k_axpby_sc<<<kDotBlocks, 256, 0, ctx->stream>>>(0, rho[slot], kScSQ + slot, kScAlpha + slot,
                                                     w.sc, w.Y + slot * n, 1.f, w.d, n);
    CKL();
  }
  if (hist_len > 0) {
    const int newest = (head - 1 + m) % m;
    RET_IF(dot_sc(ctx, w, w.S + newest * n, w.Y + newest * n, kScSYN));
    RET_IF(dot_sc(ctx, w, w.Y + newest * n, w.Y + newest * n, kScYY));
    k_scal_sc<<<kDotBlocks, 256, 0, ctx->stream>>>(w.sc, kScSYN, kScYY, w.d, w.d, n);
    CKL();
  }
  for (int t = hist_len - 1; t >= 0; --t) {
    const int slot = (head - 1 - t + m) % m;
    RET_IF(dot_sc(ctx, w, w.Y + slot * n, w.d, kScYQ + slot));
    k_axpby_sc<<<kDotBlocks, 256, 0, ctx->stream>>>(1, rho[slot], kScYQ + slot, kScAlpha + slot,
                                                     w.sc, w.S + slot * n, 1.f, w.d, n);
    CKL();
  }
  return scal(ctx, w, -1.f, w.d, w.d);
}

// Coarse level `level` coefficients cc -> the next finer level's cf by dyadic
// cubic B-spline subdivision, values doubled.  Queued.
srwcr_status refine_queue(srwcr_ctx* ctx, int level, const float* cc, float* cf) {
  const Geo& gc = ctx->lev[level].g;
  const Geo& gf = ctx->lev[level - 1].g;
  k_subdivide<<<256, 256, 0, ctx->stream>>>(cc, ctx->cfg.ndim, gc.nf[0], gc.nf[1], gc.nf[2], cf,
                                            gf.nf[0], gf.nf[1], gf.nf[2]);
  CKL();
  return SRWCR_OK;
}

// Cost of Eq. (1) at x: f = D + w_p C_p, g = its gradient; queued, the
// cost's terms copied to w.host[1], w.host[2] (read after a synchronise with
// eval_cost).  The rigid model's bending energy is zero (an affine
// displacement), so its cost is D alone.
srwcr_status eval_queue(srwcr_ctx* ctx, int level, LbfgsWork& w, const float* x, float* g) {
  Level& lv = ctx->lev[level];
  if (w.rigid) {
    RET_IF(run_rigid(ctx, lv, x, g, w.ang_scale));
  } else {
    RET_IF(run_value_and_grad(ctx, lv, x, g));
    if (w.wp > 0.0) RET_IF(bending_energy(ctx, level, x, w.Edev, g, (float)w.wp));
  }
  CK(cudaMemcpyAsync(w.host + 1, lv.D, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (!w.rigid && w.wp > 0.0)
    CK(cudaMemcpyAsync(w.host + 2, w.Edev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return SRWCR_OK;
}

double eval_cost(const LbfgsWork& w) {
  return w.host[1] + (!w.rigid && w.wp > 0.0 ? w.wp * w.host[2] : 0.0);
}

srwcr_status eval(srwcr_ctx* ctx, int level, LbfgsWork& w, const float* x, float* g, double* f) {
  RET_IF(eval_queue(ctx, level, w, x, g));
  CK(cudaStreamSynchronize(ctx->stream));
  *f = eval_cost(w);
  return SRWCR_OK;
}

// One level of L-BFGS starting from w.x; result left in w.x.
srwcr_status lbfgs_level(srwcr_ctx* ctx, int level, LbfgsWork& w, const srwcr_lbfgs_opts& o,
                         int max_iter, int* iters, int* evals, double* fout) {
  double f;
  RET_IF(eval(ctx, level, w, w.x, w.g, &f));
  int ne = 1, hist_len = 0, head = 0;  // ring buffer of (s, y); head = next slot
  double rho[16];
  std::vector<double> fh{f};
  bool restart = true;
  srwcr_status status = SRWCR_ENOTCONVERGED;
  int it = 0;
  const long long n = w.n;
  for (it = 1; it <= max_iter; ++it) {
    RET_IF(dot_sc(ctx, w, w.g, w.g, kScGG));
    RET_IF(two_loop(ctx, w, o.m, hist_len, head, rho));  // w.d = -H g
    RET_IF(dot_sc(ctx, w, w.g, w.d, kScGD));
    RET_IF(dot_sc(ctx, w, w.d, w.d, kScDD));
    RET_IF(read_sc(ctx, w, kScGG, 3));
    const double gg = w.hsc[kScGG];
    double gd = w.hsc[kScGD], dd = w.hsc[kScDD];
    if (!(gg > 0.0)) { status = SRWCR_OK; --it; break; }
    if (!(gd < 0.0)) {
      hist_len = 0;
      head = 0;
      RET_IF(scal(ctx, w, -1.f, w.g, w.d));
      gd = -gg;
      dd = gg;  // d = -g: the same products, summed in the same order
      restart = true;
    }
    double alpha = restart ? 1.0 / std::sqrt(dd) : 1.0;
    bool accepted = false;
    double fn = f, sy = 0.0;
    // Each trial also forms s = xn - x, y = gn - g in the history slot head
    // (the two-loop above is done with it) and s.y, so an accepted trial
    // needs no further round trip.
    float* s = w.S + head * n;
    float* y = w.Y + head * n;
    for (int ls = 0; ls < o.max_ls; ++ls) {
      k_xpay<<<kDotBlocks, 256, 0, ctx->stream>>>(w.x, (float)alpha, w.d, w.xn, n);
      CKL();
      RET_IF(eval_queue(ctx, level, w, w.xn, w.gn));
      ++ne;
      RET_IF(dot_sc(ctx, w, w.gn, w.d, kScGND));
      k_xpay<<<kDotBlocks, 256, 0, ctx->stream>>>(w.xn, -1.f, w.x, s, n);
      CKL();
      k_xpay<<<kDotBlocks, 256, 0, ctx->stream>>>(w.gn, -1.f, w.g, y, n);
      CKL();
      RET_IF(dot_sc(ctx, w, s, y, kScSY));
      RET_IF(read_sc(ctx, w, kScGND, 2));
      fn = eval_cost(w);
      if (!std::isfinite(fn) || fn > f + o.c1 * alpha * gd) { alpha *= 0.5; continue; }
      if (w.hsc[kScGND] < o.c2 * gd) { alpha *= 2.0; continue; }
      accepted = true;
      sy = w.hsc[kScSY];
      break;
    }
    if (!accepted) { status = SRWCR_ELINESEARCH; --it; break; }
    std::swap(w.x, w.xn);
    std::swap(w.g, w.gn);
    f = fn;
    if (sy > 0.0) {
      rho[head] = 1.0 / sy;
      head = (head + 1) % o.m;
      hist_len = std::min(hist_len + 1, o.m);
    }
    restart = false;
    fh.push_back(f);
    const int win = o.stable_window;
    if (win > 0 && (int)fh.size() > win &&
        std::fabs(fh.back() - fh[fh.size() - 1 - win]) <= o.stable_rtol * std::fabs(fh.back())) {
      status = SRWCR_OK;
      break;
    }
  }
  if (it > max_iter) it = max_iter;
  *iters = it;
  *evals = ne;
  *fout = f;
  return status;
}

}  // namespace

extern "C" srwcr_status srwcr_register(srwcr_ctx* ctx, float* c_dev_inout, int n_levels,
                                       const srwcr_lbfgs_opts* opts, srwcr_report* report) {
  RET_IF(check_level(ctx, 0));
  if (!c_dev_inout) return fail(SRWCR_EINVAL, "c_dev_inout is NULL");
  if (n_levels < 1 || n_levels > ctx->nlev)
    return fail(SRWCR_EINVAL, "n_levels %d outside [1, %d]", n_levels, ctx->nlev);
  srwcr_lbfgs_opts o;
  srwcr_lbfgs_default_opts(&o);
  if (opts) o = *opts;
  if (o.m < 1 || o.m > 16 || o.max_ls < 1) return fail(SRWCR_EINVAL, "bad L-BFGS options");
  if (!(o.penalty_weight >= 0.0)) return fail(SRWCR_EINVAL, "penalty_weight must be >= 0");
  if (!(o.start_jitter >= 0.0)) return fail(SRWCR_EINVAL, "start_jitter must be >= 0");
  if (o.penalty_weight > 0.0) RET_IF(ensure_bend(ctx));
  if (report) memset(report, 0, sizeof *report);
  const int nd = ctx->cfg.ndim;
  srwcr_status final_status = SRWCR_OK;
  float* prev = nullptr;  // coarse result (device), owned here
  for (int level = n_levels - 1; level >= 0; --level) {
    const Geo& g = ctx->lev[level].g;
    LbfgsWork w;
    w.wp = o.penalty_weight;
    srwcr_status st = alloc_work(w, g.ncoef * nd, o.m);
    if (st != SRWCR_OK) { free_work(w); if (prev) cudaFree(prev); return st; }
    if (level == n_levels - 1 && n_levels > 1) {
      cudaMemsetAsync(w.x, 0, sizeof(float) * w.n, ctx->stream);
    } else if (level == n_levels - 1) {
      cudaMemcpyAsync(w.x, c_dev_inout, sizeof(float) * w.n, cudaMemcpyDeviceToDevice, ctx->stream);
    } else {
      st = refine_queue(ctx, level + 1, prev, w.x);
      if (st != SRWCR_OK) { free_work(w); cudaFree(prev); return st; }
    }
    if (level == n_levels - 1 && o.start_jitter > 0.0) {
      k_jitter<<<256, 256, 0, ctx->stream>>>(w.x, w.n, (float)o.start_jitter, o.seed);
      cudaError_t je = cudaGetLastError();
      if (je != cudaSuccess) {
        free_work(w);
        return fail(SRWCR_ECUDA, "start jitter: %s", cudaGetErrorString(je));
      }
    }
    int iters = 0, evals = 0;
    double f = 0.0;
    st = lbfgs_level(ctx, level, w, o, o.max_iter[level], &iters, &evals, &f);
    if (report) {
      report->iterations[level] = iters;
      report->evaluations[level] = evals;
      report->final_value[level] = f;
      report->status[level] = st;
      report->levels_run++;
    }
    if (st != SRWCR_OK && st != SRWCR_ENOTCONVERGED && st != SRWCR_ELINESEARCH) {
      std::string keep = g_err;
      free_work(w);
      if (prev) cudaFree(prev);
      g_err = keep;
      return st;
    }
    if (level == 0) final_status = st;
    if (prev) cudaFree(prev);
    prev = nullptr;
    if (level > 0) {
      if (cudaMalloc((void**)&prev, sizeof(float) * w.n) != cudaSuccess) {
        free_work(w);
        return fail(SRWCR_ENOMEM, "cudaMalloc failed");
      }
      cudaMemcpyAsync(prev, w.x, sizeof(float) * w.n, cudaMemcpyDeviceToDevice, ctx->stream);
    } else {
      cudaMemcpyAsync(c_dev_inout, w.x, sizeof(float) * w.n, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    free_work(w);
    if (e != cudaSuccess) {
      if (prev) cudaFree(prev);
      return fail(SRWCR_ECUDA, "registration: %s", cudaGetErrorString(e));
    }
  }
  if (final_status == SRWCR_ELINESEARCH)
    return fail(SRWCR_ELINESEARCH, "line search exhausted at the finest level");
  if (final_status == SRWCR_ENOTCONVERGED)
    return fail(SRWCR_ENOTCONVERGED, "iteration limit reached at the finest level");
  return SRWCR_OK;
}

extern "C" srwcr_status srwcr_lbfgs_direction(srwcr_ctx* ctx, int64_t n, int hist_len,
                                              const float* S_dev, const float* Y_dev,
                                              const float* g_dev, float* d_dev) {
  if (!ctx) return fail(SRWCR_EINVAL, "null context");
  if (n < 1 || hist_len < 0 || hist_len > 16) return fail(SRWCR_EINVAL, "bad n or hist_len");
  if (!g_dev || !d_dev || (hist_len > 0 && (!S_dev || !Y_dev)))
    return fail(SRWCR_EINVAL, "null device pointer");
  const int m = hist_len > 0 ? hist_len : 1;
  LbfgsWork w;
  srwcr_status st = alloc_work(w, n, m);
  if (st != SRWCR_OK) { free_work(w); return st; }
  double rho[16];
  cudaError_t e = cudaMemcpyAsync(w.g, g_dev, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess && hist_len > 0)
    e = cudaMemcpyAsync(w.S, S_dev, sizeof(float) * n * hist_len, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess && hist_len > 0)
    e = cudaMemcpyAsync(w.Y, Y_dev, sizeof(float) * n * hist_len, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) st = fail(SRWCR_ECUDA, "copy: %s", cudaGetErrorString(e));
  // rho_i = 1 / s_i.y_i from the same FP64 device dot the driver forms.
  for (int i = 0; i < hist_len && st == SRWCR_OK; ++i) {
    st = dot_sc(ctx, w, w.S + i * n, w.Y + i * n, kScSY);
    if (st == SRWCR_OK) st = read_sc(ctx, w, kScSY, 1);
    if (st == SRWCR_OK && !(w.hsc[kScSY] > 0.0)) st = fail(SRWCR_EINVAL, "pair %d has s.y <= 0", i);
    if (st == SRWCR_OK) rho[i] = 1.0 / w.hsc[kScSY];
  }
  // Slots 0 .. hist_len-1 hold the pairs oldest first: the newest is at
  // head - 1 with head = 0 (mod m).
  if (st == SRWCR_OK) st = two_loop(ctx, w, m, hist_len, 0, rho);
  if (st == SRWCR_OK) {
    e = cudaMemcpyAsync(d_dev, w.d, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = fail(SRWCR_ECUDA, "two-loop: %s", cudaGetErrorString(e));
  }
  free_work(w);
  return st;
}

extern "C" srwcr_status srwcr_refine(srwcr_ctx* ctx, int level, const float* c_coarse_dev,
                                     float* c_fine_dev) {
  RET_IF(check_level(ctx, level));
  if (level < 1) return fail(SRWCR_EINVAL, "level %d has no finer level", level);
  if (!c_coarse_dev || !c_fine_dev) return fail(SRWCR_EINVAL, "null device pointer");
  return refine_queue(ctx, level, c_coarse_dev, c_fine_dev);
}
