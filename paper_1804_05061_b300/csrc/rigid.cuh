// Entry points of the rigid model (the pre-alignment of Sec. III-D with the
// same measure): value and gradient with respect to the rigid parameters,
// coarse-to-fine L-BFGS over them, and the exact conversion of a rigid
// transform into FFD coefficients (an affine displacement is reproduced by
// the cubic B-spline).  Included once, at the end of srwcr.cu (after
// lbfgs.cuh).
#pragma once

namespace {

int rigid_np(const srwcr_ctx* ctx) { return ctx->cfg.ndim == 3 ? 6 : 3; }

// RMS distance of a level's voxels from its centre (voxel units): the
// optimiser works on angle * radius so that a unit step in any parameter
// moves voxels by about one voxel.
double rigid_radius(const Geo& g, int nd) {
  double s = 0.0;
  for (int d = 0; d < nd; ++d) s += ((double)g.n[d] * g.n[d] - 1.0) / 12.0;
  return std::sqrt(std::max(s, 1.0));
}

void rigid_matrix_host(int nd, const double* mu, double R[3][3]) {
  if (nd == 2) {
    srwcr::rot3(2, mu[2], 0.0, R);
    return;
  }
  double E[3][3][3], t1[3][3];
  for (int a = 0; a < 3; ++a) srwcr::rot3(a, mu[3 + a], 0.0, E[a]);
  srwcr::mul3(E[1], E[0], t1);
  srwcr::mul3(E[2], t1, R);
}

// Pyramid levels are 2^d box averages with floor sizes, so coarse voxel i
// sits at fine coordinate 2 i + 1/2.  A coarse transform
// R (y - c_c) + c_c + t_c is, in fine voxels, R (x - c_f) + c_f + t_f with
// t_f = 2 t_c + (R - I) delta, delta_d = c_f - (2 c_c + 1/2) = (N_f - 2 N_c)/2;
// the angles do not change.  dir = +1: coarse -> fine, -1: fine -> coarse.
void rigid_rescale(int nd, const Geo& fine, const Geo& coarse, double* mu, int dir) {
  double R[3][3];
  rigid_matrix_host(nd, mu, R);
  double delta[3] = {0.0, 0.0, 0.0}, rd[3];
  for (int d = 0; d < nd; ++d) delta[d] = 0.5 * (fine.n[d] - 2.0 * coarse.n[d]);
  for (int k = 0; k < 3; ++k) {
    rd[k] = -delta[k];
    for (int j = 0; j < 3; ++j) rd[k] += R[k][j] * delta[j];
  }
  for (int k = 0; k < nd; ++k) mu[k] = dir > 0 ? 2.0 * mu[k] + rd[k] : 0.5 * (mu[k] - rd[k]);
}

}  // namespace

extern "C" srwcr_status srwcr_rigid_value_and_grad(srwcr_ctx* ctx, int level, const float* mu_dev,
                                                   double* D_host, float* g_dev) {
  RET_IF(check_level(ctx, level));
  if (!mu_dev) return fail(SRWCR_EINVAL, "mu_dev is NULL");
  RET_IF(ensure_rigid(ctx));
  Level& lv = ctx->lev[level];
  RET_IF(check_finite_async(ctx, mu_dev, rigid_np(ctx)));
  RET_IF(run_rigid(ctx, lv, mu_dev, g_dev, 1.0));
  return finish_sync(ctx, lv, D_host);
}

extern "C" srwcr_status srwcr_rigid_to_ffd(srwcr_ctx* ctx, int level, const float* mu_dev,
                                           float* c_dev) {
  RET_IF(check_level(ctx, level));
  if (!mu_dev || !c_dev) return fail(SRWCR_EINVAL, "null argument");
  RET_IF(ensure_rigid(ctx));
  const Geo& g = ctx->lev[level].gv;
  const int nd = ctx->cfg.ndim;
  k_rigid_setup<<<1, 32, 0, ctx->stream>>>(mu_dev, nd, 0.5 * (g.n[0] - 1), 0.5 * (g.n[1] - 1),
                                           nd == 3 ? 0.5 * (g.n[2] - 1) : 0.0, 1.0, ctx->rigid_tab);
  CKL();
  const int blocks = (int)std::min<long long>(148 * 4, (g.ncoef + 255) / 256);
  k_rigid_to_ffd<<<blocks, 256, 0, ctx->stream>>>(g, nd, ctx->rigid_tab, c_dev);
  CKL();
  ctx->launches += 2;
  return SRWCR_OK;
}

extern "C" srwcr_status srwcr_rigid_register(srwcr_ctx* ctx, float* mu_dev_inout, int n_levels,
                                             const srwcr_lbfgs_opts* opts, srwcr_report* report) {
  RET_IF(check_level(ctx, 0));
  if (!mu_dev_inout) return fail(SRWCR_EINVAL, "mu_dev_inout is NULL");
  if (n_levels < 1 || n_levels > ctx->nlev)
    return fail(SRWCR_EINVAL, "n_levels %d outside [1, %d]", n_levels, ctx->nlev);
  srwcr_lbfgs_opts o;
  srwcr_lbfgs_default_opts(&o);
  if (opts) o = *opts;
  if (o.m < 1 || o.m > 16 || o.max_ls < 1) return fail(SRWCR_EINVAL, "bad L-BFGS options");
  RET_IF(ensure_rigid(ctx));
  if (report) memset(report, 0, sizeof *report);
  const int nd = ctx->cfg.ndim, np = rigid_np(ctx);
  float hf[6];
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(hf, mu_dev_inout, sizeof(float) * np, cudaMemcpyDeviceToHost));
  double mu[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < np; ++i) {
    if (!std::isfinite(hf[i])) return fail(SRWCR_ENUMERIC, "non-finite rigid parameters");
    mu[i] = hf[i];
  }
  for (int l = 0; l + 1 < n_levels; ++l)
    rigid_rescale(nd, ctx->lev[l].g, ctx->lev[l + 1].g, mu, -1);
  srwcr_status final_status = SRWCR_OK;
  for (int level = n_levels - 1; level >= 0; --level) {
    const Geo& g = ctx->lev[level].g;
    const double rho = rigid_radius(g, nd);
    LbfgsWork w;
    w.rigid = true;
    w.ang_scale = 1.0 / rho;
    srwcr_status st = alloc_work(w, np, o.m);
    if (st != SRWCR_OK) { free_work(w); return st; }
    float xs[6];
    for (int i = 0; i < np; ++i) xs[i] = (float)(i < nd ? mu[i] : mu[i] * rho);
    cudaError_t e = cudaMemcpy(w.x, xs, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_work(w); return fail(SRWCR_ECUDA, "%s", cudaGetErrorString(e)); }
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
      g_err = keep;
      return st;
    }
    if (level == 0) final_status = st;
    e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(xs, w.x, sizeof(float) * np, cudaMemcpyDeviceToHost);
    free_work(w);
    if (e != cudaSuccess) return fail(SRWCR_ECUDA, "rigid registration: %s", cudaGetErrorString(e));
    for (int i = 0; i < np; ++i) mu[i] = i < nd ? xs[i] : xs[i] / rho;
    if (level > 0) rigid_rescale(nd, ctx->lev[level - 1].g, g, mu, +1);
  }
  for (int i = 0; i < np; ++i) hf[i] = (float)mu[i];
  CK(cudaMemcpy(mu_dev_inout, hf, sizeof(float) * np, cudaMemcpyHostToDevice));
  if (final_status == SRWCR_ELINESEARCH)
    return fail(SRWCR_ELINESEARCH, "line search exhausted at the finest level");
  if (final_status == SRWCR_ENOTCONVERGED)
    return fail(SRWCR_ENOTCONVERGED, "iteration limit reached at the finest level");
  return SRWCR_OK;
}
