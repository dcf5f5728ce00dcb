/*
 * FP64 CPU oracle for SRWCR and its gradient -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C written from the definitions of
 * Gong et al., "Non-rigid image registration using spatially region-weighted
 * correlation ratio and GPU-acceleration" (arXiv 1804.05061).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header, table or constant with the CUDA path.
 *
 * Conventions (readings of the paper where it is silent; each is listed in
 * the design notes of the repository):
 *  - Images are x-fastest arrays, index (z*ny + y)*nx + x; the domain is the
 *    integer lattice 0 <= x < N (Sec. II, first paragraph).
 *  - Control node j (offset form, j = 0 ... n-1) sits at (j-1)*delta, so the
 *    node that Eq. (17) calls p_x = floor(x/delta) - 1 has offset index
 *    floor(x/delta).  Coefficients are displacements in voxels, stored
 *    component-major c[k][nz][ny][nx].
 *  - Spatial bins (Eq. 7) use a rational spacing num/den per axis so that
 *    cell = floor(x*den/num) and eta = (x*den mod num)/num are exact.
 *  - Backward warping (Sec. II-F) samples M at T(x) by trilinear
 *    interpolation with clamp-to-border; its gradient is the analytic
 *    gradient of the interpolant, zero along an axis where T(x) left
 *    [0, N-1].  Cell [floor(y), floor(y)+1], and [N-2, N-1] at y = N-1.
 *  - Intensity bins a, b run over 0..L (Eq. 3).  The Parzen derivative in
 *    Eqs. (19)/(27) is taken inside the cell [k, k+1] holding B,
 *    k = min(floor(B), L-1) (see orc_parzen_dkappa).
 *  - A region whose p(r) is 0, or whose variance sigma_r^2 is at most
 *    1e-6 * max(1, E_r[b^2]) (an intensity standard deviation below 1e-3 bin
 *    at unit scale), is degenerate: it contributes nothing to the value or
 *    the gradient and is counted.  Eqs. (9)-(10) divide by sigma_r^2 and the
 *    paper does not treat sigma_r^2 -> 0; in such regions 1 - CR_r is a 0/0
 *    limit decided by voxels of negligible spatial weight.
 *
 * Parity: pinned by the -m "not gpu" tests (closed forms, invariants, brute
 * force on tiny inputs, central finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
  int ndim;             /* 2 or 3 */
  int64_t n[3];         /* Nx, Ny, Nz (Nz = 1 in 2-D) */
  int64_t ffd_sp[3];    /* control spacing delta per axis (voxels) */
  int64_t sb_num[3];    /* spatial-bin spacing = sb_num/sb_den voxels */
  int64_t sb_den[3];
  int nbins;            /* L + 1 */
  int sb_mode;          /* 0: cubic B-spline distribution, Eq. (7); 1: boxcar patches, Eq. (6) */
  int xform;            /* 0: FFD, Eq. (17), c = coefficients; 1: rigid, c = parameters */
} orc_problem;

/* ---------------------------------------------------------------------- */
/* Eq. (8): the four pieces of the uniform cubic B-spline.                 */
/* ---------------------------------------------------------------------- */
double orc_bspline(int l, double t) {
  switch (l) {
    case 0: return (1.0 - t) * (1.0 - t) * (1.0 - t) / 6.0;
    case 1: return (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    case 2: return (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    case 3: return t * t * t / 6.0;
    default: return 0.0;
  }
}

/* Eq. (5): second-order Parzen window of Xu et al. */
double orc_parzen(double t) {
  double a = fabs(t);
  if (a < 0.5) return -1.8 * a * a - 0.1 * a + 1.0;
  if (a < 1.0) return 1.8 * a * a - 3.7 * a + 1.9;
  return 0.0;
}

/* Left derivative of Eq. (5), dh/dkappa taken from below. */
double orc_parzen_dleft(double t) {
  if (t <= -1.0) return 0.0;
  if (t <= -0.5) return 3.6 * t + 3.7;   /* h = 1.8 t^2 + 3.7 t + 1.9 on (-1,-0.5] */
  if (t <= 0.0) return -3.6 * t + 0.1;   /* h = -1.8 t^2 + 0.1 t + 1 on (-0.5,0]  */
  if (t <= 0.5) return -3.6 * t - 0.1;   /* h = -1.8 t^2 - 0.1 t + 1 on (0,0.5]   */
  if (t <= 1.0) return 3.6 * t - 3.7;    /* h = 1.8 t^2 - 3.7 t + 1.9 on (0.5,1]  */
  return 0.0;
}

/* Right derivative of Eq. (5), dh/dkappa taken from above. */
double orc_parzen_dright(double t) {
  if (t < -1.0) return 0.0;
  if (t < -0.5) return 3.6 * t + 3.7;
  if (t < 0.0) return -3.6 * t + 0.1;
  if (t < 0.5) return -3.6 * t - 0.1;
  if (t < 1.0) return 3.6 * t - 3.7;
  return 0.0;
}

/* dh/dkappa at kappa = b - B, as it enters Eqs. (19)/(27).  h has kinks at
 * integer kappa, so the derivative is taken inside the cell [k, k+1] that
 * holds B, k = min(floor(B), L-1): from above in B (below in kappa) except
 * at the top B = L, where the cell is [L-1, L] and the derivative is from
 * below in B.  B outside [0, L] never occurs (warped values of an image in
 * [0, L] stay in [0, L]). */
double orc_parzen_dkappa(double b, double B, int L) {
  if (B >= (double)L) return orc_parzen_dright(b - B);
  return orc_parzen_dleft(b - B);
}

/* Sec. II (normalisation to [0, L_eps]): linear min-max map in FP64.
 * Returns ORC_EINVAL for a constant image. */
int orc_normalise(const float* v, int64_t n, double L, double* out) {
  if (n <= 0) return ORC_EINVAL;
  double mn = v[0], mx = v[0];
  for (int64_t i = 1; i < n; ++i) {
    if (v[i] < mn) mn = v[i];
    if (v[i] > mx) mx = v[i];
  }
  if (!(mx > mn)) return ORC_EINVAL;
  for (int64_t i = 0; i < n; ++i) out[i] = L * ((double)v[i] - mn) / (mx - mn);
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Geometry helpers                                                        */
/* ---------------------------------------------------------------------- */
static int64_t ffd_nodes(const orc_problem* P, int d) {
  if (d >= P->ndim) return 1;
  return (P->n[d] - 1) / P->ffd_sp[d] + 4;
}

int64_t orc_n_ffd_nodes(const orc_problem* P, int d) { return ffd_nodes(P, d); }

static int64_t sbins(const orc_problem* P, int d) {
  if (d >= P->ndim) return 1;
  if (P->sb_mode == 1) return (P->n[d] * P->sb_den[d] + P->sb_num[d] - 1) / P->sb_num[d];
  return (P->n[d] - 1) * P->sb_den[d] / P->sb_num[d] + 4;
}

int64_t orc_n_sbins(const orc_problem* P, int d) { return sbins(P, d); }

int64_t orc_n_regions(const orc_problem* P) { return sbins(P, 0) * sbins(P, 1) * sbins(P, 2); }

/* Spatial distribution w(r, x): the bins with (possibly) nonzero weight at
 * voxel x and their weights.  B-spline mode, Eq. (7): the 4^d bins whose
 * cubic support covers x, weight beta_l(eta) per axis.  Boxcar, Eq. (6): the
 * single patch containing x, weight 1.  Returns the number of entries. */
static int spatial_weights(const orc_problem* P, const int64_t xv[3], int64_t* bins,
                           double* w) {
  int64_t cell[3];
  double wax[3][4];
  int nax[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= P->ndim) {
      cell[d] = 0; nax[d] = 1; wax[d][0] = 1.0;
      continue;
    }
    int64_t q = xv[d] * P->sb_den[d];
    cell[d] = q / P->sb_num[d];
    if (P->sb_mode == 1) {
      nax[d] = 1; wax[d][0] = 1.0;
    } else {
      double eta = (double)(q % P->sb_num[d]) / (double)P->sb_num[d];
      nax[d] = 4;
      for (int l = 0; l < 4; ++l) wax[d][l] = orc_bspline(l, eta);
    }
  }
  int64_t nbx = sbins(P, 0), nby = sbins(P, 1);
  int cnt = 0;
  for (int k = 0; k < nax[2]; ++k)
    for (int j = 0; j < nax[1]; ++j)
      for (int i = 0; i < nax[0]; ++i) {
        bins[cnt] = ((cell[2] + k) * nby + (cell[1] + j)) * nbx + (cell[0] + i);
        w[cnt] = wax[0][i] * wax[1][j] * wax[2][k];
        ++cnt;
      }
  return cnt;
}

/* Debug/pin helper: spatial bins and weights of one voxel. */
int orc_spatial_weights(const orc_problem* P, int64_t x, int64_t y, int64_t z, int64_t* bins,
                        double* w) {
  int64_t xv[3] = {x, y, z};
  return spatial_weights(P, xv, bins, w);
}

/* FFD, Eqs. (1) and (17): u_k(x) = sum over the 4^d nodes of x of
 * beta_l(eta) beta_m(gamma) beta_n(tau) c_k[node]. */
static void rigid_displacement(const orc_problem* P, const double* c, const int64_t xv[3],
                               double u[3]);

static void displacement(const orc_problem* P, const double* c, const int64_t xv[3],
                         double u[3]) {
  if (P->xform == 1) {
    rigid_displacement(P, c, xv, u);
    return;
  }
  int64_t nfx = ffd_nodes(P, 0), nfy = ffd_nodes(P, 1), nfz = ffd_nodes(P, 2);
  int64_t ncoef = nfx * nfy * nfz;
  int64_t p[3];
  double wax[3][4];
  int nax[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= P->ndim) { p[d] = 0; nax[d] = 1; wax[d][0] = 1.0; continue; }
    p[d] = xv[d] / P->ffd_sp[d];
    double eta = (double)(xv[d] % P->ffd_sp[d]) / (double)P->ffd_sp[d];
    nax[d] = 4;
    for (int l = 0; l < 4; ++l) wax[d][l] = orc_bspline(l, eta);
  }
  u[0] = u[1] = u[2] = 0.0;
  for (int k = 0; k < P->ndim; ++k) {
    double s = 0.0;
    for (int nn = 0; nn < nax[2]; ++nn)
      for (int m = 0; m < nax[1]; ++m)
        for (int l = 0; l < nax[0]; ++l) {
          int64_t node = ((p[2] + nn) * nfy + (p[1] + m)) * nfx + (p[0] + l);
          s += wax[0][l] * wax[1][m] * wax[2][nn] * c[k * ncoef + node];
        }
    u[k] = s;
  }
}

/* Rigid model (the pre-alignment of Sec. III-D, same measure): rotation about
 * the image centre x_c = (N - 1) / 2 followed by a translation,
 *   T(x) = R (x - x_c) + x_c + t.
 * 3-D: c = (t_x, t_y, t_z, alpha, beta, gamma), R = Rz(gamma) Ry(beta) Rx(alpha)
 * (rotations about the fixed x, then y, then z axis); 2-D: c = (t_x, t_y,
 * theta), R the plane rotation by theta.  Voxel units, radians.  R is built by
 * multiplying the elementary rotations. */
static void mat3_mul(const double a[3][3], const double b[3][3], double out[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      out[i][j] = s;
    }
}

int orc_rigid_matrix(int ndim, const double* c, double R[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = i == j ? 1.0 : 0.0;
  if (ndim == 2) {
    const double th = c[2];
    R[0][0] = cos(th); R[0][1] = -sin(th);
    R[1][0] = sin(th); R[1][1] = cos(th);
    return ORC_OK;
  }
  const double a = c[3], b = c[4], g = c[5];
  const double Rx[3][3] = {{1, 0, 0}, {0, cos(a), -sin(a)}, {0, sin(a), cos(a)}};
  const double Ry[3][3] = {{cos(b), 0, sin(b)}, {0, 1, 0}, {-sin(b), 0, cos(b)}};
  const double Rz[3][3] = {{cos(g), -sin(g), 0}, {sin(g), cos(g), 0}, {0, 0, 1}};
  double t[3][3];
  mat3_mul(Ry, Rx, t);
  mat3_mul(Rz, t, R);
  return ORC_OK;
}

static void rigid_displacement(const orc_problem* P, const double* c, const int64_t xv[3],
                               double u[3]) {
  double R[3][3], q[3];
  orc_rigid_matrix(P->ndim, c, R);
  for (int d = 0; d < 3; ++d) q[d] = d < P->ndim ? (double)xv[d] - 0.5 * (double)(P->n[d] - 1) : 0.0;
  for (int k = 0; k < 3; ++k) {
    if (k >= P->ndim) { u[k] = 0.0; continue; }
    double s = 0.0;
    for (int j = 0; j < P->ndim; ++j) s += R[k][j] * q[j];
    u[k] = s + 0.5 * (double)(P->n[k] - 1) + c[k] - (double)xv[k];
  }
}

int orc_displacement(const orc_problem* P, const double* c, int64_t x, int64_t y, int64_t z,
                     double* u) {
  int64_t xv[3] = {x, y, z};
  displacement(P, c, xv, u);
  return ORC_OK;
}

/* Backward warping (Sec. II-F): trilinear interpolation of M at position y
 * with clamp-to-border, and the analytic gradient of the interpolant. */
static double interp(const orc_problem* P, const double* M, const double yv[3], double g[3]) {
  int64_t i0[3];
  double t[3];
  int inside[3];
  for (int d = 0; d < 3; ++d) {
    int64_t N = P->n[d];
    if (d >= P->ndim || N == 1) { i0[d] = 0; t[d] = 0.0; inside[d] = 0; continue; }
    double yc = yv[d];
    inside[d] = 1;
    if (yc < 0.0) { yc = 0.0; inside[d] = 0; }
    if (yc > (double)(N - 1)) { yc = (double)(N - 1); inside[d] = 0; }
    int64_t f = (int64_t)floor(yc);
    if (f > N - 2) f = N - 2;
    i0[d] = f;
    t[d] = yc - (double)f;
  }
  int64_t nx = P->n[0], ny = P->n[1];
  int ex = (P->ndim >= 1 && P->n[0] > 1), ey = (P->n[1] > 1), ez = (P->ndim == 3 && P->n[2] > 1);
  double v = 0.0;
  g[0] = g[1] = g[2] = 0.0;
  for (int dz = 0; dz <= ez; ++dz)
    for (int dy = 0; dy <= ey; ++dy)
      for (int dx = 0; dx <= ex; ++dx) {
        double wx = ex ? (dx ? t[0] : 1.0 - t[0]) : 1.0;
        double wy = ey ? (dy ? t[1] : 1.0 - t[1]) : 1.0;
        double wz = ez ? (dz ? t[2] : 1.0 - t[2]) : 1.0;
        double m = M[((i0[2] + dz) * ny + (i0[1] + dy)) * nx + (i0[0] + dx)];
        v += wx * wy * wz * m;
        if (ex) g[0] += (dx ? 1.0 : -1.0) * wy * wz * m;
        if (ey) g[1] += wx * (dy ? 1.0 : -1.0) * wz * m;
        if (ez) g[2] += wx * wy * (dz ? 1.0 : -1.0) * m;
      }
  for (int d = 0; d < 3; ++d)
    if (!inside[d]) g[d] = 0.0;
  return v;
}

int orc_interp(const orc_problem* P, const double* M, double y0, double y1, double y2,
               double* val_grad /* [4] */) {
  double yv[3] = {y0, y1, y2}, g[3];
  val_grad[0] = interp(P, M, yv, g);
  val_grad[1] = g[0]; val_grad[2] = g[1]; val_grad[3] = g[2];
  return ORC_OK;
}

/* B(x) = M(T(x)) for every voxel, with the warped position's gradient. */
static void warp_voxel(const orc_problem* P, const double* M, const double* c,
                       const int64_t xv[3], double* B, double gM[3]) {
  double u[3], yv[3];
  displacement(P, c, xv, u);
  for (int d = 0; d < 3; ++d) yv[d] = (double)xv[d] + u[d];
  *B = interp(P, M, yv, gM);
}

int orc_warp(const orc_problem* P, const double* M, const double* c, double* B_out,
             double* grad_out /* [3*N] or NULL */) {
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double g[3];
        warp_voxel(P, M, c, xv, &B_out[idx], g);
        if (grad_out)
          for (int d = 0; d < 3; ++d) grad_out[3 * idx + d] = g[d];
      }
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Eq. (3): the three-channel joint PDF p(a, b, r) over all voxels.        */
/* Output p[(r*nb + a)*nb + b] (normalised by Z) and Z itself.             */
/* ---------------------------------------------------------------------- */
int orc_joint_pdf(const orc_problem* P, const double* A, const double* M, const double* c,
                  double* p, double* Z_out) {
  const int nb = P->nbins;
  const int64_t R = orc_n_regions(P);
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  memset(p, 0, sizeof(double) * (size_t)(R * nb * nb));
  double* ha = (double*)malloc(sizeof(double) * nb);
  double* hb = (double*)malloc(sizeof(double) * nb);
  int* ia = (int*)malloc(sizeof(int) * nb);
  int* ib = (int*)malloc(sizeof(int) * nb);
  if (!ha || !hb || !ia || !ib) { free(ha); free(hb); free(ia); free(ib); return ORC_ENOMEM; }
  int64_t bins[64];
  double w[64], gM[3];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double B;
        warp_voxel(P, M, c, xv, &B, gM);
        /* Parzen weights of every bin; only the nonzero ones are kept
         * (Eq. 5 vanishes for |t| >= 1, so at most three per image). */
        int na = 0, nbb = 0;
        for (int a = 0; a < nb; ++a) {
          double h = orc_parzen((double)a - A[idx]);
          if (h != 0.0) { ia[na] = a; ha[na++] = h; }
        }
        for (int b = 0; b < nb; ++b) {
          double h = orc_parzen((double)b - B);
          if (h != 0.0) { ib[nbb] = b; hb[nbb++] = h; }
        }
        int nw = spatial_weights(P, xv, bins, w);
        for (int s = 0; s < nw; ++s) {
          if (w[s] == 0.0) continue;
          double* pr = p + bins[s] * nb * nb;
          for (int i = 0; i < na; ++i) {
            double wa = w[s] * ha[i];
            for (int j = 0; j < nbb; ++j) pr[ia[i] * nb + ib[j]] += wa * hb[j];
          }
        }
      }
  free(ha);
  free(hb);
  free(ia);
  free(ib);
  double Z = 0.0;
  for (int64_t i = 0; i < R * nb * nb; ++i) Z += p[i];
  if (Z_out) *Z_out = Z;
  if (!(Z > 0.0)) return ORC_EINVAL;
  for (int64_t i = 0; i < R * nb * nb; ++i) p[i] /= Z;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Eqs. (4), (10), (9), (12): regional statistics and the SRWCR value.     */
/* ---------------------------------------------------------------------- */
int orc_srwcr_from_pdf(const double* p, int64_t R, int nb, double* D9, double* D12,
                       double* pr_out, double* mu_r_out, double* var_r_out, double* cr_out,
                       double* mu_ra_out, unsigned char* valid_out, int64_t* n_degenerate) {
  double* pra = (double*)malloc(sizeof(double) * nb);
  double* prb = (double*)malloc(sizeof(double) * nb);
  if (!pra || !prb) { free(pra); free(prb); return ORC_ENOMEM; }
  double d9 = 0.0, d12 = 0.0;
  int64_t ndeg = 0;
  for (int64_t r = 0; r < R; ++r) {
    const double* q = p + r * nb * nb;
    double* mu_ra = mu_ra_out + r * nb;
    /* Eq. (4): p(r), then the conditional p_r(a, b) and its marginals. */
    double pr = 0.0;
    for (int i = 0; i < nb * nb; ++i) pr += q[i];
    pr_out[r] = pr;
    mu_r_out[r] = var_r_out[r] = cr_out[r] = 0.0;
    valid_out[r] = 0;
    for (int a = 0; a < nb; ++a) mu_ra[a] = 0.0;
    if (!(pr > 0.0)) { ++ndeg; continue; }
    for (int a = 0; a < nb; ++a) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += q[a * nb + b] / pr;
      pra[a] = s;
    }
    for (int b = 0; b < nb; ++b) {
      double s = 0.0;
      for (int a = 0; a < nb; ++a) s += q[a * nb + b] / pr;
      prb[b] = s;
    }
    /* Eq. (10): mu_r, sigma_r^2 of the estimated image B in region r. */
    double mu = 0.0, m2 = 0.0;
    for (int b = 0; b < nb; ++b) {
      mu += (double)b * prb[b];
      m2 += (double)b * (double)b * prb[b];
    }
    double var = m2 - mu * mu;
    mu_r_out[r] = mu;
    var_r_out[r] = var;
    if (!(var > 1e-6 * fmax(1.0, m2))) { ++ndeg; continue; }
    valid_out[r] = 1;
    /* Eq. (10): conditional mean and variance given fixed bin a; Eq. (9). */
    double within = 0.0;
    for (int a = 0; a < nb; ++a) {
      if (!(pra[a] > 0.0)) continue;
      double s1 = 0.0, s2 = 0.0;
      for (int b = 0; b < nb; ++b) {
        double pab = q[a * nb + b] / pr;
        s1 += (double)b * pab;
        s2 += (double)b * (double)b * pab;
      }
      double mua = s1 / pra[a];
      double vara = s2 / pra[a] - mua * mua;
      mu_ra[a] = mua;
      within += vara * pra[a];
    }
    double one_minus_cr = within / var;
    cr_out[r] = 1.0 - one_minus_cr;
    d9 += pr * one_minus_cr;
    /* Eq. (12): the concise three-channel form. */
    double s12 = 0.0;
    for (int a = 0; a < nb; ++a) {
      if (!(pra[a] > 0.0)) continue;
      for (int b = 0; b < nb; ++b)
        s12 += ((double)b * (double)b - mu_ra[a] * mu_ra[a]) / var * q[a * nb + b];
    }
    d12 += s12;
  }
  free(pra);
  free(prb);
  *D9 = d9;
  *D12 = d12;
  if (n_degenerate) *n_degenerate = ndeg;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Eq. (27) (= Eq. 19): dD/dB at one voxel, M acting as the estimated      */
/* image B.  Uses the regional statistics from orc_srwcr_from_pdf.          */
/* ---------------------------------------------------------------------- */
typedef struct {
  const double* mu_r;
  const double* var_r;
  const double* cr;
  const double* mu_ra;
  const unsigned char* valid;
  double Z;
} orc_tables;

static double dD_dB(const orc_problem* P, const orc_tables* T, const int64_t xv[3], double Ax,
                    double Bx) {
  const int nb = P->nbins;
  int64_t bins[64];
  double w[64];
  int nw = spatial_weights(P, xv, bins, w);
  /* Nonzero h(a - A) and dh/dkappa(b - B) terms (at most three each). */
  int ia[4], ib[4], na = 0, ndb = 0;
  double ha[4], dh[4];
  for (int a = 0; a < nb && na < 4; ++a) {
    double h = orc_parzen((double)a - Ax);
    if (h != 0.0) { ia[na] = a; ha[na++] = h; }
  }
  for (int b = 0; b < nb && ndb < 4; ++b) {
    double d = orc_parzen_dkappa((double)b, Bx, nb - 1);
    if (d != 0.0) { ib[ndb] = b; dh[ndb++] = d; }
  }
  double acc = 0.0;
  for (int s = 0; s < nw; ++s) {
    int64_t r = bins[s];
    if (w[s] == 0.0 || !T->valid[r]) continue;
    double mu = T->mu_r[r], var = T->var_r[r], omc = 1.0 - T->cr[r];
    for (int i = 0; i < na; ++i) {
      double mua = T->mu_ra[r * nb + ia[i]];
      for (int j = 0; j < ndb; ++j) {
        double bb = (double)ib[j];
        double coef = (omc * (bb * bb - 2.0 * bb * mu) + 2.0 * bb * mua - bb * bb) / var;
        acc += coef * w[s] * ha[i] * dh[j];
      }
    }
  }
  return acc / T->Z;
}

/* Per-voxel dD/dB(x) for the whole image (optional debug/pin output). */
int orc_dD_dB_image(const orc_problem* P, const double* A, const double* M, const double* c,
                    const double* mu_r, const double* var_r, const double* cr,
                    const double* mu_ra, const unsigned char* valid, double Z, double* G_out) {
  orc_tables T = {mu_r, var_r, cr, mu_ra, valid, Z};
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double B, gM[3];
        warp_voxel(P, M, c, xv, &B, gM);
        G_out[idx] = dD_dB(P, &T, xv, A[idx], B);
      }
  return ORC_OK;
}

/* Eqs. (15)-(17): dD/dphi_s = sum_x dD/dB(x) * dM/dy(T(x)) * dT/dphi_s, for
 * every control coefficient.  g has the layout of c. */
int orc_gradient(const orc_problem* P, const double* A, const double* M, const double* c,
                 const double* mu_r, const double* var_r, const double* cr, const double* mu_ra,
                 const unsigned char* valid, double Z, double* g) {
  orc_tables T = {mu_r, var_r, cr, mu_ra, valid, Z};
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  int64_t nfx = ffd_nodes(P, 0), nfy = ffd_nodes(P, 1), nfz = ffd_nodes(P, 2);
  int64_t ncoef = nfx * nfy * nfz;
  memset(g, 0, sizeof(double) * (size_t)(P->ndim * ncoef));
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double B, gM[3];
        warp_voxel(P, M, c, xv, &B, gM);
        double G = dD_dB(P, &T, xv, A[idx], B);
        if (G == 0.0) continue;
        int64_t p[3];
        double wax[3][4];
        int nax[3];
        for (int d = 0; d < 3; ++d) {
          if (d >= P->ndim) { p[d] = 0; nax[d] = 1; wax[d][0] = 1.0; continue; }
          p[d] = xv[d] / P->ffd_sp[d];
          double eta = (double)(xv[d] % P->ffd_sp[d]) / (double)P->ffd_sp[d];
          nax[d] = 4;
          for (int l = 0; l < 4; ++l) wax[d][l] = orc_bspline(l, eta);
        }
        for (int nn = 0; nn < nax[2]; ++nn)
          for (int m = 0; m < nax[1]; ++m)
            for (int l = 0; l < nax[0]; ++l) {
              int64_t node = ((p[2] + nn) * nfy + (p[1] + m)) * nfx + (p[0] + l);
              double jac = wax[0][l] * wax[1][m] * wax[2][nn]; /* Eq. (17) */
              for (int k = 0; k < P->ndim; ++k) g[k * ncoef + node] += G * gM[k] * jac;
            }
      }
  return ORC_OK;
}

/* The same sum restricted to selected coefficients (flat indices into the
 * layout of c): each entry loops over its node's support only, so large
 * problems can be checked one coefficient at a time. */
int orc_gradient_at(const orc_problem* P, const double* A, const double* M, const double* c,
                    const double* mu_r, const double* var_r, const double* cr,
                    const double* mu_ra, const unsigned char* valid, double Z,
                    const int64_t* which, int64_t n_which, double* g_out) {
  orc_tables T = {mu_r, var_r, cr, mu_ra, valid, Z};
  int64_t nx = P->n[0], ny = P->n[1];
  int64_t nfx = ffd_nodes(P, 0), nfy = ffd_nodes(P, 1), nfz = ffd_nodes(P, 2);
  int64_t ncoef = nfx * nfy * nfz;
  for (int64_t q = 0; q < n_which; ++q) {
    int64_t flat = which[q];
    if (flat < 0 || flat >= P->ndim * ncoef) return ORC_EINVAL;
    int k = (int)(flat / ncoef);
    int64_t node = flat % ncoef;
    int64_t j[3] = {node % nfx, (node / nfx) % nfy, node / (nfx * nfy)};
    int64_t lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      if (d >= P->ndim) { lo[d] = 0; hi[d] = 0; continue; }
      /* node j (offset) sits at (j-1)*delta; support ((j-3)delta, (j+1)delta). */
      lo[d] = (j[d] - 3) * P->ffd_sp[d];
      hi[d] = (j[d] + 1) * P->ffd_sp[d];
      if (lo[d] < 0) lo[d] = 0;
      if (hi[d] > P->n[d] - 1) hi[d] = P->n[d] - 1;
    }
    double acc = 0.0;
    for (int64_t z = lo[2]; z <= hi[2]; ++z)
      for (int64_t y = lo[1]; y <= hi[1]; ++y)
        for (int64_t x = lo[0]; x <= hi[0]; ++x) {
          int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
          double jac = 1.0;
          int hit = 1;
          for (int d = 0; d < P->ndim; ++d) {
            int64_t pd = xv[d] / P->ffd_sp[d];
            int l = (int)(j[d] - pd);
            if (l < 0 || l > 3) { hit = 0; break; }
            double eta = (double)(xv[d] % P->ffd_sp[d]) / (double)P->ffd_sp[d];
            jac *= orc_bspline(l, eta);
          }
          if (!hit || jac == 0.0) continue;
          double B, gM[3];
          warp_voxel(P, M, c, xv, &B, gM);
          double G = dD_dB(P, &T, xv, A[idx], B);
          acc += G * gM[k] * jac;
        }
    g_out[q] = acc;
  }
  return ORC_OK;
}


/* ---------------------------------------------------------------------- */
/* Moving image as the model image A (Sec. II-E, Eqs. 20, 21): the warped  */
/* moving image M(T(x)) is binned by Eq. (5) and the fixed image F is the  */
/* estimated image B.  Joint PDF p[(r*nb + a)*nb + b], a from M(T(x)), b   */
/* from F(x); orc_srwcr_from_pdf then gives D and the regional statistics. */
/* ---------------------------------------------------------------------- */
int orc_joint_pdf_mas_a(const orc_problem* P, const double* F, const double* M, const double* c,
                        double* p, double* Z_out) {
  const int nb = P->nbins;
  const int64_t R = orc_n_regions(P);
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  memset(p, 0, sizeof(double) * (size_t)(R * nb * nb));
  int64_t bins[64];
  double w[64], gM[3];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double Av;
        warp_voxel(P, M, c, xv, &Av, gM);
        int ia[4], ib[4], na = 0, nbb = 0;
        double ha[4], hb[4];
        for (int a = 0; a < nb && na < 4; ++a) {
          double h = orc_parzen((double)a - Av);
          if (h != 0.0) { ia[na] = a; ha[na++] = h; }
        }
        for (int b = 0; b < nb && nbb < 4; ++b) {
          double h = orc_parzen((double)b - F[idx]);
          if (h != 0.0) { ib[nbb] = b; hb[nbb++] = h; }
        }
        int nw = spatial_weights(P, xv, bins, w);
        for (int s = 0; s < nw; ++s) {
          if (w[s] == 0.0) continue;
          double* pr = p + bins[s] * nb * nb;
          for (int i = 0; i < na; ++i)
            for (int j = 0; j < nbb; ++j) pr[ia[i] * nb + ib[j]] += w[s] * ha[i] * hb[j];
        }
      }
  double Z = 0.0;
  for (int64_t i = 0; i < R * nb * nb; ++i) Z += p[i];
  if (Z_out) *Z_out = Z;
  if (!(Z > 0.0)) return ORC_EINVAL;
  for (int64_t i = 0; i < R * nb * nb; ++i) p[i] /= Z;
  return ORC_OK;
}

/* Eq. (21): dD/dM(T(x)) at one voxel when M is A:
 *   (1/Z) sum_r sum_a sum_b (2b - mu_r(a)) mu_r(a) / sigma_r^2
 *         * w(r, x) h(b - F(x)) dh/dkappa at kappa = a - A(x),
 * with the in-cell derivative convention of orc_parzen_dkappa (A in the
 * role of its second argument) and mu_r(a) = 0 for an empty bin. */
static double dD_dA(const orc_problem* P, const orc_tables* T, const int64_t xv[3], double Ax,
                    double Fx) {
  const int nb = P->nbins;
  int64_t bins[64];
  double w[64];
  int nw = spatial_weights(P, xv, bins, w);
  int ia[4], ib[4], nda = 0, nbb = 0;
  double da[4], hb[4];
  for (int a = 0; a < nb && nda < 4; ++a) {
    double d = orc_parzen_dkappa((double)a, Ax, nb - 1);
    if (d != 0.0) { ia[nda] = a; da[nda++] = d; }
  }
  for (int b = 0; b < nb && nbb < 4; ++b) {
    double h = orc_parzen((double)b - Fx);
    if (h != 0.0) { ib[nbb] = b; hb[nbb++] = h; }
  }
  double acc = 0.0;
  for (int s = 0; s < nw; ++s) {
    int64_t r = bins[s];
    if (w[s] == 0.0 || !T->valid[r]) continue;
    double var = T->var_r[r];
    for (int i = 0; i < nda; ++i) {
      double mua = T->mu_ra[r * nb + ia[i]];
      for (int j = 0; j < nbb; ++j)
        acc += (2.0 * (double)ib[j] - mua) * mua / var * w[s] * hb[j] * da[i];
    }
  }
  return acc / T->Z;
}

/* Eqs. (15)-(17) with Eq. (21): dD/dc when M is A.  g has the layout of c. */
int orc_gradient_mas_a(const orc_problem* P, const double* F, const double* M, const double* c,
                       const double* mu_r, const double* var_r, const double* cr,
                       const double* mu_ra, const unsigned char* valid, double Z, double* g) {
  orc_tables T = {mu_r, var_r, cr, mu_ra, valid, Z};
  int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
  int64_t nfx = ffd_nodes(P, 0), nfy = ffd_nodes(P, 1), nfz = ffd_nodes(P, 2);
  int64_t ncoef = nfx * nfy * nfz;
  memset(g, 0, sizeof(double) * (size_t)(P->ndim * ncoef));
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xv[3] = {x, y, z}, idx = (z * ny + y) * nx + x;
        double Av, gM[3];
        warp_voxel(P, M, c, xv, &Av, gM);
        double G = dD_dA(P, &T, xv, Av, F[idx]);
        if (G == 0.0) continue;
        int64_t p[3];
        double wax[3][4];
        int nax[3];
        for (int d = 0; d < 3; ++d) {
          if (d >= P->ndim) { p[d] = 0; nax[d] = 1; wax[d][0] = 1.0; continue; }
          p[d] = xv[d] / P->ffd_sp[d];
          double eta = (double)(xv[d] % P->ffd_sp[d]) / (double)P->ffd_sp[d];
          nax[d] = 4;
          for (int l = 0; l < 4; ++l) wax[d][l] = orc_bspline(l, eta);
        }
        for (int nn = 0; nn < nax[2]; ++nn)
          for (int m = 0; m < nax[1]; ++m)
            for (int l = 0; l < nax[0]; ++l) {
              int64_t node = ((p[2] + nn) * nfy + (p[1] + m)) * nfx + (p[0] + l);
              double jac = wax[0][l] * wax[1][m] * wax[2][nn]; /* Eq. (17) */
              for (int k = 0; k < P->ndim; ++k) g[k * ncoef + node] += G * gM[k] * jac;
            }
      }
  return ORC_OK;
}
