/*
 * srwcr.h -- C ABI of libsrwcr, a B300 (sm_103a) implementation of the
 * spatially region-weighted correlation ratio (SRWCR) and its analytic
 * gradient with respect to cubic B-spline FFD coefficients (Gong et al.,
 * arXiv 1804.05061, Sec. II).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images are float32 arrays, x fastest: index (z*Ny + y)*Nx + x (Nz = 1 in
 * 2-D).  The fixed image F plays the model image A and the moving image M
 * the estimated image B of Eq. (2) ("M as B", gradient Eq. 19).
 *
 * FFD coefficients c (displacements in voxels of the level) and gradients g
 * are float32, component-major: c[k][nz][ny][nx] with k = 0 (x), 1 (y),
 * 2 (z); node j along an axis sits at (j-1)*delta, j = 0 .. floor((N-1)/delta)+3
 * (Eq. 17 with p_x = floor(x/delta) - 1).
 *
 * Every function returns an srwcr_status and never aborts; on failure
 * srwcr_last_error() returns a thread-local message.  Device pointers must
 * belong to the device that was current when the context was created.  All
 * work is queued on the context's stream; the *_async variants return
 * without synchronising, the others synchronise that stream before
 * returning.
 *
 * Ownership: the caller owns every pointer it passes; the context owns the
 * device memory it allocates (normalised images, pyramid, accumulators,
 * tables) and frees it in srwcr_destroy.  Calls on one context must not
 * overlap (they share its accumulators).
 */
#ifndef SRWCR_H
#define SRWCR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srwcr_ctx srwcr_ctx;

typedef enum {
  SRWCR_OK = 0,
  SRWCR_EINVAL = 1,        /* bad argument, constant image, size out of range */
  SRWCR_ENOMEM = 2,        /* device or host allocation failed */
  SRWCR_ECUDA = 3,         /* a CUDA call or kernel launch failed */
  SRWCR_ENUMERIC = 4,      /* non-finite coefficients or value */
  SRWCR_ELINESEARCH = 5,   /* L-BFGS line search exhausted its trials */
  SRWCR_ETIMEOUT = 6,      /* a bounded device wait gave up */
  SRWCR_ENOTCONVERGED = 7  /* L-BFGS stopped at its iteration limit */
} srwcr_status;

enum { SRWCR_STORAGE_F32 = 0, SRWCR_STORAGE_BF16 = 1 };

/* Which image is binned (Sec. II-E).  M as B (default): the fixed image F is
 * the model image A and the warped moving image the estimated image B
 * (gradient Eq. 19).  M as A: the warped moving image is A, binned by
 * Eq. (5), and F is B (gradient Eq. 21).  Either role runs on the
 * row-parallel kernels where the level's geometry allows them, else on the
 * general per-voxel kernels (srwcr_level_desc.kernel_path). */
enum { SRWCR_ROLE_M_AS_B = 0, SRWCR_ROLE_M_AS_A = 1 };

/* Spatial distribution w(r, x) of Eq. (3).  B-spline (default): the cubic
 * B-spline bins of Eq. (7), K+3 per axis.  Boxcar: Eq. (6) over a regular
 * partition into K patches per axis, patch floor(x K / N) holding voxel x with
 * weight 1 (the RaPTOR-style distribution of Eqs. 13-14, with the Parzen
 * window of Eq. 5 kept); needs sbin_intervals > 0.  Either distribution
 * runs on the kernels the level's geometry selects (srwcr_level_desc). */
enum { SRWCR_SPATIAL_BSPLINE = 0, SRWCR_SPATIAL_BOXCAR = 1 };

/* Problem configuration (Sec. II-F gives the paper's defaults: delta = 5,
 * L_eps = 31, i.e. 32 intensity bins). */
typedef struct {
  int ndim;               /* 2 or 3 */
  int dims[3];            /* Nx, Ny, Nz (Nz = 1 when ndim == 2); each 2..65535 */
  int ffd_spacing[3];     /* integer control spacing delta per axis, >= 1 */
  int sbin_intervals[3];  /* K per axis: spatial bins are cubic B-splines of
                             spacing N/K (K+3 bins, Eq. 7); 0 = bins on the
                             FFD grid (Sec. II-C) */
  int n_intensity_bins;   /* L_eps + 1, 2..256 (Eq. 3) */
  int storage;            /* SRWCR_STORAGE_F32 | SRWCR_STORAGE_BF16 */
  int pyramid_levels;     /* 1..4; level 0 is the full resolution */
  int tile[3];            /* voxel tile (x, y, z); 0 = chosen by the library */
  int bins_per_pass;      /* row-parallel value kernel: at most this many of a
                             tile's fixed-image bins per pass over its rows
                             (a tile using more takes several passes); 0 = as
                             many as fit in shared memory */
  int role;               /* SRWCR_ROLE_M_AS_B (0) | SRWCR_ROLE_M_AS_A */
  int finalize_lanes;     /* lanes per spatial bin in the per-bin moment
                             finalisation (Eqs. 9-12): 1, 2, 4, 8, 16 or 32;
                             0 = chosen per level from the number of
                             fixed-image bins each spatial bin holds */
  int spatial;            /* SRWCR_SPATIAL_BSPLINE (0) | SRWCR_SPATIAL_BOXCAR */
  int keep_warp;          /* value+gradient on the row-parallel kernels: the
                             value pass stores the warped intensity and the
                             moving-image gradient (16 bytes per voxel) for
                             the adjoint (1), or the adjoint recomputes them
                             (-1); 0 = stored for levels of at most 2^25
                             voxels, recomputed for larger ones */
} srwcr_config;

/* Geometry of one pyramid level. */
typedef struct {
  int dims[3];            /* voxels per axis */
  int ffd_nodes[3];       /* control nodes per axis (1 for an absent axis) */
  int sbins[3];           /* spatial bins per axis */
  int64_t n_voxels;
  int64_t n_params;       /* ndim * prod(ffd_nodes) = length of c and g */
  int64_t n_regions;      /* prod(sbins) */
  int tile[3];            /* voxel tile used by the kernels */
  int kernel_path;        /* 1: row-parallel kernels (32-wide tiles; a row
                             meets at most 11 FFD x-nodes and 12 spatial
                             x-bins: spacings >= 4 voxels along x);
                             0: general per-voxel kernels */
  int finalize_lanes;     /* lanes per spatial bin in the finalisation */
} srwcr_level_desc;

/* Create a context: validate cfg, upload both images, normalise each to
 * [0, L_eps] by its own min and max in FP64 (Sec. II, first paragraph),
 * round to the storage type, build the pyramid (2^d box averages, floor
 * sizes) and the fixed-image statistics p(r), p_r(a) of Eq. (4), which do
 * not depend on the transform.
 *   fixed, moving  Nx*Ny*Nz float32 each; host memory when
 *                  images_on_device == 0, device memory otherwise; not
 *                  retained.
 *   stream         cudaStream_t to queue all work on (NULL = legacy default).
 * Errors: SRWCR_EINVAL (bad cfg, constant image), SRWCR_ENOMEM, SRWCR_ECUDA. */
srwcr_status srwcr_create(const srwcr_config* cfg, const float* fixed, const float* moving,
                          int images_on_device, void* stream, srwcr_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
void srwcr_destroy(srwcr_ctx* ctx);

/* Thread-local description of the last failure on this thread. */
const char* srwcr_last_error(void);

/* Geometry of pyramid level `level` (0 = finest). */
srwcr_status srwcr_level_info(const srwcr_ctx* ctx, int level, srwcr_level_desc* out);

/* SRWCR value D of Eq. (9) (equivalently Eq. 12) at coefficients c_dev
 * (device, n_params floats).  D_host receives the FP64 value. */
srwcr_status srwcr_value(srwcr_ctx* ctx, int level, const float* c_dev, double* D_host);

/* D and its gradient dD/dc (Eqs. 15-17 with dD/dM from Eq. 19 / Eq. 27).
 * g_dev (device, n_params floats) is overwritten. */
srwcr_status srwcr_value_and_grad(srwcr_ctx* ctx, int level, const float* c_dev, double* D_host,
                                  float* g_dev);

/* Same, without synchronising: D is written to D_dev (device double).
 * Safe to capture in a CUDA graph once the context exists.  From the second
 * consecutive call with the same (level, c_dev, D_dev, g_dev) the library
 * captures the call once as its own CUDA graph (on a private stream) and
 * replays it on the context's stream while the arguments stay the same;
 * not while the context's stream is being captured by the caller or the
 * benchmark profiling events are on.  srwcr_autotune drops the graph. */
srwcr_status srwcr_value_and_grad_async(srwcr_ctx* ctx, int level, const float* c_dev,
                                        double* D_dev, float* g_dev);

/* End-to-end form with host buffers: copies c_host (n_params floats) to the
 * device, evaluates, copies g back to g_host (n_params floats) and D to
 * D_host (may be NULL).  Uses context-owned staging buffers; host buffers
 * may be pageable or pinned; the call synchronises.  A buffer counts as
 * page-locked only if its first and last byte lie in page-locked memory
 * mapped at one contiguous device range: then c is read by a kernel through
 * that mapping, and with both buffers page-locked the whole call is captured
 * as a CUDA graph on first use for this (level, c_host, g_host) and replayed
 * afterwards (the graph is dropped when srwcr_autotune re-selects a level's
 * kernels).  Buffers shorter than n_params floats are undefined behaviour.
 * Errors: SRWCR_EINVAL for a bad level or a NULL buffer, SRWCR_ENUMERIC for a
 * non-finite coefficient or value (g_host then holds no meaningful values). */
srwcr_status srwcr_value_and_grad_host(srwcr_ctx* ctx, int level, const float* c_host,
                                       double* D_host, float* g_host);

/* Forward half used by the autograd form: evaluates D (to D_dev) and keeps
 * the per-region tables of the finalisation (Table I) in the
 * context for a later srwcr_backward at the same level. */
srwcr_status srwcr_forward(srwcr_ctx* ctx, int level, const float* c_dev, double* D_dev);

/* Backward half: g_dev = gD * dD/dc using the tables of the most recent
 * srwcr_forward at this level.  The warp is recomputed, not stored.
 * gD_dev: device float scalar (NULL means 1). */
srwcr_status srwcr_backward(srwcr_ctx* ctx, int level, const float* c_dev, const float* gD_dev,
                            float* g_dev);

/* Per-region statistics of the last evaluation at `level`, copied to host:
 * out[4*r + 0..3] = p(r), sigma_r^2, CR(A,B|r), contribution p(r)(1-CR_r)
 * (Eqs. 4, 9, 10); degenerate regions (p(r) = 0, or sigma_r^2 <=
 * 1e-6 * max(1, mean square of B in the region)) report sigma^2 = CR = 0 and
 * contribute nothing to the value or the gradient.
 * n_degenerate (may be NULL) receives their number. */
srwcr_status srwcr_region_stats(srwcr_ctx* ctx, int level, double* out, int64_t* n_degenerate);

/* Debug: voxel-to-bin indexing exactly as the kernels compute it.  For each
 * voxel, out_dev[4*i + 0..2] = spatial-bin cell (x, y, z) (the voxel lies in
 * bins cell..cell+3 per axis, Eq. 7) and out_dev[4*i + 3] = fixed-image
 * intensity bin floor(A) clamped to [0, L_eps-1] (Eq. 5 support).
 * out_dev: device int32 array of 4*n_voxels. */
srwcr_status srwcr_debug_bins(srwcr_ctx* ctx, int level, int32_t* out_dev);

/* Debug: the warped, normalised moving image B(x) = M(T(x)) (Sec. II-F) as
 * the kernels compute it, to out_dev (device float, n_voxels). */
srwcr_status srwcr_debug_warp(srwcr_ctx* ctx, int level, const float* c_dev, float* out_dev);

/* Debug: the warped moving image and the gradient of its interpolant at the
 * warped point, as the kernels compute them (Sec. II-F; the gradient is the
 * dM/dT(x) factor of Eq. 16): out_dev[4*i + 0..3] = (B, dM/dy_x, dM/dy_y,
 * dM/dy_z) for voxel i (y_z = 0 in 2-D).  out_dev: device float array of
 * 4*n_voxels, 16-byte aligned.  Synchronises. */
srwcr_status srwcr_debug_warp_grad(srwcr_ctx* ctx, int level, const float* c_dev, float* out_dev);

/* The normalised images of pyramid level `level` as the kernels read them
 * (Sec. II: [0, L_eps]; coarser levels are 2^d box averages with floor sizes,
 * the multi-resolution scheme of Sec. II-F), converted to float32.
 * fixed_dev, moving_dev: device float arrays of n_voxels (either may be
 * NULL).  Synchronises. */
srwcr_status srwcr_level_images(srwcr_ctx* ctx, int level, float* fixed_dev, float* moving_dev);

/* Debug: the fixed-point conversions of the histogram flushes, written with
 * 32-bit operations (64-bit integer <-> float conversions run on this GPU's
 * narrow FP64 unit).  For i < n: fixed_dev[i] = the nearest integer to
 * v_dev[i] (ties to even), for 0 <= v < 2^64.  For i < m: float_dev[i] = the
 * nearest float (ties to even) to hi_dev[i] * 2^24 + lo_dev[i], for
 * hi <= 256 * (2^24 - 1) (the 48-bit word pairs of the row kernels' plane
 * histograms).  reference != 0 computes the same with CUDA's 64-bit
 * conversions instead, so a caller can compare the two bit for bit.  All
 * pointers are device arrays (may be NULL where their count is 0); runs on
 * the legacy default stream and synchronises the device.  SRWCR_EINVAL on a
 * negative count or a missing array. */
srwcr_status srwcr_debug_fixed_point(const float* v_dev, int64_t n, const uint32_t* hi_dev,
                                     const uint32_t* lo_dev, int64_t m, uint64_t* fixed_dev,
                                     float* float_dev, int reference);

/* Launch order of the row kernels' tiles, computed on the host (no device
 * work; the library builds it once per tile choice for every level that
 * keeps the static row distances).  A launch ends on its cheap tiles when
 * the costly ones go first (longest-first scheduling).
 * rowdist_host: one byte per 32-voxel x-row segment, laid out [z][y][x block]
 * with ceil(dims[0] / 32) blocks per row: the L-infinity distance from the
 * segment to the nearest nonzero moving-image voxel (the library's own maps
 * cap it at 64; any byte value is accepted).
 * dims: voxels per axis (x, y, z; 1 for the z axis of a 2-D image).  tile:
 * 32 x tile[1] x tile[2] voxels.  Tiles are numbered x block fastest, then
 * y, then z, as the row kernels number their CTAs; there are
 * ntiles = ceil(dims[0] / 32) * ceil(dims[1] / tile[1]) * ceil(dims[2] / tile[2]).
 * order_out (ntiles ints) receives the tiles in launch order, cost_out (may
 * be NULL, ntiles ints) each tile's cost.  A tile's cost is its number of
 * segments at distance <= 8.  Tiles are ordered by cost class
 * (cost * 16 / (max cost + 1)), classes in decreasing order, tiles of one
 * class in increasing index.  Errors: SRWCR_EINVAL for a NULL array, a size
 * out of range (more than 2^31 - 1 row segments included) or tile[0] != 32. */
srwcr_status srwcr_tile_order(const unsigned char* rowdist_host, const int* dims, const int* tile,
                              int* order_out, int* cost_out);

/* Benchmark hooks.  With profiling enabled the library brackets each of its
 * kernels with CUDA events on the context's stream.  srwcr_profile_read
 * synchronises the stream and reports, per kernel kind (0 = fused warp and
 * statistics, 1 = finalisation and value reduction, 2 = adjoint), the summed
 * device time in ms and the number of launches bracketed; `launches`
 * receives the number of kernels the context launched since the last reset
 * (profiled or not).  Arrays ms and counts hold 3 entries; any pointer may
 * be NULL.  reset != 0 clears the records. */
srwcr_status srwcr_set_profiling(srwcr_ctx* ctx, int enable);
srwcr_status srwcr_profile_read(srwcr_ctx* ctx, double* ms, int64_t* counts, int64_t* launches,
                                int reset);

/* Tile autotuner: times value+gradient at coefficients c_dev (device) for
 * each 32-wide voxel tile that fits the row-parallel kernels, `reps` runs
 * each, and keeps the fastest for this level.  The choice is cached per
 * problem signature (dimensions, spacings, bins, storage) for the life of
 * the process and, if the environment variable SRWCR_AUTOTUNE_CACHE names a
 * file, appended to that file and read back by later processes, which then
 * skip the timing.  tile_out (may be NULL) receives the chosen tile.  Uses
 * scratch allocations; not for use under stream capture. */
srwcr_status srwcr_autotune(srwcr_ctx* ctx, int level, const float* c_dev, int reps,
                            int* tile_out);

/* Allocation-free SRWCR value, for callers that may not allocate device
 * memory: code inside a CUDA-graph capture or an allocator callback, plugins
 * whose host application owns every cudaMalloc, real-time loops that must
 * not touch the allocator.  The paper has no counterpart; it is a deployment
 * variant of srwcr_value (general per-voxel kernels) that needs no context.
 *   cfg            problem as for srwcr_create (storage and pyramid_levels
 *                  are ignored: level 0, float32 images)
 *   fixed_dev, moving_dev  device float32 images ALREADY normalised to
 *                  [0, L_eps] (L_eps = n_intensity_bins - 1), e.g.
 *                  L*(v - min)/(max - min) in FP64 rounded to float32
 *   c_dev          device coefficients (layout as for srwcr_value)
 *   D_dev          device double receiving D of Eq. (9)
 *   stream         cudaStream_t (NULL = legacy default)
 * Work is queued on `stream`; the call does not synchronise.  Scratch is a
 * file-scope device array of 16 MiB that every device that loads the library
 * holds until exit.  A problem needs 28 bytes per (spatial bin, intensity
 * bin) pair plus 48 bytes per spatial bin, each of 8 blocks rounded up to 256
 * bytes: up to about 590 k pairs (the 512x512x300 workload with 3971 spatial
 * bins and 128 intensity bins needs 14.4 MB); larger problems are rejected
 * with SRWCR_EINVAL, the message stating the bytes needed.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it, so make that first call before any stream capture.  The
 * cache assumes one primary context per device for the life of the process:
 * do not call this entry point on a device after cudaDeviceReset.  Every call
 * shares the array and re-zeroes the parts it accumulates into: calls that
 * overlap on the GPU (other streams, other host threads) race.  The
 * normalising factor Z is the voxel count (weights sum to one per voxel),
 * so D can differ from srwcr_value's in the last digits.  No cudaMalloc,
 * cudaFree or other allocation happens. */
srwcr_status srwcr_value_noalloc(const srwcr_config* cfg, const float* fixed_dev,
                                 const float* moving_dev, const float* c_dev, double* D_dev,
                                 void* stream);

/* L-BFGS options (Sec. II-F: 5 corrections; 200/200/120 iterations per
 * level; backtracking with a Wolfe condition; stop when the metric is stable
 * over the last 20 steps). */
typedef struct {
  int m;                  /* history length (5) */
  int max_iter[4];        /* per level, finest first (e.g. 120, 200, 200) */
  int stable_window;      /* 20 */
  double stable_rtol;     /* 1e-5 */
  int max_ls;             /* line-search trials (20) */
  double c1, c2;          /* Armijo and curvature constants (1e-4, 0.9) */
  double penalty_weight;  /* w_p of Eq. (1): the cost is D + w_p * C_p with C_p
                             the bending energy (srwcr_bending_energy); 0 =
                             D alone (default).  The paper uses 0.1 for
                             mono-modal and 30 for multi-modal pairs. */
  double start_jitter;    /* > 0: srwcr_register adds to the start of its first
                             (coarsest) level coefficients drawn uniformly
                             from [-start_jitter, start_jitter] voxels
                             (SplitMix64 of seed and the coefficient index).
                             The identity map samples the moving image on
                             the lattice, where a two-valued image puts
                             every voxel at a kink of the Parzen window
                             (Eq. 5) and the gradient of Eqs. 19/21 is
                             one-sided; a start off the lattice avoids
                             it.  0 = no jitter (default).  The rigid and
                             batched drivers start where they are given. */
  unsigned long long seed;
} srwcr_lbfgs_opts;

typedef struct {
  int levels_run;
  int iterations[4];      /* per level, finest first */
  int evaluations[4];
  double final_value[4];  /* minimised cost (D, or D + w_p C_p) */
  int status[4];          /* srwcr_status per level */
} srwcr_report;

/* Fill opts with the defaults above. */
void srwcr_lbfgs_default_opts(srwcr_lbfgs_opts* opts);

/* Bending energy of the displacement, the penalty C_p of Eq. (1): the
 * thin-plate energy (1/|Omega|) * integral over Omega = prod_d [0, N_d - 1]
 * (voxel units) of sum_k sum_{i,j} (d^2 u_k / dx_i dx_j)^2, over ordered
 * pairs (i, j), u the FFD displacement at level `level`.  The paper takes
 * C_p from its ref. [26] without a formula; this is the standard definition,
 * integrated exactly (u is a tensor-product cubic B-spline).
 *   c_dev   device coefficients (layout as for srwcr_value)
 *   E_dev   device double receiving C_p, or NULL
 *   g_dev   device gradient to which weight * dC_p/dc is ADDED, or NULL
 * Queued on the context's stream without synchronising.  The first call at a
 * level allocates that level's work buffers (8 floats per parameter). */
srwcr_status srwcr_bending_energy(srwcr_ctx* ctx, int level, const float* c_dev, double* E_dev,
                                  float* g_dev, float weight);

/* Multi-resolution L-BFGS registration minimising D (Sec. II-F), or
 * D + w_p C_p when opts->penalty_weight > 0.
 * c_dev_inout (device, n_params of level 0) holds the finest-level start
 * and receives the result; levels run coarse to fine, each coarse result is
 * refined to the next level by cubic B-spline subdivision (values x2).
 * n_levels <= the context's pyramid_levels.  report may be NULL. */
srwcr_status srwcr_register(srwcr_ctx* ctx, float* c_dev_inout, int n_levels,
                            const srwcr_lbfgs_opts* opts, srwcr_report* report);

/* Coefficients of pyramid level `level` (>= 1) refined to level - 1, the
 * coarse-to-fine transfer of srwcr_register (Sec. II-F: the control grids of
 * the levels are concatenated): dyadic subdivision of the uniform cubic
 * B-spline (fine node 2i-1 takes (c[i-1] + 6 c[i] + c[i+1]) / 8, fine node
 * 2i takes (c[i] + c[i+1]) / 2, coarse indices clamped to the grid), values
 * doubled because displacements are in voxels of their level.  Where no
 * index is clamped, the fine displacement at fine voxel 2x equals twice the
 * coarse displacement at coarse voxel x.
 *   c_coarse_dev  device, n_params of `level`
 *   c_fine_dev    device, n_params of level - 1 (overwritten)
 * Queued on the context's stream.  Errors: SRWCR_EINVAL, SRWCR_ECUDA. */
srwcr_status srwcr_refine(srwcr_ctx* ctx, int level, const float* c_coarse_dev, float* c_fine_dev);

/* One L-BFGS search direction d = -H g (Sec. II-F) from the two-loop
 * recursion srwcr_register runs (Nocedal & Wright, Alg. 7.4: H0 = (s.y /
 * y.y) I from the newest pair, rho_i = 1 / s_i.y_i, FP32 vectors with FP64
 * inner products on the device), for an explicit history.
 *   n             vector length
 *   hist_len      number of (s, y) pairs, 0..16 (0 gives d = -g)
 *   S_dev, Y_dev  device float [hist_len][n], oldest pair first; each
 *                 s_i.y_i must be > 0 (else SRWCR_EINVAL)
 *   g_dev         device float [n]; d_dev device float [n] (overwritten)
 * Runs on the context's stream with scratch of its own; synchronises. */
srwcr_status srwcr_lbfgs_direction(srwcr_ctx* ctx, int64_t n, int hist_len, const float* S_dev,
                                   const float* Y_dev, const float* g_dev, float* d_dev);

/* ------------------------------------------------------------------------
 * Rigid model: the pre-alignment the paper runs with the same measure before
 * the non-rigid registration (Sec. III-D).  The transform rotates about the
 * level's centre x_c = (N - 1) / 2 (voxel units) and translates:
 *   T(x) = R (x - x_c) + x_c + t.
 * mu (device float32): 3-D (t_x, t_y, t_z, alpha, beta, gamma) with
 * R = Rz(gamma) Ry(beta) Rx(alpha) (rotations about the fixed x, y, z axes in
 * that order); 2-D (t_x, t_y, theta).  Translations in voxels of the level,
 * angles in radians.  The value is Eq. (9) with B(x) = M(T(x)) (the moving
 * image as B only: SRWCR_EINVAL for SRWCR_ROLE_M_AS_A); the gradient is
 * Eq. (16) with dT/dmu in place of the FFD basis.  On a row-parallel level
 * the transform is evaluated through the FFD kernels in its exact FFD form
 * (srwcr_rigid_to_ffd) and dD/dmu is dD/dc chained through that form; on a
 * general-path level the per-voxel kernels take the rigid map directly. */

/* D (host) and, when g_dev != NULL, dD/dmu (device, 6 or 3 floats) at mu.
 * Synchronises.  Errors: SRWCR_EINVAL, SRWCR_ENUMERIC (non-finite mu or
 * value), SRWCR_ECUDA. */
srwcr_status srwcr_rigid_value_and_grad(srwcr_ctx* ctx, int level, const float* mu_dev,
                                        double* D_host, float* g_dev);

/* c_dev (device, n_params of `level`) <- FFD coefficients whose warp equals
 * the rigid transform mu: the rigid displacement sampled at the control
 * nodes (node j at (j - 1) delta), which the cubic B-spline reproduces
 * exactly at every voxel (the displacement is affine).  This hands a rigid
 * pre-alignment to srwcr_register.  Queued on the context's stream. */
srwcr_status srwcr_rigid_to_ffd(srwcr_ctx* ctx, int level, const float* mu_dev, float* c_dev);

/* Multi-resolution L-BFGS over the rigid parameters (the options and report
 * of srwcr_register; penalty_weight is ignored: a rigid displacement has
 * zero bending energy).  mu_dev_inout holds the start in level-0 voxels and
 * receives the result.  Levels run coarse to fine; the transform is mapped
 * exactly between levels (coarse voxel i sits at fine coordinate 2i + 1/2:
 * translations double, plus (R - I) times the centre offset of odd sizes).
 * Each level optimises (t, angle * rho), rho the RMS distance of the level's
 * voxels from its centre, so both kinds of parameter move voxels on the same
 * scale. */
srwcr_status srwcr_rigid_register(srwcr_ctx* ctx, float* mu_dev_inout, int n_levels,
                                  const srwcr_lbfgs_opts* opts, srwcr_report* report);

/* ------------------------------------------------------------------------
 * Batched form: many pairs (contexts) of uneven sizes evaluated and
 * registered together.  The paper treats one pair at a time; this is a
 * throughput form of the same method.  Each phase of an evaluation (clear,
 * fused warp + statistics, per-region finalisation, value reduction,
 * per-plane contraction of the gradient tables, adjoint) is ONE launch over
 * every (pair, tile) work item, so a batched
 * value+gradient costs a handful of launches whatever the number of pairs,
 * and can be replayed from a CUDA graph.
 *
 * The batch owns packed device buffers: c and g (float32, pair i at
 * offsets[i] .. offsets[i] + n_params[i], each pair's layout as for
 * srwcr_value) and D (n_pairs doubles).  It reads each member context's
 * images and statistics and writes into that context's accumulators and
 * tables at `level`: while the batch exists its contexts must stay alive,
 * must not be re-tuned (srwcr_autotune), and must not run work of their own
 * at that level concurrently with the batch.  After a batched call, a
 * member's srwcr_backward needs a fresh srwcr_forward. */
typedef struct srwcr_batch srwcr_batch;

typedef struct {
  int n_pairs;
  int launches_per_eval;  /* kernels in one batched value+gradient */
  int64_t n_params_total; /* floats in the packed c and g buffers */
  int64_t n_voxels_total;
  int64_t work_items;     /* (pair, tile) items of one fused-kernel launch */
  int64_t launches;       /* kernels queued by this batch so far */
  int finalize_lanes;     /* lanes per spatial bin in the batched
                             finalisation (the first pair's setting, else
                             chosen over all pairs) */
} srwcr_batch_desc;

/* Build a batch over ctxs[0..n_pairs-1] at pyramid level `level`.  All
 * contexts must be on the current device, share ndim and storage, and run
 * that level on the row-parallel kernels (srwcr_level_desc.kernel_path = 1).
 * stream: cudaStream_t for all batch work; NULL = a stream the batch creates
 * (graph capture needs a stream other than the legacy default).  c and g
 * start at zero.  Errors: SRWCR_EINVAL, SRWCR_ENOMEM, SRWCR_ECUDA. */
srwcr_status srwcr_batch_create(srwcr_ctx* const* ctxs, int n_pairs, int level, void* stream,
                                srwcr_batch** out);

/* As srwcr_batch_create, with pair i at pyramid level levels[i] (pairs at
 * different levels, e.g. the coarse stage of one registration beside the
 * fine stage of another, share the same launches).  Each pair's level must
 * run on the row-parallel kernels. */
srwcr_status srwcr_batch_create_levels(srwcr_ctx* const* ctxs, const int* levels, int n_pairs,
                                       void* stream, srwcr_batch** out);
void srwcr_batch_destroy(srwcr_batch* b);
srwcr_status srwcr_batch_info(const srwcr_batch* b, srwcr_batch_desc* out);

/* offsets: n_pairs + 1 entries (may be NULL); n_params: n_pairs entries
 * (may be NULL). */
srwcr_status srwcr_batch_layout(const srwcr_batch* b, int64_t* offsets, int64_t* n_params);

/* Device pointers of the packed buffers (owned by the batch). */
srwcr_status srwcr_batch_buffers(srwcr_batch* b, float** c_dev, float** g_dev, double** D_dev);

/* Queue D_i and dD_i/dc_i for every pair at the coefficients in the packed c
 * buffer (results in D and g) without synchronising.  use_graph != 0 replays
 * a CUDA graph of the phases, captured on the first such call. */
srwcr_status srwcr_batch_value_and_grad(srwcr_batch* b, int use_graph);

/* Synchronise the batch stream; D_host (n_pairs doubles, may be NULL)
 * receives D. */
srwcr_status srwcr_batch_sync(srwcr_batch* b, double* D_host);

/* Single-level L-BFGS (Sec. II-F, the method of srwcr_register) for every
 * pair at once, from the coefficients in the packed c buffer, with
 * opts->max_iter[level] iterations at most (each pair's own level).  The optimiser state lives on
 * the device and each round (one batched evaluation plus one decision
 * kernel) is the same launch sequence for every pair, replayed from a CUDA
 * graph when use_graph != 0; pairs that stop drop out of later rounds.  On
 * return c holds each pair's last accepted point, g its gradient and D its
 * value.  Per-pair outputs (n_pairs entries each, any may be NULL):
 * iterations, evaluations, final value, srwcr_status (SRWCR_OK when the value
 * was stable over the window or the gradient vanished, SRWCR_ENOTCONVERGED
 * at the iteration limit, SRWCR_ELINESEARCH when the line search failed).
 * Returns SRWCR_ENUMERIC if some pair's value was not finite at its start,
 * SRWCR_EINVAL for bad options (stable_window must be below 64; the
 * bending-energy penalty is not supported here: penalty_weight must be 0). */
srwcr_status srwcr_batch_register(srwcr_batch* b, const srwcr_lbfgs_opts* opts, int use_graph,
                                  int* iterations, int* evaluations, double* final_value,
                                  int* status);

#ifdef __cplusplus
}
#endif

#endif /* SRWCR_H */
