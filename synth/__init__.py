"""Seeded synthetic image pairs and coefficient draws for SRWCR registration.

This module only *generates inputs*.  It holds none of the similarity
measure's arithmetic: deformations used to build moving images are evaluated
with SciPy's B-spline design matrices and resampled with
``scipy.ndimage.map_coordinates``; the measure itself (binning, Parzen
windows, moments, gradients) lives elsewhere.  Both the FP64 oracle tests and
the GPU tests/bench draw their inputs from here, so the two sides always see
the same arrays.

Workloads are stand-ins for the paper's data (Sec. III), which are not
available: a 2-D ellipse phantom (Sec. III-A style), a thoracic-CT-shaped
volume (Sec. III-B, DIR-Lab 4D-CT shape), an OCT-shaped layered volume
(Sec. III-C), PET/CT-shaped label/uptake pairs (Sec. III-D) and a large CT
volume.  All arrays are float32, x fastest: shape (nz, ny, nx) for 3-D and
(ny, nx) for 2-D.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np
from scipy import ndimage
from scipy.interpolate import BSpline

__all__ = [
    "Problem", "PairSpec", "CONFIGS", "problem", "make_pair", "coefficients",
    "n_ffd_nodes", "random_ffd_warp", "batch_specs", "downsample2", "grid_pair",
    "displacement_field", "inverse_displacement",
]


# ----------------------------------------------------------------------------
# Problem description (sizes only; no arithmetic of the measure)
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Problem:
    """Geometry of one SRWCR evaluation.

    dims          (nx, ny, nz), nz == 1 for 2-D
    ffd_spacing   integer control spacing delta per axis (voxels)
    sbin_intervals  K per axis: spatial bins are cubic B-splines with spacing
                  N/K (K+3 bins per axis).  0 means "spatial bins on the FFD
                  grid" (Sec. II-C: same nodes as the FFD).
    n_bins        number of intensity bins, L_eps + 1 (paper default 32)
    """
    ndim: int
    dims: Tuple[int, int, int]
    ffd_spacing: Tuple[int, int, int]
    sbin_intervals: Tuple[int, int, int]
    n_bins: int

    @property
    def n_voxels(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    @property
    def ffd_nodes(self) -> Tuple[int, int, int]:
        return tuple(n_ffd_nodes(self.dims[d], self.ffd_spacing[d]) if d < self.ndim else 1
                     for d in range(3))

    @property
    def n_params(self) -> int:
        n = self.ffd_nodes
        return self.ndim * n[0] * n[1] * n[2]

    @property
    def image_shape(self) -> Tuple[int, ...]:
        nx, ny, nz = self.dims
        return (ny, nx) if self.ndim == 2 else (nz, ny, nx)

    @property
    def coef_shape(self) -> Tuple[int, ...]:
        n = self.ffd_nodes
        return (self.ndim, n[1], n[0]) if self.ndim == 2 else (self.ndim, n[2], n[1], n[0])


def n_ffd_nodes(n: int, spacing: int) -> int:
    """Control nodes per axis for an image of n voxels: nodes at (j-1)*spacing,
    j = 0 .. floor((n-1)/spacing)+3, i.e. every node whose cubic support meets
    [0, n-1]."""
    return (n - 1) // spacing + 4


def problem(ndim, dims, ffd_spacing, sbin_intervals=(0, 0, 0), n_bins=32) -> Problem:
    dims = tuple(int(v) for v in dims) + (1,) * (3 - len(dims))
    fs = tuple(int(v) for v in ffd_spacing) + (1,) * (3 - len(ffd_spacing))
    sb = tuple(int(v) for v in sbin_intervals) + (0,) * (3 - len(sbin_intervals))
    if ndim == 2:
        dims = (dims[0], dims[1], 1)
        fs = (fs[0], fs[1], 1)
        sb = (sb[0], sb[1], 0)
    return Problem(ndim, dims, fs, sb, int(n_bins))


# The five workloads: sizes follow the configurations quoted with the
# headline metric.  C3 and C4 name no spatial/intensity bins: the paper's
# defaults apply (bins on the FFD grid, Sec. II-C; L_eps = 31, Sec. II-F).
CONFIGS = {
    "c1_2d_128": problem(2, (128, 128), (16, 16), (4, 4), 32),
    "c2_ct_256x256x96": problem(3, (256, 256, 96), (8, 8, 8), (8, 8, 4), 64),
    "c3_oct_160": problem(3, (160, 160, 160), (10, 10, 10), (0, 0, 0), 32),
    # C4 problems are per pair (uneven edges); see batch_specs().
    "c5_ct_512x512x300": problem(3, (512, 512, 300), (5, 5, 5), (16, 16, 8), 128),
}


# ----------------------------------------------------------------------------
# Random B-spline deformation used to *build* moving images
# ----------------------------------------------------------------------------
def _design(n: int, spacing: int, n_nodes: int) -> np.ndarray:
    """Dense (n, n_nodes) cubic B-spline design matrix from SciPy: basis j is
    centred at (j-1)*spacing (knots t_i = (i-3)*spacing)."""
    knots = (np.arange(n_nodes + 4, dtype=np.float64) - 3.0) * spacing
    x = np.arange(n, dtype=np.float64)
    return BSpline.design_matrix(x, knots, 3).toarray()


def _displacement(shape_zyx, spacing_xyz, coef) -> List[np.ndarray]:
    """Per-axis displacement fields (x, y[, z]) from control coefficients
    ``coef`` of shape (d, [nz,] ny, nx), via SciPy design matrices."""
    d = coef.shape[0]
    if d == 2:
        ny, nx = shape_zyx
        Bx = _design(nx, spacing_xyz[0], coef.shape[2])
        By = _design(ny, spacing_xyz[1], coef.shape[1])
        return [np.einsum("yj,ji,xi->yx", By, coef[k], Bx, optimize=True) for k in range(2)]
    nz, ny, nx = shape_zyx
    Bx = _design(nx, spacing_xyz[0], coef.shape[3])
    By = _design(ny, spacing_xyz[1], coef.shape[2])
    Bz = _design(nz, spacing_xyz[2], coef.shape[1])
    out = []
    for k in range(3):
        t = np.einsum("xi,kji->kjx", Bx, coef[k], optimize=True)
        t = np.einsum("yj,kjx->kyx", By, t, optimize=True)
        out.append(np.einsum("zk,kyx->zyx", Bz, t, optimize=True))
    return out


def random_ffd_warp(img: np.ndarray, spacing, sigma: float, rng: np.random.Generator,
                    chunk: int = 16) -> np.ndarray:
    """Backward-warp ``img`` by a random cubic B-spline deformation whose
    control displacements are iid N(0, sigma^2) voxels (trilinear resampling,
    edge clamp; SciPy map_coordinates)."""
    shape = img.shape
    d = img.ndim
    nodes = [n_ffd_nodes(shape[d - 1 - a], spacing[a]) for a in range(d)]  # x, y[, z]
    coef = rng.normal(0.0, sigma, size=(d,) + tuple(reversed(nodes)))
    if d == 2:
        ux, uy = _displacement(shape, spacing, coef)
        yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
        coords = np.stack([yy + uy, xx + ux])
        return ndimage.map_coordinates(img.astype(np.float64), coords, order=1,
                                       mode="nearest").astype(np.float32)
    nz, ny, nx = shape
    Bx = _design(nx, spacing[0], nodes[0])
    By = _design(ny, spacing[1], nodes[1])
    Bz = _design(nz, spacing[2], nodes[2])
    out = np.empty(shape, np.float32)
    src = img.astype(np.float64)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    # Contract x and y once; z in chunks to bound memory at large sizes.
    txy = []
    for k in range(3):
        t = np.einsum("xi,kji->kjx", Bx, coef[k], optimize=True)
        txy.append(np.einsum("yj,kjx->kyx", By, t, optimize=True))
    for z0 in range(0, nz, chunk):
        z1 = min(nz, z0 + chunk)
        u = [np.einsum("zk,kyx->zyx", Bz[z0:z1], txy[k], optimize=True) for k in range(3)]
        zz = np.arange(z0, z1)[:, None, None]
        coords = np.stack([zz + u[2], yy[None] + u[1], xx[None] + u[0]])
        out[z0:z1] = ndimage.map_coordinates(src, coords, order=1, mode="nearest")
    return out


# ----------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------
def _ellipses_2d(n: int, rng) -> np.ndarray:
    img = np.zeros((n, n), np.float64)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for _ in range(6):
        cx, cy = rng.uniform(0, n, 2)
        a, b = rng.uniform(8, 40, 2)
        th = rng.uniform(0, np.pi)
        val = rng.uniform(0, 1)
        dx, dy = xx - cx, yy - cy
        u = dx * np.cos(th) + dy * np.sin(th)
        v = -dx * np.sin(th) + dy * np.cos(th)
        img[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = val
    return img


def _ellipsoid(shape, c, r):
    nz, ny, nx = shape
    z = (np.arange(nz) - c[2])[:, None, None] / r[2]
    y = (np.arange(ny) - c[1])[None, :, None] / r[1]
    x = (np.arange(nx) - c[0])[None, None, :] / r[0]
    return x * x + y * y + z * z <= 1.0


def _ct_phantom(nx, ny, nz, rng, n_vessels=40) -> np.ndarray:
    """Thoracic-CT-shaped volume in HU: air, body, two lungs, vessels, noise."""
    shape = (nz, ny, nx)
    sx, sy, sz = nx / 256.0, ny / 256.0, nz / 96.0
    img = np.full(shape, -1000.0)
    c = (nx / 2.0, ny / 2.0, nz / 2.0)
    img[_ellipsoid(shape, c, (110 * sx, 80 * sy, 44 * sz))] = 0.0
    lungs = np.zeros(shape, bool)
    for side in (-1, 1):
        lc = (c[0] + side * 45 * sx, c[1], c[2])
        lr = (38 * sx, 55 * sy, 36 * sz)
        m = _ellipsoid(shape, lc, lr)
        lungs |= m
        img[m] = -850.0
    # Vessels: random straight tube segments, painted only inside the lungs.
    for _ in range(n_vessels):
        side = rng.choice([-1, 1])
        lc = np.array([c[0] + side * 45 * sx, c[1], c[2]])
        lr = np.array([38 * sx, 55 * sy, 36 * sz])
        p0 = lc + rng.uniform(-0.7, 0.7, 3) * lr
        p1 = lc + rng.uniform(-0.7, 0.7, 3) * lr
        rad = rng.uniform(1.0, 3.0)
        lo = np.maximum(np.floor(np.minimum(p0, p1) - rad - 1), 0).astype(int)
        hi = np.minimum(np.ceil(np.maximum(p0, p1) + rad + 2), [nx, ny, nz]).astype(int)
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                                 np.arange(lo[0], hi[0]), indexing="ij")
        pts = np.stack([xx, yy, zz], -1).astype(np.float64)
        seg = p1 - p0
        t = np.clip(((pts - p0) @ seg) / max(seg @ seg, 1e-12), 0.0, 1.0)
        dist = np.linalg.norm(pts - (p0 + t[..., None] * seg), axis=-1)
        sub = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        paint = (dist <= rad) & lungs[sub]
        img[sub][paint] = 40.0
    img += rng.normal(0.0, 20.0, shape)
    return np.clip(img, -1000.0, 1500.0)


def _oct_phantom(n, rng) -> np.ndarray:
    """OCT-shaped: 12 layers along y with smooth undulating boundaries,
    layer intensities U[0.2, 0.9], multiplicative Rayleigh speckle (0.5)."""
    nz, ny, nx = n, n, n
    xs = np.arange(nx)[None, :] / nx
    zs = np.arange(nz)[:, None] / nz
    base = np.linspace(0.1 * ny, 0.9 * ny, 12)
    bounds = []
    for k in range(12):
        b = np.full((nz, nx), base[k])
        for _ in range(3):
            amp = rng.uniform(0.5, 4.0 / 3.0)
            fx, fz = rng.uniform(0.5, 2.0, 2)
            ph = rng.uniform(0, 2 * np.pi)
            b = b + amp * np.sin(2 * np.pi * (fx * xs + fz * zs) + ph)
        bounds.append(b)
    vals = rng.uniform(0.2, 0.9, 13)
    y = np.arange(ny)[None, :, None].astype(np.float64)
    img = np.full((nz, ny, nx), vals[0])
    for k in range(12):
        img = np.where(y >= bounds[k][:, None, :], vals[k + 1], img)
    img = img * rng.rayleigh(0.5, img.shape)
    return img


def _label_phantom(n, rng) -> np.ndarray:
    """5-class nested random ellipsoids (labels 0..4)."""
    shape = (n, n, n)
    lab = np.zeros(shape, np.float64)
    centre = np.array([n / 2.0] * 3)
    scale = 0.45 * n
    for cls in range(1, 5):
        r = scale * (1.0 - 0.18 * (cls - 1)) * rng.uniform(0.8, 1.0, 3)
        cc = centre + rng.uniform(-0.05, 0.05, 3) * n
        lab[_ellipsoid(shape, cc, r)] = cls
    return lab


@dataclasses.dataclass
class PairSpec:
    name: str
    prob: Problem
    fixed: np.ndarray
    moving: np.ndarray
    storage: str = "f32"


def make_pair(name: str, seed: Optional[int] = None) -> PairSpec:
    """Fixed/moving pair for one named workload (C1, C2, C3, C5)."""
    prob = CONFIGS[name]
    idx = {"c1_2d_128": 1, "c2_ct_256x256x96": 2, "c3_oct_160": 3,
           "c5_ct_512x512x300": 5}[name]
    rng = np.random.default_rng(1000 * idx if seed is None else seed)
    if name == "c1_2d_128":
        f = _ellipses_2d(128, rng) + rng.normal(0, 0.02, (128, 128))
        fw = random_ffd_warp(f.astype(np.float32), (16, 16), 3.0, rng).astype(np.float64)
        ramp = (np.arange(128)[None, :] / 128.0)
        m = 1.0 - fw * fw + 0.1 * ramp
        return PairSpec(name, prob, f.astype(np.float32), m.astype(np.float32))
    if name == "c3_oct_160":
        f = _oct_phantom(160, rng)
        m = random_ffd_warp(f.astype(np.float32), (10, 10, 10), 3.0, rng)
        return PairSpec(name, prob, f.astype(np.float32), m.astype(np.float32))
    nx, ny, nz = prob.dims
    f = _ct_phantom(nx, ny, nz, rng)
    sp = prob.ffd_spacing if name == "c5_ct_512x512x300" else (8, 8, 8)
    m = random_ffd_warp(f.astype(np.float32), sp, 4.0, rng)
    m = np.clip(1.10 * m, -1000.0, 1500.0)
    return PairSpec(name, prob, f.astype(np.float32), m.astype(np.float32))


def batch_specs(n_pairs: int = 32, seed: int = 4000,
                edges=(64, 96, 128, 160, 192)) -> List[PairSpec]:
    """PET/CT-shaped batch: fixed = 5-class label volume, moving = per-class
    uptake U[1,100], Gaussian blur (FWHM 3 voxels), Poisson noise, random
    FFD warp (spacing 8, sigma 3).  Spatial bins on the FFD grid, 32 bins."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_pairs):
        e = int(rng.choice(edges))
        prob = problem(3, (e, e, e), (8, 8, 8), (0, 0, 0), 32)
        lab = _label_phantom(e, rng)
        uptake = rng.uniform(1.0, 100.0, 5)
        mv = uptake[lab.astype(int)]
        mv = ndimage.gaussian_filter(mv, 3.0 / 2.3548)
        mv = rng.poisson(mv).astype(np.float64)
        mv = random_ffd_warp(mv.astype(np.float32), (8, 8, 8), 3.0, rng)
        out.append(PairSpec(f"c4_pair{p:02d}_{e}", prob, lab.astype(np.float32),
                            mv.astype(np.float32), storage="bf16"))
    return out


def coefficients(prob: Problem, seed: int, sigma: float) -> np.ndarray:
    """Coefficient array (d, [nz,] ny, nx) float32, iid N(0, sigma^2) voxels."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, prob.coef_shape).astype(np.float32)


def downsample2(img: np.ndarray) -> np.ndarray:
    """2x box average per axis (floor sizes), used to build pyramid inputs."""
    if img.ndim == 2:
        ny, nx = (img.shape[0] // 2) * 2, (img.shape[1] // 2) * 2
        v = img[:ny, :nx].astype(np.float64)
        return (0.25 * (v[0::2, 0::2] + v[1::2, 0::2] + v[0::2, 1::2] + v[1::2, 1::2])).astype(np.float32)
    nz, ny, nx = [(s // 2) * 2 for s in img.shape]
    v = img[:nz, :ny, :nx].astype(np.float64)
    acc = np.zeros((nz // 2, ny // 2, nx // 2))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                acc += v[dz::2, dy::2, dx::2]
    return (acc / 8.0).astype(np.float32)


def small_pair(kind: str, dims, ffd_spacing, sigma: float, seed: int):
    """A fixed/moving pair of any size with one of the workload recipes:
    'ellipse' (2-D phantom, nonlinear intensity map with bias), 'ct' (3-D
    thoracic CT with 10% drift), 'oct' (layered speckle volume) or 'pet'
    (label volume vs. smoothed Poisson uptake).  dims = (nx, ny[, nz])."""
    rng = np.random.default_rng(seed)
    if kind == "ellipse":
        nx, ny = dims
        n = max(nx, ny)
        f = _ellipses_2d(n, rng)[:ny, :nx] + rng.normal(0, 0.02, (ny, nx))
        fw = random_ffd_warp(f.astype(np.float32), ffd_spacing, sigma, rng).astype(np.float64)
        m = 1.0 - fw * fw + 0.1 * (np.arange(nx)[None, :] / nx)
        return f.astype(np.float32), m.astype(np.float32)
    nx, ny, nz = dims
    if kind == "ct":
        f = _ct_phantom(nx, ny, nz, rng, n_vessels=8)
        m = np.clip(1.10 * random_ffd_warp(f.astype(np.float32), ffd_spacing, sigma, rng),
                    -1000.0, 1500.0)
    elif kind == "oct":
        n = max(nx, ny, nz)
        f = _oct_phantom(n, rng)[:nz, :ny, :nx]
        m = random_ffd_warp(f.astype(np.float32), ffd_spacing, sigma, rng)
    elif kind == "pet":
        n = max(nx, ny, nz)
        lab = _label_phantom(n, rng)[:nz, :ny, :nx]
        up = rng.uniform(1.0, 100.0, 5)[lab.astype(int)]
        up = rng.poisson(ndimage.gaussian_filter(up, 3.0 / 2.3548)).astype(np.float32)
        f, m = lab, random_ffd_warp(up, ffd_spacing, sigma, rng)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(f, np.float32), np.ascontiguousarray(m, np.float32)


# ----------------------------------------------------------------------------
# Synthetic grid experiment (known deformation)
# ----------------------------------------------------------------------------
def displacement_field(shape_zyx, spacing_xyz, coef) -> np.ndarray:
    """Displacement (d, [nz,] ny, nx) of cubic B-spline control coefficients
    ``coef`` (SciPy design matrices; node j at (j-1)*spacing)."""
    return np.stack(_displacement(tuple(shape_zyx), spacing_xyz, np.asarray(coef, np.float64)))


@dataclasses.dataclass
class GridPair:
    original: np.ndarray      # binary grid O
    warped: np.ndarray        # W(x) = O(x + v(x)) times a smooth bias field
    true_coef: np.ndarray     # control coefficients of v
    true_spacing: tuple       # their control spacing (x, y, z)


def grid_pair(n: int = 128, seed: int = 0, amplitude: float = 15.0, true_spacing: int = 16,
              period: int = 16, thickness: int = 2, bias: float = 0.3) -> GridPair:
    """Binary black-and-white 3-D grid (planes of ``thickness`` voxels every
    ``period`` along each axis) and a warped copy: control displacements iid
    uniform in [-amplitude, amplitude] voxels on a grid of spacing
    ``true_spacing``, trilinear resampling, then a smooth multiplicative bias
    field 1 + bias * (x/n - 1/2) + bias/2 * (y/n - 1/2)^2."""
    rng = np.random.default_rng(seed)
    idx = np.arange(n)
    line = (idx % period) < thickness
    O = (line[:, None, None] | line[None, :, None] | line[None, None, :]).astype(np.float64)
    nodes = n_ffd_nodes(n, true_spacing)
    coef = rng.uniform(-amplitude, amplitude, size=(3, nodes, nodes, nodes))
    u = displacement_field((n, n, n), (true_spacing,) * 3, coef)
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    coords = np.stack([zz + u[2], yy + u[1], xx + u[0]])
    W = ndimage.map_coordinates(O, coords, order=1, mode="nearest")
    xr, yr = xx / n - 0.5, yy / n - 0.5
    W = W * (1.0 + bias * xr + 0.5 * bias * yr * yr)
    return GridPair(O.astype(np.float32), W.astype(np.float32), coef, (true_spacing,) * 3)


def inverse_displacement(v: np.ndarray, iterations: int = 30) -> np.ndarray:
    """Displacement w of the inverse map of x -> x + v(x) on the voxel grid
    (x + w(x) + v(x + w(x)) = x), by the fixed-point iteration
    w <- -v(x + w) with trilinear interpolation of v (converges for smooth,
    moderate v)."""
    v = np.asarray(v, np.float64)
    d = v.shape[0]
    grids = np.meshgrid(*[np.arange(n) for n in v.shape[1:]], indexing="ij")  # z, y, x order
    w = -v.copy()
    for _ in range(iterations):
        # coordinates in (z, y, x) order; component k of w displaces axis k (x first)
        coords = np.stack([grids[a] + w[d - 1 - a] for a in range(d)])
        w = -np.stack([ndimage.map_coordinates(v[k], coords, order=1, mode="nearest")
                       for k in range(d)])
    return w


# ----------------------------------------------------------------------------
# Rigid pre-alignment (known rigid transform)
# ----------------------------------------------------------------------------
def rigid_rotation(mu) -> np.ndarray:
    """Rotation matrix of rigid parameters (x, y[, z] order): 3-D
    (t_x, t_y, t_z, alpha, beta, gamma) with extrinsic x-y-z Euler angles,
    2-D (t_x, t_y, theta); via SciPy's Rotation."""
    from scipy.spatial.transform import Rotation
    mu = np.asarray(mu, np.float64)
    if mu.size == 6:
        return Rotation.from_euler("xyz", mu[3:6]).as_matrix()
    return Rotation.from_euler("z", mu[2]).as_matrix()[:2, :2]


def rigid_pair(kind: str, dims, mu, seed: int, contrast: str = "inverted"):
    """Fixed phantom F (the 'ct' or 'ellipse' recipe of small_pair) and a
    moving image M = g(F o T^-1) such that M(T(x)) = g(F(x)) for the rigid
    map T(x) = R (x - x_c) + x_c + t, x_c = (N - 1) / 2: M is F resampled at
    T^-1(y) = R^T (y - x_c - t) + x_c (trilinear, clamped) and passed through
    the intensity map g (inverted contrast: a multi-modal pair)."""
    nd = len(dims)
    rng = np.random.default_rng(seed)
    if kind == "ct":
        nx, ny, nz = dims
        f = _ct_phantom(nx, ny, nz, rng, n_vessels=8) + rng.normal(0, 20.0, (nz, ny, nx))
    elif kind == "ellipse":
        nx, ny = dims
        f = _ellipses_2d(max(nx, ny), rng)[:ny, :nx] + rng.normal(0, 0.02, (ny, nx))
    else:
        raise ValueError(kind)
    R = rigid_rotation(mu)
    t = np.asarray(mu, np.float64)[:nd]
    ctr = np.array([0.5 * (dims[d] - 1) for d in range(nd)])
    grids = np.meshgrid(*[np.arange(dims[d]) for d in reversed(range(nd))], indexing="ij")
    pts = np.stack([g.ravel() for g in reversed(grids)], axis=1).astype(np.float64)  # x, y[, z]
    src = (pts - ctr - t) @ R + ctr            # R^T (y - x_c - t) + x_c, row-vector form
    coords = src[:, ::-1].T                    # (z, y, x) order for map_coordinates
    m = ndimage.map_coordinates(f, coords, order=1, mode="nearest").reshape(f.shape)
    if contrast == "inverted":
        m = m.max() - 0.5 * m
    return np.ascontiguousarray(f, np.float32), np.ascontiguousarray(m, np.float32)
