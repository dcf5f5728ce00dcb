"""Rigid-model SRWCR -- TEST INFRASTRUCTURE ONLY.

The paper pre-aligns its CT/PET pairs by a rigid registration with the same
measure (Sec. III-D).  The rigid model restated here rotates about the image
centre x_c = (N - 1) / 2 (voxel units) and then translates:

    T(x) = R (x - x_c) + x_c + t,

3-D parameters mu = (t_x, t_y, t_z, alpha, beta, gamma) with
R = Rz(gamma) Ry(beta) Rx(alpha) (rotations about the fixed x, y, z axes in
that order); 2-D mu = (t_x, t_y, theta).  The value is Eq. (9) with B(x) =
M(T(x)) (the C oracle's warp in its rigid mode); the gradient is the chain
rule of Eq. (16) with dT/dmu in place of the FFD basis:

    dD/dmu_i = sum_x dD/dB(x) * grad M(T(x)) . dT/dmu_i(x),

dD/dB from Eq. (27), dT/dt_k = e_k, dT/dangle = (dR/dangle)(x - x_c).
Plain NumPy in FP64 over the C oracle's per-voxel quantities.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import Geometry, Stats, _d, dD_dB_image, lib, value, warp


def rigid_geometry(geo: Geometry) -> Geometry:
    return dataclasses.replace(geo, rigid=True)


def n_params(ndim: int) -> int:
    return 6 if ndim == 3 else 3


def matrix(ndim: int, mu) -> np.ndarray:
    """R of the rigid model (3 x 3; the 2-D rotation in the upper-left block)."""
    mu = np.ascontiguousarray(mu, np.float64)
    out = np.zeros(9)
    lib().orc_rigid_matrix(int(ndim), _d(mu), _d(out))
    return out.reshape(3, 3)


def matrix_derivatives(ndim: int, mu) -> list:
    """dR/d(angle) for each angle of mu, from the elementary rotations."""
    mu = np.asarray(mu, np.float64)
    if ndim == 2:
        th = mu[2]
        d = np.zeros((3, 3))
        d[:2, :2] = [[-np.sin(th), -np.cos(th)], [np.cos(th), -np.sin(th)]]
        return [d]
    a, b, g = mu[3], mu[4], mu[5]
    ca, sa, cb, sb, cg, sg = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(g), np.sin(g)
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    dRx = np.array([[0, 0, 0], [0, -sa, -ca], [0, ca, -sa]])
    dRy = np.array([[-sb, 0, cb], [0, 0, 0], [-cb, 0, -sb]])
    dRz = np.array([[-sg, -cg, 0], [cg, -sg, 0], [0, 0, 0]])
    return [Rz @ Ry @ dRx, Rz @ dRy @ Rx, dRz @ Ry @ Rx]


def _centred_grid(geo: Geometry) -> np.ndarray:
    """(N, 3) voxel coordinates minus the centre, x fastest."""
    nx, ny, nz = geo.dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    for d in range(3):
        q[:, d] -= 0.5 * (geo.dims[d] - 1) if d < geo.ndim else q[:, d]
    return q


def value_rigid(geo: Geometry, A, M, mu) -> Stats:
    return value(rigid_geometry(geo), A, M, np.ascontiguousarray(mu, np.float64))


def gradient_rigid(geo: Geometry, A, M, mu, st: Stats) -> np.ndarray:
    g_r = rigid_geometry(geo)
    mu = np.ascontiguousarray(mu, np.float64)
    G = dD_dB_image(g_r, A, M, mu, st)
    _, gM = warp(g_r, M, mu)
    nd = geo.ndim
    out = np.zeros(n_params(nd))
    for k in range(nd):
        out[k] = np.sum(G * gM[:, k])
    q = _centred_grid(geo)
    for i, dR in enumerate(matrix_derivatives(nd, mu)):
        v = q @ dR.T                      # (dR/dangle) (x - x_c) per voxel
        out[nd + i] = np.sum(G * np.sum(gM[:, :nd] * v[:, :nd], axis=1))
    return out


def value_and_grad_rigid(geo: Geometry, A, M, mu):
    st = value_rigid(geo, A, M, mu)
    return st.D, gradient_rigid(geo, A, M, mu, st), st


def to_ffd(geo: Geometry, mu) -> np.ndarray:
    """FFD coefficients whose cubic B-spline reproduces the rigid
    displacement: node j of an axis sits at (j - 1) delta, and the
    displacement R (p - x_c) + x_c + t - p is affine, which the uniform cubic
    B-spline reproduces exactly from its values at the nodes."""
    nd = geo.ndim
    R = matrix(nd, mu)
    nodes = [(geo.dims[d] - 1) // geo.ffd_spacing[d] + 4 for d in range(nd)]
    axes = [(np.arange(nodes[d]) - 1.0) * geo.ffd_spacing[d] for d in range(nd)]
    if nd == 2:
        py, px = np.meshgrid(axes[1], axes[0], indexing="ij")
        p = np.stack([px, py, np.zeros_like(px)], axis=-1)
    else:
        pz, py, px = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        p = np.stack([px, py, pz], axis=-1)
    ctr = np.array([0.5 * (geo.dims[d] - 1) if d < nd else 0.0 for d in range(3)])
    t = np.array([mu[d] if d < nd else 0.0 for d in range(3)])
    u = (p - ctr) @ R.T + ctr + t - p
    return np.moveaxis(u[..., :nd], -1, 0).copy()
