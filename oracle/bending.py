"""Bending energy of the FFD displacement -- TEST INFRASTRUCTURE ONLY.

The cost of Eq. (1) adds w_p * C_p, C_p being the bending energy of the
deformation field (Sec. II-F; the paper takes it from its ref. [26]).  The
definition restated here is the thin-plate bending energy of the displacement
u = T(x) - x, averaged over the image box Omega = prod_d [0, N_d - 1] (voxel
units):

    C_p = 1/|Omega| * integral over Omega of
          sum_k sum_{i,j} (d^2 u_k / dx_i dx_j)^2 dx,

the sum over ordered pairs (i, j), so each mixed derivative counts twice.  u
is the tensor-product cubic B-spline of Eq. (17), node j of an axis at
(j - 1) * delta.  This module evaluates the second derivatives of u at
4-point Gauss-Legendre nodes inside every knot interval of every axis (the
integrand is a polynomial of degree <= 6 per axis on each cell, so the
quadrature is exact) and sums them; the gradient is the same sum
differentiated term by term.  Plain NumPy in FP64.
"""
from __future__ import annotations

import numpy as np

_GX, _GW = np.polynomial.legendre.leggauss(4)


def _piece(l: int, t: np.ndarray, order: int) -> np.ndarray:
    """Piece l of the uniform cubic B-spline (Eq. 8) or its t-derivatives."""
    u = 1.0 - t
    if order == 0:
        return [u ** 3 / 6.0, (3 * t ** 3 - 6 * t ** 2 + 4) / 6.0,
                (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6.0, t ** 3 / 6.0][l]
    if order == 1:
        return [-(u ** 2) / 2.0, (9 * t ** 2 - 12 * t) / 6.0,
                (-9 * t ** 2 + 6 * t + 3) / 6.0, t ** 2 / 2.0][l]
    return [u, 3 * t - 2, -3 * t + 1, t][l]


def axis_quadrature(n: int, delta: int, n_nodes: int):
    """Gauss points and weights over [0, n-1] and, per point, the basis of
    every node: Phi[order][point][node] with derivatives in voxel units."""
    xs, ws = [], []
    p = 0
    while p * delta < n - 1:
        a, b = p * delta, min((p + 1) * delta, n - 1)
        xs.append(0.5 * (b - a) * _GX + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * _GW)
        p += 1
    x = np.concatenate(xs)
    w = np.concatenate(ws)
    phi = np.zeros((3, x.size, n_nodes))
    cell = np.floor(x / delta).astype(int)
    t = x / delta - cell
    rows = np.arange(x.size)
    for order in range(3):
        for l in range(4):
            phi[order, rows, cell + l] = _piece(l, t, order) / float(delta) ** order
    return w, phi


def _setup(dims, spacing, ndim):
    nodes = [(dims[d] - 1) // spacing[d] + 4 for d in range(ndim)]
    quad = [axis_quadrature(dims[d], spacing[d], nodes[d]) for d in range(ndim)]
    vol = float(np.prod([dims[d] - 1 for d in range(ndim)]))
    return quad, vol


def _terms(ndim):
    """(derivative orders per axis (x, y[, z]), multiplicity) of the integrand."""
    if ndim == 2:
        return [((2, 0), 1.0), ((0, 2), 1.0), ((1, 1), 2.0)]
    return [((2, 0, 0), 1.0), ((0, 2, 0), 1.0), ((0, 0, 2), 1.0),
            ((1, 1, 0), 2.0), ((1, 0, 1), 2.0), ((0, 1, 1), 2.0)]


def _eval(ck, quad, orders):
    """A derivative of one component at the tensor quadrature grid."""
    if len(quad) == 2:
        (_, px), (_, py) = quad
        return np.einsum("yb,xa,ba->yx", py[orders[1]], px[orders[0]], ck, optimize=True)
    (_, px), (_, py), (_, pz) = quad
    return np.einsum("zc,yb,xa,cba->zyx", pz[orders[2]], py[orders[1]], px[orders[0]], ck,
                     optimize=True)


def _adjoint(field, quad, orders):
    if len(quad) == 2:
        (_, px), (_, py) = quad
        return np.einsum("yx,yb,xa->ba", field, py[orders[1]], px[orders[0]], optimize=True)
    (_, px), (_, py), (_, pz) = quad
    return np.einsum("zyx,zc,yb,xa->cba", field, pz[orders[2]], py[orders[1]], px[orders[0]],
                     optimize=True)


def _weights(quad):
    ws = [w for w, _ in quad]
    if len(ws) == 2:
        return np.einsum("y,x->yx", ws[1], ws[0])
    return np.einsum("z,y,x->zyx", ws[2], ws[1], ws[0])


def bending_energy(dims, spacing, c: np.ndarray, grad: bool = False):
    """C_p (and dC_p/dc) for coefficients c of shape (d, [nz,] ny, nx)."""
    c = np.asarray(c, np.float64)
    ndim = c.shape[0]
    quad, vol = _setup(dims, spacing, ndim)
    W = _weights(quad)
    E = 0.0
    g = np.zeros_like(c) if grad else None
    for k in range(ndim):
        for orders, mult in _terms(ndim):
            f = _eval(c[k], quad, orders)
            E += mult * float(np.sum(W * f * f))
            if grad:
                g[k] += (2.0 * mult / vol) * _adjoint(W * f, quad, orders)
    return (E / vol, g) if grad else E / vol
