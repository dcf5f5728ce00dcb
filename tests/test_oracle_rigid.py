"""Pins of the oracle's rigid model (pre-alignment with the same measure,
Sec. III-D): T(x) = R (x - x_c) + x_c + t about the image centre.

* The rotation convention is pinned to SciPy's extrinsic x-y-z Euler angles
  and the warp to SciPy's map_coordinates at SciPy-rotated positions;
* zero parameters are the identity (the pinned FFD value at c = 0);
* a pure translation equals the FFD with constant coefficients (the B-spline
  partition of unity);
* a quarter turn about z maps the voxel lattice onto itself, so the value
  equals that of the index-permuted moving image;
* the chain-rule gradient equals central differences;
* FFD coefficients sampled from the rigid displacement at the control nodes
  reproduce the rigid displacement at every voxel (affine reproduction).
"""
import numpy as np
import pytest
from scipy import ndimage
from scipy.spatial.transform import Rotation

import oracle
from oracle import rigid
import synth
from test_oracle_pins import TINY, random_case

PROBS = [TINY[0], TINY[1], TINY[3]]


def random_mu(ndim, seed, t_sig=0.7, a_sig=0.08):
    rng = np.random.default_rng(seed)
    if ndim == 3:
        return np.concatenate([rng.normal(0, t_sig, 3), rng.normal(0, a_sig, 3)])
    return np.concatenate([rng.normal(0, t_sig, 2), rng.normal(0, a_sig, 1)])


def scipy_positions(prob, mu):
    """T(x) for every voxel from SciPy's rotation, (ndim, N) in x, y, z order."""
    nd = prob.ndim
    grids = np.meshgrid(*[np.arange(prob.dims[d]) for d in reversed(range(nd))], indexing="ij")
    pts = np.stack([g.ravel() for g in reversed(grids)], axis=1).astype(np.float64)  # x, y[, z]
    ctr = np.array([0.5 * (prob.dims[d] - 1) for d in range(nd)])
    if nd == 3:
        R = Rotation.from_euler("xyz", mu[3:6]).as_matrix()
    else:
        R = Rotation.from_euler("z", mu[2]).as_matrix()[:2, :2]
    return ((pts - ctr) @ R.T + ctr + mu[:nd]).T, pts.T


@pytest.mark.parametrize("prob", PROBS)
def test_rigid_displacement_matches_scipy_rotation(oracle_lib, prob):
    geo = rigid.rigid_geometry(oracle.Geometry.from_problem(prob))
    mu = random_mu(prob.ndim, 3)
    T, pts = scipy_positions(prob, mu)
    for i in np.random.default_rng(4).choice(pts.shape[1], 20, replace=False):
        xyz = [int(pts[d, i]) if d < prob.ndim else 0 for d in range(3)]
        u = oracle.displacement(geo, mu, *xyz)
        assert np.allclose(u[:prob.ndim], T[:, i] - pts[:, i], atol=1e-12)


@pytest.mark.parametrize("prob", PROBS)
def test_rigid_warp_matches_scipy_map_coordinates(oracle_lib, prob):
    geo = rigid.rigid_geometry(oracle.Geometry.from_problem(prob))
    mu = random_mu(prob.ndim, 5, t_sig=1.5, a_sig=0.2)
    _, M, _ = random_case(prob, 6)
    B, _ = oracle.warp(geo, M, mu)
    T, _ = scipy_positions(prob, mu)
    coords = T[::-1]  # map_coordinates wants (z, y, x)
    ref = ndimage.map_coordinates(M.reshape(prob.image_shape), coords, order=1, mode="nearest")
    assert np.allclose(B, ref, atol=1e-11)


@pytest.mark.parametrize("prob", PROBS)
def test_zero_parameters_are_the_identity(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, _ = random_case(prob, 7)
    a = rigid.value_rigid(geo, A, M, np.zeros(rigid.n_params(prob.ndim)))
    b = oracle.value(geo, A, M, np.zeros(prob.coef_shape))
    assert a.D == b.D


@pytest.mark.parametrize("prob", PROBS)
def test_translation_equals_constant_ffd_coefficients(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, _ = random_case(prob, 8)
    mu = random_mu(prob.ndim, 9, t_sig=1.3)
    mu[prob.ndim:] = 0.0
    c = np.zeros(prob.coef_shape)
    for k in range(prob.ndim):
        c[k] = mu[k]
    a = rigid.value_rigid(geo, A, M, mu)
    b = oracle.value(geo, A, M, c)
    assert abs(a.D - b.D) < 1e-12


@pytest.mark.parametrize("shape", [(10, 10), (8, 8, 5)])
def test_quarter_turn_about_z_permutes_the_lattice(oracle_lib, shape):
    nd = len(shape)
    dims = shape if nd == 2 else shape
    prob = synth.problem(nd, dims, (4,) * nd, (2,) * nd, 8)
    geo = oracle.Geometry.from_problem(prob)
    A, M, _ = random_case(prob, 10)
    mu = np.zeros(rigid.n_params(nd))
    mu[-1] = np.pi / 2           # theta (2-D) or gamma (3-D)
    n = shape[0]
    img = M.reshape(prob.image_shape)
    # T(x, y) = (n - 1 - y, x): B[.., y, x] = M[.., x, n - 1 - y]
    B = np.empty_like(img)
    for y in range(n):
        for x in range(n):
            B[..., y, x] = img[..., x, n - 1 - y]
    a = rigid.value_rigid(geo, A, M, mu)
    b = oracle.value(geo, A, B.ravel(), np.zeros(prob.coef_shape))
    assert abs(a.D - b.D) < 1e-10


@pytest.mark.parametrize("prob", PROBS)
def test_rigid_gradient_matches_central_differences(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, _ = random_case(prob, 11)
    mu = random_mu(prob.ndim, 12)
    D, g, st = rigid.value_and_grad_rigid(geo, A, M, mu)
    scale = np.abs(g).max()
    assert scale > 0
    h = 1e-6
    for i in range(mu.size):
        mp, mm = mu.copy(), mu.copy()
        mp[i] += h
        mm[i] -= h
        fd = (rigid.value_rigid(geo, A, M, mp).D - rigid.value_rigid(geo, A, M, mm).D) / (2 * h)
        assert abs(fd - g[i]) <= 2e-4 * scale + 1e-4 * abs(fd), (i, fd, g[i])


@pytest.mark.parametrize("prob", PROBS)
def test_ffd_from_rigid_reproduces_the_rigid_displacement(oracle_lib, prob):
    g0 = oracle.Geometry.from_problem(prob)
    gr = rigid.rigid_geometry(g0)
    mu = random_mu(prob.ndim, 13, t_sig=2.0, a_sig=0.3)
    c = rigid.to_ffd(g0, mu)
    assert c.shape == tuple(prob.coef_shape)
    rng = np.random.default_rng(14)
    for _ in range(20):
        xyz = [int(rng.integers(prob.dims[d])) if d < prob.ndim else 0 for d in range(3)]
        assert np.allclose(oracle.displacement(g0, c, *xyz), oracle.displacement(gr, mu, *xyz),
                           atol=1e-11)
