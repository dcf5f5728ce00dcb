"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each test ties one part of the oracle to a closed form, an invariant, a
textbook identity or an independent brute-force computation:

* Eq. (8) pieces equal the centred cubic B-spline and sum to one;
* Eq. (5) Parzen weights sum to one over the integer bins (Z = N, Sec. II-B);
* the FFD reproduces constant and linear displacement fields (Eq. 17 index
  convention), trilinear warping reproduces linear images;
* the joint PDF of Eq. (3) and the value of Eq. (9) equal a dense brute-force
  computation built from SciPy resampling and the law of total variance;
* CR in [0, 1], D in [0, 1], D = 0 under exact functional dependence;
* D is invariant to an affine map of the moving intensities (Sec. II);
* one whole-domain boxcar region (Eq. 6) gives 1 - CR of Eq. (2);
* the gradient of Eqs. (16)/(17)/(27) equals central finite differences and
  obeys the partition-of-unity shift rule.
"""
import numpy as np
import pytest

import oracle
import synth


# --- textbook forms written independently of the oracle -------------------
def centred_cubic_bspline(t):
    t = np.abs(np.asarray(t, np.float64))
    return np.where(t < 1, 2.0 / 3.0 - t * t + 0.5 * t ** 3,
                    np.where(t < 2, (2.0 - t) ** 3 / 6.0, 0.0))


def parzen_np(t):
    a = np.abs(np.asarray(t, np.float64))
    return np.where(a < 0.5, -1.8 * a * a - 0.1 * a + 1.0,
                    np.where(a < 1.0, 1.8 * a * a - 3.7 * a + 1.9, 0.0))


def scipy_warp(prob, M, c):
    """Independent backward warp: SciPy design-matrix FFD + map_coordinates."""
    from scipy import ndimage
    shape = prob.image_shape
    u = synth._displacement(shape, prob.ffd_spacing, np.asarray(c, np.float64))
    img = M.reshape(shape)
    if prob.ndim == 2:
        yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
        coords = np.stack([yy + u[1], xx + u[0]])
    else:
        zz, yy, xx = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
        coords = np.stack([zz + u[2], yy + u[1], xx + u[0]])
    return ndimage.map_coordinates(img, coords, order=1, mode="nearest").ravel()


def dense_spatial_weights(geo):
    """W[x, r] from the centred cubic B-spline at every (voxel, bin) pair."""
    nb = geo.sbins()
    per_axis = []
    for d in range(3):
        n = geo.dims[d]
        if d >= geo.ndim:
            per_axis.append(np.ones((n, 1)))
            continue
        spacing = geo.sbin_num[d] / geo.sbin_den[d]
        centres = (np.arange(nb[d]) - 1.0) * spacing
        per_axis.append(centred_cubic_bspline((np.arange(n)[:, None] - centres[None, :]) / spacing))
    wx, wy, wz = per_axis
    W = np.einsum("zk,yj,xi->zyxkji", wz, wy, wx)
    return W.reshape(geo.n_voxels, -1)


def brute_force_D(geo, A, B):
    """Dense p(a,b,r) (no sparsity shortcut) and D via the law of total variance."""
    nb = geo.n_bins
    bins = np.arange(nb, dtype=np.float64)
    W = dense_spatial_weights(geo)
    Ha = parzen_np(bins[None, :] - A[:, None])
    Hb = parzen_np(bins[None, :] - B[:, None])
    p = np.einsum("xr,xa,xb->rab", W, Ha, Hb)
    Z = p.sum()
    p = p / Z
    D = 0.0
    for r in range(p.shape[0]):
        pr = p[r].sum()
        if pr <= 0:
            continue
        q = p[r] / pr
        pa, pb = q.sum(1), q.sum(0)
        mu = (bins * pb).sum()
        var = (bins ** 2 * pb).sum() - mu ** 2
        if var <= 1e-6 * max(1.0, (bins ** 2 * pb).sum()):
            continue
        ok = pa > 0
        mua = (q[ok] * bins[None, :]).sum(1) / pa[ok]
        between = (pa[ok] * (mua - mu) ** 2).sum()
        D += pr * (1.0 - between / var)
    return p, Z, D


TINY = [
    synth.problem(3, (8, 8, 8), (3, 3, 3), (2, 2, 2), 8),
    synth.problem(2, (8, 8), (3, 3), (2, 2), 8),
    synth.problem(3, (9, 7, 6), (4, 4, 4), (0, 0, 0), 6),   # bins on the FFD grid, ragged
    synth.problem(2, (12, 10), (4, 4), (3, 2), 8),
]


def random_case(prob, seed, csig=0.8):
    rng = np.random.default_rng(seed)
    L = prob.n_bins - 1
    A = rng.uniform(0, L, prob.n_voxels)
    M = rng.uniform(0, L, prob.n_voxels)
    c = rng.normal(0, csig, prob.coef_shape)
    return A, M, c


# --- Eq. (8) and Eq. (5) --------------------------------------------------
def test_bspline_pieces_are_the_centred_cubic_and_sum_to_one(oracle_lib):
    for t in np.linspace(0, 1, 41):
        vals = [oracle.bspline(l, t) for l in range(4)]
        assert abs(sum(vals) - 1.0) < 1e-15
        for l in range(4):
            assert vals[l] >= -1e-18
            assert abs(vals[l] - centred_cubic_bspline(t + 1 - l)) < 1e-15
    assert np.allclose([oracle.bspline(l, 0.0) for l in range(4)], [1 / 6, 4 / 6, 1 / 6, 0])


def test_parzen_window_partition_of_unity_and_shape(oracle_lib):
    L = 31
    for t in np.random.default_rng(0).uniform(0, L, 500).tolist() + [0.0, 0.5, 1.0, 30.5, 31.0]:
        s = sum(oracle.parzen(b - t) for b in range(L + 1))
        assert abs(s - 1.0) < 1e-14, t
    assert oracle.parzen(0.0) == 1.0
    assert abs(oracle.parzen(0.5) - 0.5) < 1e-15 and abs(oracle.parzen(-0.5) - 0.5) < 1e-15
    assert oracle.parzen(1.0) == 0.0 and oracle.parzen(-1.0) == 0.0
    for t in np.linspace(-1.2, 1.2, 49):
        assert oracle.parzen(t) == oracle.parzen(-t)


def test_parzen_left_derivative_matches_difference_quotient(oracle_lib):
    eps = 1e-7
    for t in np.linspace(-1.5, 1.5, 301):
        num = (oracle.parzen(t) - oracle.parzen(t - eps)) / eps
        assert abs(num - oracle.parzen_dleft(t)) < 1e-5, t


# --- FFD (Eq. 17) and warping (Sec. II-F) ---------------------------------
@pytest.mark.parametrize("prob", TINY)
def test_ffd_reproduces_constant_and_linear_fields(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    nodes = prob.ffd_nodes
    rng = np.random.default_rng(3)
    const = rng.normal(size=prob.ndim)
    c = np.stack([np.full(prob.coef_shape[1:], const[k]) for k in range(prob.ndim)])
    # Linear: coefficient of node j along axis k = slope_k * (j - 1) * delta_k.
    slope = rng.normal(size=prob.ndim)
    lin = []
    for k in range(prob.ndim):
        pos = (np.arange(nodes[k]) - 1.0) * prob.ffd_spacing[k] * slope[k]
        shape = [1] * prob.ndim
        shape[prob.ndim - 1 - k] = nodes[k]
        lin.append(np.broadcast_to(pos.reshape(shape), prob.coef_shape[1:]))
    lin = np.stack(lin)
    for (x, y, z) in [(0, 0, 0), (prob.dims[0] - 1, prob.dims[1] - 1, prob.dims[2] - 1),
                      (3, 2, min(1, prob.dims[2] - 1))]:
        u = oracle.displacement(geo, c, x, y, z)
        assert np.allclose(u[:prob.ndim], const, atol=1e-13)
        u = oracle.displacement(geo, lin, x, y, z)
        assert np.allclose(u[:prob.ndim], slope * np.array([x, y, z])[:prob.ndim], atol=1e-12)


def test_trilinear_reproduces_linear_images_and_clamps(oracle_lib):
    prob = synth.problem(3, (7, 6, 5), (3, 3, 3), (0, 0, 0), 8)
    geo = oracle.Geometry.from_problem(prob)
    zz, yy, xx = np.meshgrid(*[np.arange(s) for s in prob.image_shape], indexing="ij")
    M = (0.5 * xx - 0.25 * yy + 0.75 * zz + 2.0).ravel().astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(50):
        y = rng.uniform([0, 0, 0], [6, 5, 4])
        v, g = oracle.interp(geo, M, y)
        assert abs(v - (0.5 * y[0] - 0.25 * y[1] + 0.75 * y[2] + 2.0)) < 1e-13
        assert np.allclose(g, [0.5, -0.25, 0.75], atol=1e-13)
    v, g = oracle.interp(geo, M, [-3.0, 2.5, 9.0])   # x below, z above the domain
    assert abs(v - (0.0 - 0.625 + 3.0 + 2.0)) < 1e-13
    assert g[0] == 0.0 and g[2] == 0.0 and abs(g[1] + 0.25) < 1e-13


@pytest.mark.parametrize("prob", TINY)
def test_warp_matches_scipy_resampling(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 11, 1.5)
    B, _ = oracle.warp(geo, M, c)
    assert np.allclose(B, scipy_warp(prob, M, c), atol=1e-11)


# --- Eqs. (3), (7), (9) against a dense brute force ------------------------
@pytest.mark.parametrize("prob", TINY)
def test_spatial_weights_match_dense_centred_bspline(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    W = dense_spatial_weights(geo)
    assert np.allclose(W.sum(1), 1.0, atol=1e-14)          # sum_r w(r, x) = 1
    nx, ny, _ = prob.dims
    for idx in range(prob.n_voxels):
        x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
        bins, w = oracle.spatial_weights(geo, x, y, z)
        assert len(bins) == 4 ** prob.ndim                   # 64 bins in 3-D (Sec. II-E)
        dense = np.zeros(W.shape[1])
        np.add.at(dense, bins, w)
        assert np.allclose(dense, W[idx], atol=1e-15)


@pytest.mark.parametrize("prob", TINY)
def test_joint_pdf_and_value_match_brute_force(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 5)
    p, Z = oracle.joint_pdf(geo, A, M, c)
    B = scipy_warp(prob, M, c)
    p_ref, Z_ref, D_ref = brute_force_D(geo, A, B)
    assert abs(Z - prob.n_voxels) < 1e-9 * prob.n_voxels   # Z = N
    assert abs(Z_ref - prob.n_voxels) < 1e-9 * prob.n_voxels
    assert np.allclose(p, p_ref, atol=1e-15, rtol=1e-10)
    st = oracle.stats_from_pdf(p, Z)
    assert abs(st.D - D_ref) < 1e-12
    assert abs(st.D - st.D12) < 1e-12                        # Eq. (9) = Eq. (12)


@pytest.mark.parametrize("name", ["c1_2d_128"])
def test_ranges_on_phantom(oracle_lib, name):
    pair = synth.make_pair(name)
    geo = oracle.Geometry.from_problem(pair.prob)
    A, M = oracle.prepare(pair.fixed, pair.moving, pair.prob.n_bins)
    for sig in (0.0, 2.0):
        c = synth.coefficients(pair.prob, 9, sig)
        st = oracle.value(geo, A, M, c)
        assert 0.0 <= st.D <= 1.0
        v = st.valid.astype(bool)
        assert np.all(st.cr[v] >= -1e-12) and np.all(st.cr[v] <= 1 + 1e-12)
        assert abs(st.Z - pair.prob.n_voxels) < 1e-8 * pair.prob.n_voxels
        assert abs(st.pr.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("prob", TINY[:2])
def test_exact_functional_dependence_gives_zero(oracle_lib, prob):
    """Integer A and B = f(A) (any map): every regional CR is 1, so D = 0."""
    rng = np.random.default_rng(2)
    L = prob.n_bins - 1
    A = rng.integers(0, L + 1, prob.n_voxels).astype(np.float64)
    A[0], A[1] = 0, L
    f = np.array([(3 * a + 1) % (L + 1) for a in range(L + 1)], np.float64)
    M = f[A.astype(int)]
    geo = oracle.Geometry.from_problem(prob)
    An = oracle.normalise(A.astype(np.float32), L).ravel()
    Mn = oracle.normalise(M.astype(np.float32), L).ravel()
    st = oracle.value(geo, An, Mn, np.zeros(prob.coef_shape))
    assert st.n_degenerate == 0
    assert abs(st.D) < 1e-12
    assert np.allclose(st.cr, 1.0, atol=1e-12)


def test_affine_intensity_invariance(oracle_lib):
    prob = synth.problem(3, (10, 9, 8), (4, 4, 4), (2, 2, 2), 16)
    geo = oracle.Geometry.from_problem(prob)
    rng = np.random.default_rng(4)
    F = rng.integers(0, 4000, prob.n_voxels).astype(np.float32) / 64.0
    Mraw = rng.integers(0, 4000, prob.n_voxels).astype(np.float32) / 64.0
    c = rng.normal(0, 1.0, prob.coef_shape)
    A = oracle.normalise(F, 15).ravel()
    D0 = oracle.value(geo, A, oracle.normalise(Mraw, 15).ravel(), c).D
    for alpha, beta in [(2.0, 3.0), (-1.0, 1.0), (-0.5, 7.0)]:
        Mt = (alpha * Mraw + beta).astype(np.float32)
        D1 = oracle.value(geo, A, oracle.normalise(Mt, 15).ravel(), c).D
        assert abs(D1 - D0) < 1e-12 * max(1.0, abs(D0)), (alpha, beta)


def test_whole_domain_boxcar_is_one_minus_classic_cr(oracle_lib):
    """Eq. (6) with one region spanning the image reduces SRWCR to 1 - CR
    (Eq. 2); CR here comes from the law of total variance instead."""
    prob = synth.problem(3, (12, 10, 9), (4, 4, 4), (0, 0, 0), 16)
    geo = oracle.Geometry.from_problem(prob, boxcar_patches=(1, 1, 1))
    assert geo.n_regions() == 1
    rng = np.random.default_rng(8)
    A = rng.uniform(0, 15, prob.n_voxels)
    M = np.clip(0.5 * A + rng.normal(0, 2.0, prob.n_voxels), 0, 15)
    st = oracle.value(geo, A, M, np.zeros(prob.coef_shape))
    bins = np.arange(16.0)
    H = parzen_np(bins[None, :] - A[:, None]).T @ parzen_np(bins[None, :] - M[:, None])
    H /= H.sum()
    pa, pb = H.sum(1), H.sum(0)
    mu = (bins * pb).sum()
    var = (bins ** 2 * pb).sum() - mu ** 2
    mua = (H * bins).sum(1)[pa > 0] / pa[pa > 0]
    cr = (pa[pa > 0] * (mua - mu) ** 2).sum() / var
    assert abs(st.D - (1.0 - cr)) < 1e-12


def test_degenerate_region_is_skipped(oracle_lib):
    """A boxcar patch where B is a constant integer has sigma_r^2 = 0: it is
    counted as degenerate and contributes nothing; the other patch gives
    its own p(r) (1 - CR)."""
    prob = synth.problem(2, (16, 8), (4, 4), (0, 0), 8)
    geo = oracle.Geometry.from_problem(prob, boxcar_patches=(2, 1, 1))
    rng = np.random.default_rng(12)
    A = rng.uniform(0, 7, (8, 16))
    M = rng.uniform(0, 7, (8, 16))
    M[:, :8] = 3.0
    st = oracle.value(geo, A.ravel(), M.ravel(), np.zeros(prob.coef_shape))
    assert st.n_degenerate == 1 and st.valid.tolist() == [0, 1]
    right = synth.problem(2, (8, 8), (4, 4), (0, 0), 8)
    geo_r = oracle.Geometry.from_problem(right, boxcar_patches=(1, 1, 1))
    st_r = oracle.value(geo_r, np.ascontiguousarray(A[:, 8:]).ravel(),
                        np.ascontiguousarray(M[:, 8:]).ravel(), np.zeros(right.coef_shape))
    assert abs(st.D - 0.5 * st_r.D) < 1e-12


def test_normalise_rejects_constant_image(oracle_lib):
    with pytest.raises(ValueError):
        oracle.normalise(np.ones(10, np.float32), 31)


# --- gradient: Eqs. (16), (17), (27) --------------------------------------
@pytest.mark.parametrize("prob", TINY)
def test_gradient_matches_central_differences(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 21)
    D, g, st = oracle.value_and_grad(geo, A, M, c)
    flat = c.ravel()
    rng = np.random.default_rng(0)
    h = 1e-6
    scale = np.abs(g).max()
    for idx in rng.choice(flat.size, min(flat.size, 24), replace=False):
        cp, cm = flat.copy(), flat.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (oracle.value(geo, A, M, cp.reshape(c.shape)).D
              - oracle.value(geo, A, M, cm.reshape(c.shape)).D) / (2 * h)
        assert abs(fd - g.ravel()[idx]) <= 2e-4 * scale + 1e-4 * abs(fd), (idx, fd, g.ravel()[idx])


@pytest.mark.parametrize("prob", TINY[:2])
def test_gradient_sum_is_derivative_of_global_shift(oracle_lib, prob):
    """B-spline partition of unity: adding t to every coefficient of
    component k translates T by t e_k, so sum_j g[k][j] = dD/dt."""
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 31)
    D, g, st = oracle.value_and_grad(geo, A, M, c)
    h = 1e-6
    for k in range(prob.ndim):
        e = np.zeros_like(c)
        e[k] = 1.0
        fd = (oracle.value(geo, A, M, c + h * e).D - oracle.value(geo, A, M, c - h * e).D) / (2 * h)
        assert abs(fd - g[k].sum()) <= 1e-4 * np.abs(g[k]).sum() + 1e-9


@pytest.mark.parametrize("prob", TINY)
def test_gradient_at_matches_full_gradient(oracle_lib, prob):
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 41)
    D, g, st = oracle.value_and_grad(geo, A, M, c)
    idx = np.arange(g.size)
    assert np.allclose(oracle.gradient_at(geo, A, M, c, st, idx), g.ravel(), atol=1e-15,
                       rtol=1e-11)


def test_gradient_chain_rule_from_per_voxel_derivative(oracle_lib):
    """g = sum_x G(x) dM/dy(T(x)) dT/dc: rebuild it from the per-voxel dD/dB
    and the SciPy design matrices (an independent Jacobian of Eq. 17)."""
    prob = TINY[0]
    geo = oracle.Geometry.from_problem(prob)
    A, M, c = random_case(prob, 51)
    D, g, st = oracle.value_and_grad(geo, A, M, c)
    G = oracle.dD_dB_image(geo, A, M, c, st)
    _, gradM = oracle.warp(geo, M, c)
    nodes = prob.ffd_nodes
    Bx = synth._design(prob.dims[0], prob.ffd_spacing[0], nodes[0])
    By = synth._design(prob.dims[1], prob.ffd_spacing[1], nodes[1])
    Bz = synth._design(prob.dims[2], prob.ffd_spacing[2], nodes[2])
    for k in range(3):
        field = (G * gradM[:, k]).reshape(prob.image_shape)
        gk = np.einsum("zyx,zc,yb,xa->cba", field, Bz, By, Bx)
        assert np.allclose(gk, g[k], atol=1e-14 * max(1, np.abs(g).max()) + 1e-16)


def test_parzen_derivative_convention_is_one_sided_inside_the_cell(oracle_lib):
    """dh/dkappa as used in Eq. (27): the moments m1(B) = sum_b b h(b-B) and
    m2(B) = sum_b b^2 h(b-B) must be differentiated inside [0, L] -- from
    above in B, and from below at the top bin B = L."""
    L = 15
    bins = np.arange(L + 1.0)
    eps = 1e-7
    for B in [0.0, 0.3, 0.5, 4.0, 7.25, 14.6, 14.999, 15.0]:
        for p in (1, 2):
            mom = lambda v: float((bins ** p * parzen_np(bins - v)).sum())
            if B >= L:
                num = (mom(B) - mom(B - eps)) / eps
            else:
                num = (mom(B + eps) - mom(B)) / eps
            ana = -sum(b ** p * oracle.parzen_dkappa(b, B, L) for b in bins)
            assert abs(num - ana) < 1e-5 * max(1.0, abs(ana)), (B, p, num, ana)
