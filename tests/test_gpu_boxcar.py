"""GPU tests of the boxcar spatial distribution (Eq. 6): each voxel belongs
to one patch of a regular K-per-axis partition, patch floor(x K / N), with
weight 1; the rest of the method (Parzen window, Eqs. 9-12, gradient
Eqs. 16-21) is unchanged.  With the moving image as B it runs on the row
kernels (their per-axis spatial weights become 1, 0, 0, 0); with the moving
image as A, or a forced narrow tile, on the general per-voxel kernels.

Against the FP64 oracle (its boxcar geometry): D within 1e-5 relative,
gradient norm within 1e-4, elementwise within 1e-3 of the largest entry, for
both roles; a patch where B is a constant integer is counted degenerate;
one whole-domain patch gives the oracle's 1 - CR of Eq. (2).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D_RTOL, GNORM_RTOL, G_ELEM = 1e-5, 1e-4, 1e-3

CASES = [
    # patch counts that do not divide the sizes (ragged patches)
    ("ellipse_2d_ragged", "ellipse", synth.problem(2, (100, 77), (7, 7), (3, 2), 16), 1.5),
    ("ct_3d_ragged", "ct", synth.problem(3, (70, 45, 23), (6, 5, 4), (3, 2, 2), 24), 1.5),
    ("pet_labels", "pet", synth.problem(3, (48, 40, 36), (8, 8, 8), (4, 3, 3), 32), 2.0),
    ("ct_one_patch", "ct", synth.problem(3, (40, 33, 20), (5, 5, 5), (1, 1, 1), 32), 1.5),
]


def engine(prob, f, m, **kw):
    import paper_1804_05061_b300 as eng
    return eng.from_problem(prob, f, m, spatial="boxcar", **kw)


def oracle_case(prob, f, m, c, role):
    geo = oracle.Geometry.from_problem(prob, boxcar_patches=prob.sbin_intervals[:prob.ndim])
    A, M = oracle.prepare(f, m, prob.n_bins)
    if role == "mas_a":
        st = oracle.value_mas_a(geo, A, M, c)
        return st, oracle.gradient_mas_a(geo, A, M, c, st)
    st = oracle.value(geo, A, M, c)
    return st, oracle.gradient(geo, A, M, c, st)


@pytest.mark.parametrize("role", ["mas_b", "mas_a"])
@pytest.mark.parametrize("name,kind,prob,sig", CASES)
def test_boxcar_value_gradient_and_regions_match_oracle(name, kind, prob, sig, role):
    f, m = synth.small_pair(kind, prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 600)
    c = synth.coefficients(prob, 601, sig)
    e = engine(prob, f, m, role=role)
    lv = e.levels[0]
    assert lv.kernel_path == 1     # both roles run on the row kernels
    assert lv.sbins[:prob.ndim] == tuple(prob.sbin_intervals[:prob.ndim])
    assert lv.n_regions == int(np.prod(prob.sbin_intervals[:prob.ndim]))
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    stats, ndeg = e.region_stats()
    st, go = oracle_case(prob, f, m, c, role)
    assert abs(D - st.D) <= D_RTOL * abs(st.D), (D, st.D)
    assert ndeg == st.n_degenerate
    v = st.valid.astype(bool)
    assert np.allclose(stats[:, 0], st.pr, rtol=1e-6, atol=1e-15)
    ms = st.var_r[v] + st.mu_r[v] ** 2
    assert np.all(np.abs(stats[v, 1] - st.var_r[v]) <= 1e-6 * np.maximum(ms, 1.0))
    g = g.cpu().numpy().astype(np.float64)
    gn, gon = np.linalg.norm(g), np.linalg.norm(go)
    assert abs(gn - gon) <= GNORM_RTOL * gon, (gn, gon)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


@pytest.mark.parametrize("name,kind,prob,sig", CASES[:2])
def test_boxcar_on_the_general_kernels_matches_oracle(name, kind, prob, sig):
    # A 16-wide tile puts the level on the general per-voxel kernels.
    f, m = synth.small_pair(kind, prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 604)
    c = synth.coefficients(prob, 605, sig)
    tile = (16, 4, 4) if prob.ndim == 3 else (16, 8)
    e = engine(prob, f, m, tile=tile)
    assert e.levels[0].kernel_path == 0
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go = oracle_case(prob, f, m, c, "mas_b")
    assert abs(D - st.D) <= D_RTOL * abs(st.D), (D, st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


def test_boxcar_patch_with_constant_integer_b_is_degenerate():
    prob = synth.problem(2, (64, 40), (8, 8), (2, 1), 16)
    rng = np.random.default_rng(602)
    f = rng.uniform(0.0, 1.0, (40, 64)).astype(np.float32)
    m = rng.uniform(1.0, 7.0, (40, 64)).astype(np.float32)
    m[:, :32] = 0.0   # the image minimum: normalised B = 0 exactly in patch 0
    e = engine(prob, f, m)
    c = np.zeros(prob.coef_shape, np.float32)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    stats, ndeg = e.region_stats()
    st, go = oracle_case(prob, f, m, c, "mas_b")
    assert ndeg == st.n_degenerate == 1 and st.valid.tolist() == [0, 1]
    assert stats[0, 1] == 0.0 and stats[0, 3] == 0.0
    assert abs(D - st.D) <= D_RTOL * abs(st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)


def test_boxcar_registration_lowers_the_value():
    prob = synth.problem(3, (48, 40, 36), (8, 8, 8), (3, 3, 3), 32)
    f, m = synth.small_pair("ct", prob.dims, prob.ffd_spacing, 2.0, 603)
    e = engine(prob, f, m)
    c = e.zeros()
    D0 = e.value(c)
    o = e.default_opts()
    o.max_iter[0] = 15
    r = e.register(c, 1, o)
    assert r.final_value[0] < D0
    assert abs(e.value(c) - r.final_value[0]) <= 1e-12 * D0
