"""Pins of the oracle's "moving image as A" form (Sec. II-E, Eqs. 20, 21).

With the warped moving image M(T(x)) as the binned model image A and the
fixed image F as the estimated image B:
* p(a, b, r) and D equal the dense brute force of the definition with the
  roles exchanged;
* at c = 0 the warp is the identity, so D equals the already pinned
  "M as B" value with the two images exchanged;
* the Eq. (21) gradient equals central differences of D and obeys the
  partition-of-unity shift rule;
* D = 0 when F is an exact function of an integer-valued moving image.
"""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import TINY, brute_force_D, random_case, scipy_warp


@pytest.mark.parametrize("prob", TINY)
def test_mas_a_joint_pdf_and_value_match_brute_force(prob):
    geo = oracle.Geometry.from_problem(prob)
    F, M, c = random_case(prob, 15)
    p, Z = oracle.joint_pdf_mas_a(geo, F, M, c)
    Aw = scipy_warp(prob, M, c)
    p_ref, Z_ref, D_ref = brute_force_D(geo, Aw, F)
    assert abs(Z - prob.n_voxels) < 1e-9 * prob.n_voxels
    assert np.allclose(p, p_ref, atol=1e-15, rtol=1e-10)
    st = oracle.value_mas_a(geo, F, M, c)
    assert abs(st.D - D_ref) < 1e-12
    assert abs(st.D - st.D12) < 1e-12


@pytest.mark.parametrize("prob", TINY)
def test_identity_warp_exchanges_the_roles(prob):
    geo = oracle.Geometry.from_problem(prob)
    F, M, _ = random_case(prob, 17)
    c0 = np.zeros(prob.coef_shape)
    a = oracle.value_mas_a(geo, F, M, c0)
    b = oracle.value(geo, M, F, c0)       # M binned as A, F warped by the identity as B
    assert abs(a.D - b.D) < 1e-13
    assert np.allclose(a.cr, b.cr, atol=1e-13)


@pytest.mark.parametrize("prob", TINY)
def test_mas_a_gradient_matches_central_differences(prob):
    geo = oracle.Geometry.from_problem(prob)
    F, M, c = random_case(prob, 23)
    st = oracle.value_mas_a(geo, F, M, c)
    g = oracle.gradient_mas_a(geo, F, M, c, st)
    flat = c.ravel()
    rng = np.random.default_rng(1)
    h = 1e-6
    scale = np.abs(g).max()
    assert scale > 0
    for idx in rng.choice(flat.size, min(flat.size, 24), replace=False):
        cp, cm = flat.copy(), flat.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (oracle.value_mas_a(geo, F, M, cp.reshape(c.shape)).D
              - oracle.value_mas_a(geo, F, M, cm.reshape(c.shape)).D) / (2 * h)
        assert abs(fd - g.ravel()[idx]) <= 2e-4 * scale + 1e-4 * abs(fd), (idx, fd, g.ravel()[idx])


@pytest.mark.parametrize("prob", TINY[:2])
def test_mas_a_gradient_sum_is_derivative_of_global_shift(prob):
    geo = oracle.Geometry.from_problem(prob)
    F, M, c = random_case(prob, 29)
    st = oracle.value_mas_a(geo, F, M, c)
    g = oracle.gradient_mas_a(geo, F, M, c, st)
    h = 1e-6
    for k in range(prob.ndim):
        e = np.zeros_like(c)
        e[k] = 1.0
        fd = (oracle.value_mas_a(geo, F, M, c + h * e).D
              - oracle.value_mas_a(geo, F, M, c - h * e).D) / (2 * h)
        assert abs(fd - g[k].sum()) <= 1e-4 * np.abs(g[k]).sum() + 1e-9


def test_fixed_image_as_exact_function_of_integer_labels_gives_zero():
    prob = synth.problem(3, (10, 9, 8), (3, 3, 3), (2, 2, 2), 8)
    geo = oracle.Geometry.from_problem(prob)
    rng = np.random.default_rng(3)
    M = rng.integers(0, 8, prob.n_voxels).astype(np.float64)
    lut = rng.permutation(8).astype(np.float64)
    F = lut[M.astype(int)]
    st = oracle.value_mas_a(geo, F, M, np.zeros(prob.coef_shape))
    assert abs(st.D) < 1e-12
