"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 path): SRWCR value relative 1e-5; gradient norm relative
1e-4; gradient elementwise within 1e-3 of the largest entry (isolated voxels
whose warped intensity sits within FP32 rounding of an integer may take the
other one-sided Parzen derivative, Eq. 19); voxel-to-bin indices bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D_RTOL = 1e-5
GNORM_RTOL = 1e-4
G_ELEM = 1e-3


def engine_for(prob, fixed, moving, storage="f32", **kw):
    import paper_1804_05061_b300 as eng
    return eng.from_problem(prob, fixed, moving, storage=storage, **kw)


def oracle_eval(prob, fixed, moving, c, storage="f32", grad=True):
    geo = oracle.Geometry.from_problem(prob)
    A, M = oracle.prepare(fixed, moving, prob.n_bins, storage)
    st = oracle.value(geo, A, M, c)
    g = oracle.gradient(geo, A, M, c, st) if grad else None
    return st, g, geo, A, M


SMALL = [
    ("ellipse_2d_ragged", "ellipse", synth.problem(2, (100, 77), (7, 7), (3, 2), 16), 1.5),
    ("ct_3d_ragged", "ct", synth.problem(3, (70, 45, 23), (6, 5, 4), (3, 2, 2), 24), 1.5),
    ("oct_ffd_grid_bins", "oct", synth.problem(3, (41, 37, 29), (5, 5, 5), (0, 0, 0), 32), 1.0),
    ("ct_128_bins", "ct", synth.problem(3, (64, 48, 40), (5, 5, 5), (2, 2, 1), 128), 1.5),
    ("pet_labels", "pet", synth.problem(3, (48, 40, 36), (8, 8, 8), (0, 0, 0), 32), 2.0),
    # spacing 5 with the bins on the FFD grid (the paper's defaults): a
    # 32-voxel row meets up to 11 spatial x-bins (the 12-bin row kernels)
    ("ellipse_2d_spacing5", "ellipse", synth.problem(2, (100, 77), (5, 5), (0, 0), 16), 1.0),
]


@pytest.fixture(scope="module")
def small_cases():
    out = {}
    for i, (name, kind, prob, sig) in enumerate(SMALL):
        f, m = synth.small_pair(kind, prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 100 + i)
        c = synth.coefficients(prob, 200 + i, sig)
        out[name] = (prob, f, m, c)
    return out


@pytest.mark.parametrize("name", [s[0] for s in SMALL])
def test_value_gradient_and_regions_match_oracle(small_cases, name):
    prob, f, m, c = small_cases[name]
    e = engine_for(prob, f, m)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    stats, ndeg = e.region_stats()
    st, go, _, _, _ = oracle_eval(prob, f, m, c)
    assert abs(D - st.D) <= D_RTOL * abs(st.D), (D, st.D)
    assert ndeg == st.n_degenerate
    # p(r): FP32 products w*h summed exactly in fixed point -> ~1e-7 relative.
    assert np.allclose(stats[:, 0], st.pr, rtol=1e-6, atol=1e-15)
    # sigma_r^2 = E[b^2] - mu^2 is formed from FP32 per-voxel moments whose
    # rounding (~1e-7 of E[b^2]) survives the cancellation: compare on the
    # scale of E_r[b^2]; CR inherits that error divided by sigma_r^2.
    # The moment sums are fixed point with one quantum per level, so the
    # quantisation error of a region's sigma^2 is about (a few half quanta) /
    # W_r, W_r = p(r) Z its total weight: above the 1e-6 bar only for regions
    # whose support meets the image in a few voxels at B-spline weights near
    # 1e-3 per axis (p(r) ~ 1e-10, W_r ~ 1e-5 voxels).  Regions with p(r) <
    # 1e-8 are checked loosely and shown to hold a negligible share of D.
    v = st.valid.astype(bool)
    tiny = v & (st.pr < 1e-8)
    assert np.sum(st.pr[tiny] * (1.0 - st.cr[tiny])) <= 1e-6 * abs(st.D)
    assert np.all(np.abs(stats[tiny, 1] - st.var_r[tiny]) <= 1e-3 * np.maximum(st.var_r[tiny], 1.0))
    v = v & ~tiny
    ms = st.var_r[v] + st.mu_r[v] ** 2
    assert np.all(np.abs(stats[v, 1] - st.var_r[v]) <= 1e-6 * np.maximum(ms, 1.0))
    assert np.all(np.abs(stats[v, 2] - st.cr[v]) <= 1e-6 + 4e-6 * np.maximum(ms, 1.0) / st.var_r[v])
    g = g.cpu().numpy().astype(np.float64)
    gn, gon = np.linalg.norm(g), np.linalg.norm(go)
    assert abs(gn - gon) <= GNORM_RTOL * gon, (gn, gon)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


@pytest.mark.parametrize("name", ["ct_128_bins", "ellipse_2d_ragged", "pet_labels"])
def test_value_in_several_bin_passes_equals_one_pass(small_cases, name):
    # A tile whose fixed-image bins exceed bins_per_pass takes several passes
    # over its rows; every (region, bin) entry receives the same row sums.
    # With the same tile the value is bit-identical; a different tile (the
    # smaller histogram may allow a taller one) changes only the FP32
    # combination of the z-plane sums.
    prob, f, m, c = small_cases[name]
    e1 = engine_for(prob, f, m)
    e8 = engine_for(prob, f, m, bins_per_pass=8)
    assert e1.levels[0].kernel_path == 1 and e8.levels[0].kernel_path == 1
    ct = torch.from_numpy(c).cuda()
    D1, g1 = e1.value_and_grad(ct)
    D8, g8 = e8.value_and_grad(ct)
    s1, _ = e1.region_stats()
    s8, _ = e8.region_stats()
    if e1.levels[0].tile == e8.levels[0].tile:
        assert D8 == D1 and np.array_equal(s1, s8)
    assert abs(D8 - D1) <= 1e-6 * D1
    assert torch.allclose(g8, g1, rtol=1e-5, atol=1e-5 * float(g1.abs().max()))
    e8b = engine_for(prob, f, m, bins_per_pass=8, tile=e1.levels[0].tile)
    assert e8b.value(ct) == D1
    st, _, _, _, _ = oracle_eval(prob, f, m, c, grad=False)
    assert abs(D8 - st.D) <= D_RTOL * abs(st.D)


@pytest.mark.parametrize("name", ["ct_128_bins", "pet_labels", "ellipse_2d_ragged"])
def test_every_finalisation_lane_count_matches_oracle(small_cases, name):
    # G lanes per spatial bin: the bin lists of "ct_128_bins" take several
    # rounds at small G, those of "pet_labels" fit one.  Moment sums are exact
    # integers, so only the FP64 sum of S1 mu_r(a) changes order with G.
    prob, f, m, c = small_cases[name]
    ct = torch.from_numpy(c).cuda()
    st, go, _, _, _ = oracle_eval(prob, f, m, c)
    auto = engine_for(prob, f, m)
    assert auto.levels[0].finalize_lanes in (1, 2, 4, 8, 16, 32)
    D0, g0 = auto.value_and_grad(ct)
    s0, n0 = auto.region_stats()
    for lanes in (1, 2, 4, 8, 16, 32):
        e = engine_for(prob, f, m, finalize_lanes=lanes)
        assert e.levels[0].finalize_lanes == lanes
        D, g = e.value_and_grad(ct)
        s, n = e.region_stats()
        assert n == n0 == st.n_degenerate
        assert abs(D - D0) <= 1e-12 * abs(D0) and abs(D - st.D) <= D_RTOL * abs(st.D)
        assert np.allclose(s, s0, rtol=1e-12, atol=1e-12)
        assert torch.allclose(g, g0, rtol=1e-6, atol=1e-6 * float(g0.abs().max()))
        gn = np.linalg.norm(g.cpu().numpy().astype(np.float64))
        assert abs(gn - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)


def test_finalisation_lane_count_is_validated(small_cases):
    import paper_1804_05061_b300 as eng
    prob, f, m, _ = small_cases["pet_labels"]
    for bad in (3, 64, -1):
        with pytest.raises(eng.SrwcrError):
            engine_for(prob, f, m, finalize_lanes=bad)


EXPECTED_PATH = {"ellipse_2d_ragged": 1, "ct_3d_ragged": 1, "oct_ffd_grid_bins": 1,
                 "ct_128_bins": 1, "pet_labels": 1, "ellipse_2d_spacing5": 1}


@pytest.mark.parametrize("name", [s[0] for s in SMALL])
def test_kernel_path_selection(small_cases, name):
    prob, f, m, c = small_cases[name]
    assert engine_for(prob, f, m).levels[0].kernel_path == EXPECTED_PATH[name]


@pytest.mark.parametrize("name", ["ellipse_2d_ragged", "ct_3d_ragged", "ct_128_bins"])
def test_general_kernels_match_oracle(small_cases, name):
    """The per-voxel kernels (forced by a 16-wide tile) against the oracle."""
    prob, f, m, c = small_cases[name]
    tile = (16, 4, 4) if prob.ndim == 3 else (16, 8)
    e = engine_for(prob, f, m, tile=tile)
    assert e.levels[0].kernel_path == 0 and e.levels[0].tile[0] == 16
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, f, m, c)
    assert abs(D - st.D) <= D_RTOL * abs(st.D), (D, st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


@pytest.mark.parametrize("name", ["ellipse_2d_ragged", "oct_ffd_grid_bins", "ct_128_bins"])
def test_voxel_to_bin_indexing_is_bit_exact(small_cases, name):
    prob, f, m, c = small_cases[name]
    e = engine_for(prob, f, m)
    bins = e.debug_bins().cpu().numpy()
    geo = oracle.Geometry.from_problem(prob)
    A, _ = oracle.prepare(f, m, prob.n_bins)
    nx, ny, _ = prob.dims
    nbx, nby, _ = geo.sbins()
    idx = np.arange(prob.n_voxels)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    L = prob.n_bins - 1
    first = np.array([oracle.spatial_weights(geo, int(a), int(b), int(cc))[0][0]
                      for a, b, cc in zip(x, y, z)])
    assert np.array_equal(bins[:, 0], first % nbx)
    assert np.array_equal(bins[:, 1], (first // nbx) % nby)
    assert np.array_equal(bins[:, 2], first // (nbx * nby))
    assert np.array_equal(bins[:, 3], np.minimum(np.floor(A), L - 1).astype(np.int64))


@pytest.mark.parametrize("name", ["ellipse_2d_ragged", "ct_3d_ragged"])
def test_warp_matches_oracle(small_cases, name):
    prob, f, m, c = small_cases[name]
    e = engine_for(prob, f, m)
    B = e.debug_warp(torch.from_numpy(c).cuda()).cpu().numpy()
    geo = oracle.Geometry.from_problem(prob)
    _, M = oracle.prepare(f, m, prob.n_bins)
    Bo, _ = oracle.warp(geo, M, c)
    assert np.abs(B - Bo).max() <= 2e-5 * (prob.n_bins - 1)


def test_bf16_storage_matches_oracle_on_rounded_inputs(small_cases):
    prob, f, m, c = small_cases["pet_labels"]
    e = engine_for(prob, f, m, storage="bf16")
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, f, m, c, storage="bf16")
    assert abs(D - st.D) <= D_RTOL * abs(st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)


def test_value_is_deterministic(small_cases):
    prob, f, m, c = small_cases["ct_3d_ragged"]
    e = engine_for(prob, f, m)
    ct = torch.from_numpy(c).cuda()
    vals = [e.value_and_grad(ct)[0] for _ in range(3)]
    assert vals[0] == vals[1] == vals[2]


def test_value_only_equals_value_of_value_and_grad(small_cases):
    prob, f, m, c = small_cases["oct_ffd_grid_bins"]
    e = engine_for(prob, f, m)
    ct = torch.from_numpy(c).cuda()
    assert e.value(ct) == e.value_and_grad(ct)[0]


def test_host_buffer_entry_point_equals_device_entry_point(small_cases):
    prob, f, m, c = small_cases["ellipse_2d_ragged"]
    e = engine_for(prob, f, m)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    gh = np.zeros(c.size, np.float32)
    Dh = e.value_and_grad_host(np.ascontiguousarray(c.ravel()), gh)
    assert Dh == D
    assert np.allclose(gh, g.cpu().numpy().ravel(), rtol=1e-5, atol=1e-7 * np.abs(gh).max())


def test_host_buffer_entry_point_with_page_locked_buffers_replays_one_graph(small_cases):
    # Page-locked host buffers: the call is captured once per (level, buffers)
    # and replayed; results equal the device entry point's, a new buffer or a
    # re-tuned level is captured again, and a bad input is still reported.
    import paper_1804_05061_b300 as eng
    prob, f, m, c = small_cases["pet_labels"]   # a problem no other test autotunes
    e = engine_for(prob, f, m)
    ct = torch.from_numpy(c).cuda()
    D, g = e.value_and_grad(ct)
    cp = torch.from_numpy(np.ascontiguousarray(c.ravel())).pin_memory()
    gp = torch.zeros_like(cp).pin_memory()
    for _ in range(3):
        gp.zero_()
        assert e.value_and_grad_host(cp.numpy(), gp.numpy()) == D
        assert np.allclose(gp.numpy(), g.cpu().numpy().ravel(), rtol=1e-5,
                           atol=1e-7 * float(g.abs().max()))
    gp2 = torch.zeros_like(cp).pin_memory()
    assert e.value_and_grad_host(cp.numpy(), gp2.numpy()) == D
    # (the gradient's FP32 atomics make it reproducible to rounding only)
    assert np.allclose(gp2.numpy(), gp.numpy(), rtol=1e-5, atol=1e-7 * float(g.abs().max()))
    e.autotune(ct, reps=1)
    D2, _ = e.value_and_grad(ct)
    assert e.value_and_grad_host(cp.numpy(), gp.numpy()) == D2
    bad = cp.clone().pin_memory()
    bad[3] = float("nan")
    with pytest.raises(eng.SrwcrError, match="ENUMERIC"):
        e.value_and_grad_host(bad.numpy(), gp.numpy())
    assert e.value_and_grad_host(cp.numpy(), gp.numpy()) == D2


def test_host_buffer_entry_point_with_one_page_locked_buffer(small_cases):
    # A page-locked c with a pageable g: no graph (that needs both buffers
    # page-locked), c uploaded and checked through its device mapping, D
    # stored into mapped host memory; a pageable c with a page-locked g takes
    # the copy path.  Both equal the device entry point, and a non-finite c is
    # reported on either path.
    import paper_1804_05061_b300 as eng
    prob, f, m, c = small_cases["ct_3d_ragged"]
    e = engine_for(prob, f, m)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    g_ref = g.cpu().numpy().ravel()
    tol = 1e-7 * float(np.abs(g_ref).max())
    cp = torch.from_numpy(np.ascontiguousarray(c.ravel())).pin_memory()
    g_pageable = np.zeros(c.size, np.float32)
    assert e.value_and_grad_host(cp.numpy(), g_pageable) == D
    assert np.allclose(g_pageable, g_ref, rtol=1e-5, atol=tol)
    gp = torch.zeros_like(cp).pin_memory()
    c_pageable = np.ascontiguousarray(c.ravel()).copy()
    assert e.value_and_grad_host(c_pageable, gp.numpy()) == D
    assert np.allclose(gp.numpy(), g_ref, rtol=1e-5, atol=tol)
    bad = cp.clone().pin_memory()
    bad[5] = float("inf")
    with pytest.raises(eng.SrwcrError, match="ENUMERIC"):
        e.value_and_grad_host(bad.numpy(), g_pageable)
    assert e.value_and_grad_host(cp.numpy(), g_pageable) == D


def test_exact_functional_dependence_gives_zero_on_gpu():
    prob = synth.problem(3, (40, 36, 20), (5, 5, 5), (3, 3, 2), 16)
    rng = np.random.default_rng(3)
    A = rng.integers(0, 16, prob.image_shape).astype(np.float32)
    A.flat[0], A.flat[1] = 0, 15
    f = np.array([(5 * a + 2) % 16 for a in range(16)], np.float32)
    M = f[A.astype(int)]
    e = engine_for(prob, A, M)
    D = e.value(e.zeros())
    _, ndeg = e.region_stats()
    assert ndeg == 0
    assert abs(D) < 1e-7


def test_errors_are_reported_not_raised_as_crashes(small_cases):
    import paper_1804_05061_b300 as eng
    prob, f, m, c = small_cases["ellipse_2d_ragged"]
    with pytest.raises(eng.SrwcrError) as ei:
        engine_for(prob, np.ones_like(f), m)
    assert ei.value.status == 1
    e = engine_for(prob, f, m)
    bad = torch.from_numpy(c).cuda()
    bad.view(-1)[3] = float("nan")
    with pytest.raises(eng.SrwcrError) as ei:
        e.value(bad)
    assert ei.value.status == 4
    with pytest.raises(eng.SrwcrError):
        e.level_info(5)
    with pytest.raises(ValueError):
        e.value(torch.zeros(7, device="cuda"))
    # The context stays usable after a rejected call.
    D = e.value(torch.from_numpy(c).cuda())
    assert np.isfinite(D)


def test_caller_buffers_are_checked_before_the_library_sees_them(small_cases):
    # The C ABI takes plain pointers and reads or writes exactly the level's
    # coefficient count: the binding rejects a buffer of the wrong size,
    # dtype, device or layout (a buffer the library writes must be contiguous
    # itself) before any call, and the context stays usable.
    prob, f, m, c = small_cases["ct_3d_ragged"]
    e = engine_for(prob, f, m)
    ct = torch.from_numpy(c).cuda()
    n = ct.numel()
    D_ref, g_ref = e.value_and_grad(ct)
    f32, f64 = torch.float32, torch.float64
    short = torch.zeros(n - 1, device="cuda")
    strided = torch.zeros(2 * n, device="cuda")[::2]
    D_dev = torch.zeros((), dtype=f64, device="cuda")
    g_dev = torch.zeros(n, device="cuda")
    cases = [
        (TypeError, lambda: e.value(ct.cpu())),
        (TypeError, lambda: e.value(ct.double())),
        (ValueError, lambda: e.value(short)),
        (ValueError, lambda: e.value_and_grad(ct, out=short)),
        (TypeError, lambda: e.value_and_grad(ct, out=torch.zeros(n, dtype=f64, device="cuda"))),
        (ValueError, lambda: e.value_and_grad(ct, out=strided)),
        (ValueError, lambda: e.value_and_grad_async(strided, D_dev, g_dev)),
        (TypeError, lambda: e.value_and_grad_async(ct, torch.zeros((), dtype=f32, device="cuda"),
                                                   g_dev)),
        (ValueError, lambda: e.value_and_grad_async(ct, D_dev, short)),
        (ValueError, lambda: e.value_and_grad_host(np.zeros(n - 1, np.float32),
                                                   np.zeros(n, np.float32))),
        (TypeError, lambda: e.value_and_grad_host(c.ravel().astype(np.float32),
                                                  np.zeros(n, np.float64))),
        (ValueError, lambda: e.value_and_grad_host(c.ravel().astype(np.float32),
                                                   np.zeros(2 * n, np.float32)[::2])),
        (ValueError, lambda: e.value_and_grad_host(c.ravel().astype(np.float32),
                                                   _read_only(n))),
        (TypeError, lambda: e.forward(ct, torch.zeros((), dtype=f32, device="cuda"))),
        (TypeError, lambda: e.backward(ct, torch.ones(1, dtype=f64, device="cuda"), g_dev)),
        (ValueError, lambda: e.backward(ct, None, short)),
        (ValueError, lambda: e.bending_energy(ct, grad_into=short)),
        (ValueError, lambda: e.lbfgs_direction(g_dev, torch.zeros(2, n, device="cuda"),
                                               torch.zeros(2, n + 1, device="cuda"))),
        (ValueError, lambda: e.register(strided, 1)),
    ]
    for exc, call in cases:
        with pytest.raises(exc):
            call()
        torch.cuda.synchronize()
    D, g = e.value_and_grad(ct)
    assert D == D_ref
    assert float((g - g_ref).abs().max()) <= 1e-5 * float(g_ref.abs().max())
    # A non-contiguous input is passed as a contiguous copy where the library
    # only reads it.
    assert e.value(strided.copy_(ct.view(-1))) == D_ref


def _read_only(n):
    a = np.zeros(n, np.float32)
    a.setflags(write=False)
    return a


# ---------------------------------------------------------------------------
# Full-size workloads
# ---------------------------------------------------------------------------
def test_c1_full_value_and_gradient():
    pair = synth.make_pair("c1_2d_128")
    prob = pair.prob
    c = synth.coefficients(prob, 1001, 3.0)
    e = engine_for(prob, pair.fixed, pair.moving)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, pair.fixed, pair.moving, c)
    assert abs(D - st.D) <= D_RTOL * st.D
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


@pytest.fixture(scope="module")
def c2_case():
    pair = synth.make_pair("c2_ct_256x256x96")
    c = synth.coefficients(pair.prob, 2001, 2.0)
    return pair, c


def test_c2_full_value_and_gradient(c2_case):
    pair, c = c2_case
    prob = pair.prob
    e = engine_for(prob, pair.fixed, pair.moving)
    assert e.levels[0].kernel_path == 1
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, pair.fixed, pair.moving, c)
    assert abs(D - st.D) <= D_RTOL * st.D, (D, st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


def test_c2_bf16_storage(c2_case):
    pair, c = c2_case
    prob = pair.prob
    e = engine_for(prob, pair.fixed, pair.moving, storage="bf16")
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, pair.fixed, pair.moving, c, storage="bf16")
    assert abs(D - st.D) <= D_RTOL * st.D, (D, st.D)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(np.linalg.norm(g) - np.linalg.norm(go)) <= GNORM_RTOL * np.linalg.norm(go)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()


def test_c3_full_value_and_sampled_gradient():
    pair = synth.make_pair("c3_oct_160")
    prob = pair.prob
    c = synth.coefficients(prob, 3001, 1.5)
    e = engine_for(prob, pair.fixed, pair.moving)
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, _, geo, A, M = oracle_eval(prob, pair.fixed, pair.moving, c, grad=False)
    assert abs(D - st.D) <= D_RTOL * st.D, (D, st.D)
    rng = np.random.default_rng(3)
    idx = rng.choice(prob.n_params, 200, replace=False)
    go = oracle.gradient_at(geo, A, M, c, st, idx)
    gs = g.cpu().numpy().ravel()[idx].astype(np.float64)
    assert np.abs(gs - go).max() <= G_ELEM * np.abs(g.cpu().numpy()).max()


# Speckled fixed images put many fixed-image bins into one 32-voxel row (5 to
# 19 here): the value pass forms the segment sums of 8-bin chunks by the
# transpose route with up to 32 segments, and the adjoint forms the X sums
# per lane in rows whose per-segment table would exceed 64 entries.  One
# case per row width (4, 8 and 12 spatial x-bins); the 4-bin case mixes rows
# of both adjoint routes.
SPECKLE = [
    ("oct_rows4", synth.problem(3, (64, 30, 12), (8, 8, 8), (2, 2, 2), 32), 4, "f32"),
    ("oct_rows8", synth.problem(3, (64, 30, 14), (10, 10, 10), (0, 0, 0), 32), 8, "f32"),
    ("oct_rows8_bf16", synth.problem(3, (64, 30, 14), (10, 10, 10), (0, 0, 0), 32), 8, "bf16"),
    ("oct_rows12", synth.problem(3, (64, 26, 12), (5, 5, 5), (0, 0, 0), 32), 12, "f32"),
]


def lane_route_rows(fixed, nbins, nxb):
    """Share of 32-voxel rows whose segments x x-bins x 2 exceeds 64 (the
    adjoint's per-lane route), from the fixed image's bins on the host."""
    L = nbins - 1
    f = fixed.astype(np.float64)
    k = np.clip(np.floor(L * (f - f.min()) / (f.max() - f.min())), 0, L - 1).astype(int)
    rows = k.reshape(-1, 32)
    nseg = np.array([len(np.unique(r)) for r in rows])
    return float(np.mean(nseg * nxb * 2 > 64))


@pytest.mark.parametrize("name,prob,nxb,storage", SPECKLE, ids=[s[0] for s in SPECKLE])
def test_speckle_rows_match_oracle(name, prob, nxb, storage):
    i = [s[0] for s in SPECKLE].index(name)
    f, m = synth.small_pair("oct", prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 300 + i)
    c = synth.coefficients(prob, 400 + i, 1.5)
    share = lane_route_rows(f, prob.n_bins, nxb)
    assert share >= 0.5, share
    if nxb == 4:
        assert share < 1.0, share          # both adjoint routes run
    e = engine_for(prob, f, m, storage=storage)
    assert e.levels[0].kernel_path == 1
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    st, go, _, _, _ = oracle_eval(prob, f, m, c, storage=storage)
    assert abs(D - st.D) <= D_RTOL * abs(st.D), (D, st.D)
    g = g.cpu().numpy().astype(np.float64)
    gn, gon = np.linalg.norm(g), np.linalg.norm(go)
    assert abs(gn - gon) <= GNORM_RTOL * gon, (gn, gon)
    assert np.abs(g - go).max() <= G_ELEM * np.abs(go).max()
