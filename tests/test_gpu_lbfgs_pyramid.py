"""GPU parity of the L-BFGS driver and of the pyramid transfer (Sec. II-F).

* Two-loop recursion: the library's search direction (srwcr_lbfgs_direction:
  FP32 vectors, FP64 device inner products) equals the oracle's two-loop
  (FP64) on the same FP32 history, for synthetic curvature pairs and for
  pairs taken from SRWCR gradients of the 2-D workload.
* Iterations: srwcr_register run for k = 1 .. 6 iterations from zero equals,
  iteration by iteration, the oracle's L-BFGS loop fed the same GPU value and
  gradient (so the comparison isolates the optimiser's arithmetic): the same
  number of evaluations (the same line-search decisions) and close
  coefficients and values.  The bounds widen after the third iteration
  because the iteration is chaotic at the rounding level: the FP64 oracle
  alone, run once with its iterate rounded to FP32 before each evaluation,
  drifts from itself by 1e-7 (k = 4), 9e-7 (k = 6) and 5e-3 (k = 9) in D,
  and 1e-7 relative noise on its gradient gives 6e-6, 4e-5 and 4e-3; the GPU
  gradient's FP32 atomics add in a run-dependent order, so the GPU run does
  not repeat itself more closely than that either.
* Downsampling: every coarser level's normalised images equal the 2^d box
  average (floor sizes) of the finer level's, for FP32 and BF16 storage.
* Refinement: the dyadic subdivision of the coefficients reproduces the
  coarse displacement: the fine displacement at fine voxel 2x equals twice
  the coarse displacement at coarse voxel x (oracle displacement on both
  levels) wherever no coarse index of the stencil is clamped.
"""
import numpy as np
import pytest

import oracle
from oracle import lbfgs
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIR_RTOL = 1e-5


def engine(prob, f, m, **kw):
    import paper_1804_05061_b300 as eng
    return eng.from_problem(prob, f, m, **kw)


@pytest.fixture(scope="module")
def c1_engine():
    pair = synth.make_pair("c1_2d_128")
    return pair, engine(pair.prob, pair.fixed, pair.moving)


def check_direction(e, g, S, Y):
    """Library direction vs the oracle's two-loop on the same FP32 values."""
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    St = torch.from_numpy(np.stack(S).astype(np.float32)).cuda() if S else None
    Yt = torch.from_numpy(np.stack(Y).astype(np.float32)).cuda() if Y else None
    d = e.lbfgs_direction(gt, St, Yt).cpu().numpy().astype(np.float64)
    S64 = [s.astype(np.float32).astype(np.float64) for s in S]
    Y64 = [y.astype(np.float32).astype(np.float64) for y in Y]
    ref = lbfgs.two_loop(g.astype(np.float32).astype(np.float64), S64, Y64)
    assert np.linalg.norm(d - ref) <= DIR_RTOL * np.linalg.norm(ref), \
        np.linalg.norm(d - ref) / np.linalg.norm(ref)
    assert np.abs(d - ref).max() <= DIR_RTOL * np.abs(ref).max()


@pytest.mark.parametrize("k", [0, 1, 2, 5, 8])
def test_two_loop_direction_matches_oracle_synthetic_pairs(c1_engine, k):
    _, e = c1_engine
    rng = np.random.default_rng(100 + k)
    n = 20011
    diag = rng.uniform(0.5, 20.0, n)
    S = [rng.normal(size=n) for _ in range(k)]
    Y = [diag * s + 0.3 * rng.normal(size=n) for s in S]
    assert all(s @ y > 0 for s, y in zip(S, Y))
    check_direction(e, rng.normal(size=n), S, Y)


def test_two_loop_direction_matches_oracle_srwcr_pairs(c1_engine):
    """Curvature pairs from SRWCR gradients along a descent path on the 2-D
    workload (history of 5, the paper's setting)."""
    pair, e = c1_engine
    prob = pair.prob
    x = np.zeros(prob.n_params, np.float32)
    _, g = e.value_and_grad(torch.from_numpy(x.reshape(prob.coef_shape)).cuda())
    g = g.cpu().numpy().ravel().astype(np.float64)
    S, Y = [], []
    for _ in range(12):
        xn = (x - 0.4 * g / np.linalg.norm(g)).astype(np.float32)
        _, gn = e.value_and_grad(torch.from_numpy(xn.reshape(prob.coef_shape)).cuda())
        gn = gn.cpu().numpy().ravel().astype(np.float64)
        s, y = xn.astype(np.float64) - x, gn - g
        if s @ y > 0:
            S.append(s); Y.append(y)
        x, g = xn, gn
        if len(S) == 5:
            break
    assert len(S) >= 2
    check_direction(e, g, S, Y)


def test_register_iterations_match_oracle_loop_fed_gpu_values(c1_engine):
    pair, e = c1_engine
    prob = pair.prob

    def fg(x):
        c = torch.from_numpy(np.asarray(x, np.float32).reshape(prob.coef_shape)).cuda()
        D, g = e.value_and_grad(c)
        return D, g.cpu().numpy().ravel().astype(np.float64)

    for k in range(1, 7):
        o = e.default_opts()
        o.max_iter[0] = k
        o.stable_window = 0
        c = e.zeros()
        rep = e.register(c, 1, o)
        res = lbfgs.minimise(fg, np.zeros(prob.n_params),
                             lbfgs.LbfgsOptions(max_iter=k, stable_window=0))
        cg = c.cpu().numpy().ravel().astype(np.float64)
        assert rep.iterations[0] == res.n_iter == k
        assert rep.evaluations[0] == res.n_evals, (k, rep.evaluations[0], res.n_evals)
        x_tol, d_tol = (2e-5, 5e-6) if k <= 3 else (5e-3, 5e-4)
        err = np.linalg.norm(cg - res.x) / np.linalg.norm(res.x)
        assert err <= x_tol, (k, err)
        assert abs(rep.final_value[0] - res.f) <= d_tol * abs(res.f), (k, rep.final_value[0], res.f)


def box_average(img: np.ndarray) -> np.ndarray:
    """2^d box average with floor sizes, in FP64."""
    sl = tuple(slice(0, (s // 2) * 2) for s in img.shape)
    v = img[sl].astype(np.float64)
    out = np.zeros(tuple(s // 2 for s in v.shape))
    for off in np.ndindex(*(2,) * v.ndim):
        out += v[tuple(slice(o, None, 2) for o in off)]
    return out / 2 ** v.ndim


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("kind,dims,levels", [("ct", (45, 38, 21), 3), ("ellipse", (101, 66), 3),
                                              ("oct", (40, 33, 30), 2)])
def test_downsampled_levels_are_box_averages(storage, kind, dims, levels):
    nd = len(dims)
    prob = synth.problem(nd, dims, (4,) * nd, (2,) * nd, 32)
    f, m = synth.small_pair(kind, dims, (4,) * nd, 2.0, 51)
    e = engine(prob, f, m, storage=storage, pyramid_levels=levels)
    prev = [t.cpu().numpy() for t in e.level_images(0)]
    for lvl in range(1, levels):
        cur = [t.cpu().numpy() for t in e.level_images(lvl)]
        for fine, coarse in zip(prev, cur):
            ref = box_average(fine)
            assert coarse.shape == ref.shape
            if storage == "f32":
                tol = 4 * np.spacing(np.float32(prob.n_bins - 1))
                assert np.abs(coarse - ref).max() <= tol
            else:
                rb = torch.from_numpy(ref).to(torch.bfloat16).to(torch.float64).numpy()
                ulp = np.maximum(np.abs(rb), 1e-30) * 2.0 ** -7
                diff = np.abs(coarse - rb)
                assert (diff <= ulp).all()
                assert (diff == 0).mean() >= 0.999
        prev = cur


@pytest.mark.parametrize("dims,spacing", [((48, 40, 24), (6, 5, 4)), ((70, 53), (5, 7)),
                                          ((37, 41, 29), (4, 4, 5))])
def test_refinement_reproduces_the_coarse_displacement(dims, spacing):
    nd = len(dims)
    prob = synth.problem(nd, dims, spacing, (2,) * nd, 16)
    f, m = synth.small_pair("ct" if nd == 3 else "ellipse", dims, spacing, 2.0, 61)
    e = engine(prob, f, m, pyramid_levels=2)
    lc, lf = e.levels[1], e.levels[0]
    cc = synth.coefficients(synth.problem(nd, lc.dims[:nd], spacing, (2,) * nd, 16), 62, 1.5)
    cf = e.refine(torch.from_numpy(cc).cuda(), 1).cpu().numpy()
    geo_c = oracle.Geometry.from_problem(synth.problem(nd, lc.dims[:nd], spacing, (2,) * nd, 16))
    geo_f = oracle.Geometry.from_problem(synth.problem(nd, lf.dims[:nd], spacing, (2,) * nd, 16))
    nfc = lc.ffd_nodes

    def unclamped(q, d):
        # fine voxel 2q lies in fine cell p; nodes p .. p+3 need coarse
        # indices up to (j+1)//2 + 1 (odd j) or j//2 + 1 (even j)
        p = (2 * q) // spacing[d]
        for j in range(p, p + 4):
            top = (j + 1) // 2 + 1 if j % 2 else j // 2 + 1
            if top > nfc[d] - 1:
                return False
        return True

    rng = np.random.default_rng(63)
    checked = 0
    scale = np.abs(cc).max()
    for _ in range(600):
        q = [int(rng.integers(0, lc.dims[d])) for d in range(nd)]
        if not all(unclamped(q[d], d) for d in range(nd)):
            continue
        qz = q[2] if nd == 3 else 0
        uc = oracle.displacement(geo_c, cc, q[0], q[1], qz)
        uf = oracle.displacement(geo_f, cf, 2 * q[0], 2 * q[1], 2 * qz)
        assert np.abs(uf - 2 * uc).max() <= 2e-6 * scale, (q, uf, 2 * uc)
        checked += 1
    assert checked >= 200
