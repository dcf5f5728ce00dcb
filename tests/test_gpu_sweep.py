"""Seeded sweep of small random geometries against the FP64 oracle: 2-D and
3-D sizes from 5 voxels (rows narrower than one 32-voxel tile, ragged tiles
and cells), FFD spacings 3-12 (general kernels below 4, row kernels with 4,
8 or 12 spatial x-bins above), spatial bins on the FFD grid or 1-5
intervals, 2 to 256 intensity bins (the extremes of the range), FP32 and
BF16 storage, both spatial distributions.  D within 1e-5 relative, gradient
elementwise within 1e-3 of the largest entry, degenerate-region counts
equal; gradient norm within 1e-4 * max(1, L / 64): the FP32 warped
intensity B carries a rounding of about 2^-23 L, and a voxel that close to
an integer may take the other one-sided Parzen derivative (dm2/dB jumps by
0.2 (2k + 1) there), so the share of such voxels, and with it the norm's
error, grows with the number of bins (2.3e-4 measured at 256 bins)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def random_case(seed):
    rng = np.random.default_rng(seed)
    nd = int(rng.choice([2, 3]))
    dims = tuple(int(v) for v in rng.integers(5, 71 if nd == 3 else 140, nd))
    if nd == 3:
        dims = (dims[0], dims[1], int(rng.integers(5, 30)))
    sp = tuple(int(min(v, d)) for v, d in zip(rng.integers(3, 13, nd), dims))
    boxcar = bool(rng.random() < 0.2)
    if boxcar or rng.random() < 0.6:
        sb = tuple(int(min(v, d)) for v, d in zip(rng.integers(1, 6, nd), dims))
    else:
        sb = (0,) * nd
    nbins = int(rng.choice([2, 7, 32, 64, 256]))
    storage = "bf16" if rng.random() < 0.3 else "f32"
    return nd, dims, sp, sb, nbins, storage, boxcar


@pytest.mark.parametrize("seed", range(16))
def test_random_geometry_matches_oracle(seed):
    import paper_1804_05061_b300 as eng
    nd, dims, sp, sb, nbins, storage, boxcar = random_case(800 + seed)
    prob = synth.problem(nd, dims, sp, sb, nbins)
    kind = "ct" if nd == 3 else "ellipse"
    f, m = synth.small_pair(kind, dims, sp, 1.5, 900 + seed)
    c = synth.coefficients(prob, 950 + seed, 1.2)
    e = eng.from_problem(prob, f, m, storage=storage,
                         spatial="boxcar" if boxcar else "bspline")
    D, g = e.value_and_grad(torch.from_numpy(c).cuda())
    _, ndeg = e.region_stats()
    geo = oracle.Geometry.from_problem(prob, boxcar_patches=sb if boxcar else None)
    A, M = oracle.prepare(f, m, nbins, storage)
    st = oracle.value(geo, A, M, c)
    go = oracle.gradient(geo, A, M, c, st)
    info = (dims, sp, sb, nbins, storage, boxcar, e.levels[0].kernel_path, e.levels[0].tile)
    assert abs(D - st.D) <= 1e-5 * abs(st.D) + 1e-12, (D, st.D, info)
    assert ndeg == st.n_degenerate, (ndeg, st.n_degenerate, info)
    g = g.cpu().numpy().astype(np.float64)
    gn, gon = np.linalg.norm(g), np.linalg.norm(go)
    tol = 1e-4 * max(1.0, (nbins - 1) / 64.0)
    assert abs(gn - gon) <= tol * gon + 1e-12, (gn, gon, info)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max() + 1e-12, info


def test_sweep_covers_both_paths_and_all_row_widths():
    """The seeds above reach the general kernels and the 4-, 8- and 12-bin
    row kernels (checked on the host from the geometry rules)."""
    paths = set()
    for seed in range(16):
        nd, dims, sp, sb, nbins, storage, boxcar = random_case(800 + seed)
        # FFD x-nodes and spatial x-bins a 32-voxel row meets (aligned rows).
        hf = (min(dims[0], 32) - 1) // sp[0] + 4
        if sb[0] > 0:
            hb = int((min(dims[0], 32) - 1) * sb[0] // dims[0]) + 4
        else:
            hb = (min(dims[0], 32) - 1) // sp[0] + 4
        paths.add("general" if hf > 11 or hb > 12 else ("rows4" if hb <= 4 else ("rows8" if hb <= 8 else "rows12")))
    assert {"general", "rows8"} <= paths, paths
