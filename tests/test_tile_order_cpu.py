"""Host logic of the row kernels' tile launch order (srwcr_tile_order; no
GPU): a tile's cost is its number of 32-voxel row segments within 8 voxels
of a nonzero moving-image voxel, tiles go out in 16 cost classes, costly
classes first, and tiles of one class keep their index order.  Checked
against a recount written here from that definition, on ragged 3-D and 2-D
geometries with CT-like distance maps (a body of near rows in air)."""
import numpy as np
import pytest

eng = pytest.importorskip("paper_1804_05061_b300")


def body_rowdist(dims, seed):
    """Distances of a CT-like moving image: 0 inside an ellipsoidal body,
    growing with the L-infinity distance outside it, capped at 255, plus a
    few random near rows (structure in the air)."""
    nx, ny, nz = dims
    nxb = (nx + 31) // 32
    rng = np.random.default_rng(seed)
    z, y, xb = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nxb), indexing="ij")
    cx = (xb * 32 + 16 - nx / 2) / (0.35 * nx)
    cy = (y - ny / 2) / (0.3 * ny)
    cz = (z - nz / 2) / (0.45 * nz)
    r = np.sqrt(cx ** 2 + cy ** 2 + cz ** 2)
    d = np.clip((r - 1.0) * 0.3 * ny, 0, 255).astype(np.uint8)
    near = rng.random(d.shape) < 0.02
    d[near] = rng.integers(0, 9, near.sum())
    return d


def recount(rowdist, dims, tile):
    nx, ny, nz = dims
    nxb = (nx + 31) // 32
    nt1, nt2 = -(-ny // tile[1]), -(-nz // tile[2])
    near = rowdist.reshape(nz, ny, nxb) <= 8
    cost = np.zeros(nxb * nt1 * nt2, np.int64)
    for t in range(cost.size):
        tx, ty, tz = t % nxb, (t // nxb) % nt1, t // (nxb * nt1)
        cost[t] = near[tz * tile[2]:(tz + 1) * tile[2], ty * tile[1]:(ty + 1) * tile[1], tx].sum()
    return cost


@pytest.mark.parametrize("dims,tile", [
    ((256, 256, 96), (32, 256, 1)),
    ((100, 77, 23), (32, 16, 4)),
    ((70, 45, 23), (32, 7, 3)),
    ((100, 77, 1), (32, 8, 1)),
])
def test_order_is_costly_classes_first_and_stable(dims, tile):
    rd = body_rowdist(dims, 5)
    order, cost = eng.tile_order(rd, dims, tile)
    ref = recount(rd, dims, tile)
    assert np.array_equal(cost, ref)
    assert sorted(order.tolist()) == list(range(ref.size))          # a permutation
    cls = ref * 16 // (ref.max() + 1)
    seq = cls[order]
    assert np.all(np.diff(seq) <= 0)                                 # classes descending
    for c in np.unique(cls):
        idx = order[seq == c]
        assert np.all(np.diff(idx) > 0)                              # index order within a class
    assert ref.max() > ref.min()                                     # the map does separate tiles


def test_uniform_costs_keep_index_order():
    dims, tile = (96, 40, 10), (32, 8, 2)
    nxb = 3
    for v in (0, 200):                                               # every row near, none near
        rd = np.full(nxb * 40 * 10, v, np.uint8)
        order, cost = eng.tile_order(rd, dims, tile)
        assert np.array_equal(order, np.arange(order.size))
        assert np.all(cost == (8 * 2 if v == 0 else 0))


def test_threshold_is_eight_voxels():
    dims, tile = (64, 2, 1), (32, 1, 1)
    rd = np.array([8, 9, 255, 0], np.uint8)                          # tiles (x block, y)
    order, cost = eng.tile_order(rd, dims, tile)
    assert cost.tolist() == [1, 0, 0, 1]
    assert order.tolist() == [0, 3, 1, 2]


def test_bad_arguments_are_rejected():
    rd = np.zeros(4, np.uint8)
    with pytest.raises(eng.SrwcrError):
        eng.tile_order(rd, (64, 2, 1), (16, 1, 1))                    # tiles are 32 voxels wide
    with pytest.raises(ValueError):
        eng.tile_order(rd, (64, 2, 1), (32, 0, 1))
    with pytest.raises(ValueError):
        eng.tile_order(rd[:3], (64, 2, 1), (32, 1, 1))                # map of the wrong size
