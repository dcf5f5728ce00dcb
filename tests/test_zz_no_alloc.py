"""The allocation-free value entry point (srwcr_value_noalloc).

Some callers cannot allocate device memory -- code inside a CUDA-graph
capture, plugins whose host application owns every allocation, real-time
loops that must stay off the allocator.  For them the library offers one
entry point whose scratch is a fixed device array inside the library.  These
tests call it through the C ABI twice in a row (the scratch keeps the
previous call's contents, so the second call checks that everything that
must start at zero is cleared) and compare both results with srwcr_value on
a context, within the value tolerance of the other parity tests.  Cases: two
small geometries, the boxcar spatial distribution, a requested voxel tile, a
problem just under the scratch capacity (and one just over it, which must be
rejected with the byte count the layout gives), and the 512x512x300 workload
on full-size device buffers, also checked against the stored FP64 oracle
value.  The file is collected last and passes alone or after the other
tests.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D_RTOL = 1e-5
SCRATCH_BYTES = 16 << 20
HERE = os.path.dirname(os.path.abspath(__file__))


def scratch_need(n_regions: int, n_bins: int) -> int:
    """Bytes the entry point's scratch layout needs: S (2 u64 per region and
    bin), P (double), X (float), then U, V (float), D_r (double), the region
    stats (4 doubles) and the degenerate count, each block starting on a
    256-byte boundary."""
    a = lambda b: (b + 255) & ~255
    R, nb = n_regions, n_bins
    off = a(16 * R * nb)
    off = a(off + 8 * R * nb)
    off = a(off + 4 * R * nb)
    off = a(off + 4 * R)
    off = a(off + 4 * R)
    off = a(off + 8 * R)
    off = a(off + 32 * R)
    return off + 4


def normalised(img: np.ndarray, L: int) -> torch.Tensor:
    """L (v - min) / (max - min) in FP64, rounded to float32, on the device."""
    v = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda().double()
    mn, mx = v.min(), v.max()
    out = (L * (v - mn) / (mx - mn)).float().contiguous()
    del v
    return out


def make_cfg(eng, prob, spatial="bspline", tile=None):
    cfg = eng.Config()
    cfg.ndim = prob.ndim
    for d in range(3):
        cfg.dims[d] = prob.dims[d]
        cfg.ffd_spacing[d] = prob.ffd_spacing[d]
        cfg.sbin_intervals[d] = prob.sbin_intervals[d]
        cfg.tile[d] = tile[d] if tile else 0
    cfg.n_intensity_bins = prob.n_bins
    cfg.pyramid_levels = 1
    cfg.spatial = eng.SPATIAL[spatial]
    return cfg


def noalloc_twice(eng, cfg, A, M, c):
    """Two calls in a row through the C ABI; returns both values."""
    lib = eng.load()
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(2):
        D = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.srwcr_value_noalloc(ctypes.byref(cfg), ctypes.c_void_p(A.data_ptr()),
                                     ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                     ctypes.c_void_p(D.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.srwcr_last_error()
        torch.cuda.synchronize()
        out.append(float(D.item()))
    return out


CASES = [
    ("ct", synth.problem(3, (48, 40, 24), (6, 6, 6), (2, 2, 2), 32), "bspline", None),
    ("ellipse", synth.problem(2, (100, 77), (7, 7), (3, 2), 16), "bspline", None),
    ("ct", synth.problem(3, (45, 38, 21), (5, 5, 5), (3, 2, 2), 24), "boxcar", None),
    ("ct", synth.problem(3, (40, 36, 20), (6, 6, 6), (2, 2, 2), 32), "bspline", (16, 4, 2)),
]


@pytest.mark.parametrize("kind,prob,spatial,tile", CASES)
def test_noalloc_value_matches_context_value_on_two_calls(kind, prob, spatial, tile):
    import paper_1804_05061_b300 as eng
    f, m = synth.small_pair(kind, prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 21)
    c = torch.from_numpy(synth.coefficients(prob, 22, 1.5)).cuda()
    ref = eng.from_problem(prob, f, m, spatial=spatial).value(c)
    L = prob.n_bins - 1
    vals = noalloc_twice(eng, make_cfg(eng, prob, spatial, tile), normalised(f, L),
                         normalised(m, L), c)
    for call, val in enumerate(vals):
        assert abs(val - ref) <= D_RTOL * abs(ref), (call, val, ref)


def test_noalloc_capacity_boundary():
    """A 2-D problem with 48 x 48 spatial bins and 256 intensity bins sits just
    under the scratch capacity and is accepted; with 49 x 49 it is rejected,
    and the message gives the bytes the layout needs."""
    import paper_1804_05061_b300 as eng
    under = synth.problem(2, (150, 140), (8, 8), (45, 45), 256)
    over = synth.problem(2, (150, 140), (8, 8), (46, 46), 256)
    n_under, n_over = (45 + 3) ** 2, (46 + 3) ** 2
    assert scratch_need(n_under, 256) <= SCRATCH_BYTES < scratch_need(n_over, 256)
    f, m = synth.small_pair("ellipse", under.dims[:2], under.ffd_spacing[:2], 2.0, 41)
    c = torch.from_numpy(synth.coefficients(under, 42, 1.5)).cuda()
    L = under.n_bins - 1
    A, M = normalised(f, L), normalised(m, L)
    ref = eng.from_problem(under, f, m).value(c)
    for call, val in enumerate(noalloc_twice(eng, make_cfg(eng, under), A, M, c)):
        assert abs(val - ref) <= D_RTOL * abs(ref), (call, val, ref)

    lib = eng.load()
    D = torch.zeros((), dtype=torch.float64, device="cuda")
    st = lib.srwcr_value_noalloc(ctypes.byref(make_cfg(eng, over)), ctypes.c_void_p(A.data_ptr()),
                                 ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                 ctypes.c_void_p(D.data_ptr()), None)
    assert st == 1
    msg = lib.srwcr_last_error().decode()
    assert f"needs {scratch_need(n_over, 256)} bytes" in msg, msg


def test_noalloc_full_size_512x512x300():
    """The 512x512x300 CT workload (3971 spatial bins, 128 intensity bins) on
    full-size device buffers: accepted, equal to srwcr_value on a context and
    to the stored FP64 oracle value at the same coefficients."""
    import paper_1804_05061_b300 as eng
    with open(os.path.join(HERE, "golden", "full_size_oracle.json")) as fh:
        ref = json.load(fh)["cases"]["c5_f32"]
    pair = synth.make_pair("c5_ct_512x512x300")
    prob = pair.prob
    assert scratch_need(19 * 19 * 11, 128) <= SCRATCH_BYTES
    c = torch.from_numpy(synth.coefficients(prob, ref["coef_seed"], ref["coef_sigma"])).cuda()
    e = eng.from_problem(prob, pair.fixed, pair.moving)
    D_ctx = e.value(c)
    e.close()
    del e
    torch.cuda.empty_cache()
    L = prob.n_bins - 1
    vals = noalloc_twice(eng, make_cfg(eng, prob), normalised(pair.fixed, L),
                         normalised(pair.moving, L), c)
    for call, val in enumerate(vals):
        assert abs(val - D_ctx) <= D_RTOL * abs(D_ctx), (call, val, D_ctx)
        assert abs(val - ref["D"]) <= D_RTOL * abs(ref["D"]), (call, val, ref["D"])


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    cfg = eng.Config()
    cfg.ndim = 3
    for d, (n, sp, k) in enumerate([(2048, 4, 200), (2048, 4, 200), (64, 4, 8)]):
        cfg.dims[d], cfg.ffd_spacing[d], cfg.sbin_intervals[d] = n, sp, k
    cfg.n_intensity_bins = 128
    cfg.pyramid_levels = 1
    x = torch.zeros(16, device="cuda")
    D = torch.zeros((), dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    st = lib.srwcr_value_noalloc(ctypes.byref(cfg), p, p, p, ctypes.c_void_p(D.data_ptr()), None)
    assert st == 1
    assert b"scratch" in lib.srwcr_last_error()
