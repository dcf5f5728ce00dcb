"""The allocation-free value entry point (srwcr_value_noalloc).

Some callers cannot allocate device memory -- code inside a CUDA-graph
capture, plugins whose host application owns every allocation, real-time
loops that must stay off the allocator.  For them the library offers one
entry point whose scratch is a fixed device array inside the library.  This
test calls it through the C ABI twice in a row (the scratch keeps the previous
call's contents, so the second call checks that everything that must start at
zero is cleared) and compares both results with srwcr_value on a context.
It lives in its own file, collected last, and passes alone or after the
other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D_RTOL = 1e-5


def normalised(img: np.ndarray, L: int) -> torch.Tensor:
    """L (v - min) / (max - min) in FP64, rounded to float32, on the device."""
    v = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda().double()
    mn, mx = v.min(), v.max()
    return (L * (v - mn) / (mx - mn)).float().contiguous()


@pytest.mark.parametrize("kind,prob", [
    ("ct", synth.problem(3, (48, 40, 24), (6, 6, 6), (2, 2, 2), 32)),
    ("ellipse", synth.problem(2, (100, 77), (7, 7), (3, 2), 16)),
])
def test_noalloc_value_matches_context_value_on_two_calls(kind, prob):
    import paper_1804_05061_b300 as eng
    f, m = synth.small_pair(kind, prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], 2.0, 21)
    c = torch.from_numpy(synth.coefficients(prob, 22, 1.5)).cuda()
    ref = eng.from_problem(prob, f, m).value(c)

    lib = eng.load()
    cfg = eng.Config()
    cfg.ndim = prob.ndim
    for d in range(3):
        cfg.dims[d] = prob.dims[d]
        cfg.ffd_spacing[d] = prob.ffd_spacing[d]
        cfg.sbin_intervals[d] = prob.sbin_intervals[d]
    cfg.n_intensity_bins = prob.n_bins
    cfg.pyramid_levels = 1
    L = prob.n_bins - 1
    A, M = normalised(f, L), normalised(m, L)
    stream = torch.cuda.current_stream()
    for call in range(2):
        D = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.srwcr_value_noalloc(ctypes.byref(cfg), ctypes.c_void_p(A.data_ptr()),
                                     ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                     ctypes.c_void_p(D.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.srwcr_last_error()
        torch.cuda.synchronize()
        val = float(D.item())
        assert abs(val - ref) <= D_RTOL * abs(ref), (call, val, ref)


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
