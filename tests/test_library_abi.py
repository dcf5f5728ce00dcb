"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/srwcr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "srwcr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srwcr_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("srwcr_create", "srwcr_value", "srwcr_value_and_grad", "srwcr_register",
                 "srwcr_destroy", "srwcr_last_error"):
        assert name in syms


def test_library_loads_and_exports_every_declared_symbol():
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(eng.EXPORTS) == set(declared_symbols())


def test_last_error_is_callable_without_gpu():
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    assert isinstance(lib.srwcr_last_error(), bytes)


def test_bad_config_rejected_before_touching_the_device():
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    cfg = eng.Config()
    cfg.ndim = 4
    out = ctypes.c_void_p()
    buf = (ctypes.c_float * 8)()
    st = lib.srwcr_create(ctypes.byref(cfg), ctypes.cast(buf, ctypes.c_void_p),
                          ctypes.cast(buf, ctypes.c_void_p), 0, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"ndim" in lib.srwcr_last_error()


def _valid_2d_config(eng):
    cfg = eng.Config()
    cfg.ndim = 2
    cfg.dims[0], cfg.dims[1], cfg.dims[2] = 8, 8, 1
    cfg.ffd_spacing[0], cfg.ffd_spacing[1], cfg.ffd_spacing[2] = 4, 4, 1
    cfg.sbin_intervals[0], cfg.sbin_intervals[1] = 2, 2
    cfg.n_intensity_bins = 8
    cfg.pyramid_levels = 1
    return cfg


@pytest.mark.parametrize("field,value,word", [
    ("finalize_lanes", 3, b"finalize_lanes"),
    ("finalize_lanes", 64, b"finalize_lanes"),
    ("spatial", 2, b"spatial"),
    ("role", 5, b"role"),
])
def test_bad_option_rejected_before_touching_the_device(field, value, word):
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    cfg = _valid_2d_config(eng)
    setattr(cfg, field, value)
    out = ctypes.c_void_p()
    buf = (ctypes.c_float * 64)()
    st = lib.srwcr_create(ctypes.byref(cfg), ctypes.cast(buf, ctypes.c_void_p),
                          ctypes.cast(buf, ctypes.c_void_p), 0, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert word in lib.srwcr_last_error()


def test_boxcar_needs_patch_counts_on_every_axis():
    import paper_1804_05061_b300 as eng
    lib = eng.load()
    cfg = _valid_2d_config(eng)
    cfg.spatial = eng.SPATIAL["boxcar"]
    cfg.sbin_intervals[1] = 0
    out = ctypes.c_void_p()
    buf = (ctypes.c_float * 64)()
    st = lib.srwcr_create(ctypes.byref(cfg), ctypes.cast(buf, ctypes.c_void_p),
                          ctypes.cast(buf, ctypes.c_void_p), 0, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"boxcar" in lib.srwcr_last_error()


def test_oracle_is_not_linked_into_the_product():
    """The product library and binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1804_05061_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "srwcr_oracle" not in src, f
