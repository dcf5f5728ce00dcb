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


def test_oracle_is_not_linked_into_the_product():
    """The product library and binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1804_05061_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "srwcr_oracle" not in src, f
