"""The C-ABI library builds, loads, and exports every symbol include/vif.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

from paper_2507_05064_gb300 import vif as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "vif.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vif_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(V.LIB_PATH):
        from paper_2507_05064_gb300 import build_lib
        build_lib.build()
    return V.lib()


def test_header_declares_the_expected_entry_points():
    decl = _declared_functions()
    assert set(decl) == set(V.EXPORTS), decl
    for name in ("vif_build", "vif_nll", "vif_predict", "vif_destroy", "vif_last_error"):
        assert name in decl


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    import ctypes as C
    assert C.sizeof(V.VifOpts) == 8 * 4
    assert V.VifCov.lengthscale.offset == 16 and C.sizeof(V.VifCov) == 40


def test_build_rejects_bad_arguments_before_touching_the_gpu(lib):
    import ctypes as C
    import numpy as np
    X = np.zeros((4, 2))
    ls = np.array([0.1])
    cv = V.VifCov(1, 1.0, ls.ctypes.data_as(C.POINTER(C.c_double)), 1, 0.1)
    opts = V.VifOpts(0, 0, 0, 0, (C.c_int32 * 4)())
    h = C.c_void_p()
    # d out of range, mv out of range, bad precision: rejected by argument checks
    assert lib.vif_build(V._ptr(X), 4, 17, None, 0, 2, C.byref(cv), C.byref(opts), None, C.byref(h)) == V.VIF_ERR_ARG
    assert lib.vif_build(V._ptr(X), 4, 2, None, 0, 99, C.byref(cv), C.byref(opts), None, C.byref(h)) == V.VIF_ERR_ARG
    bad = V.VifOpts(7, 0, 0, 0, (C.c_int32 * 4)())
    assert lib.vif_build(V._ptr(X), 4, 2, None, 0, 2, C.byref(cv), C.byref(bad), None, C.byref(h)) == V.VIF_ERR_ARG
    assert lib.vif_last_error(None) is not None
