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
    opts = V.VifOpts(0, 0, 0, 0, 0, (C.c_int32 * 3)())
    h = C.c_void_p()
    # d out of range, mv out of range, bad precision: rejected by argument checks
    assert lib.vif_build(V._ptr(X), 4, 17, None, 0, 2, C.byref(cv), C.byref(opts), None, C.byref(h)) == V.VIF_ERR_ARG
    assert lib.vif_build(V._ptr(X), 4, 2, None, 0, 99, C.byref(cv), C.byref(opts), None, C.byref(h)) == V.VIF_ERR_ARG
    bad = V.VifOpts(7, 0, 0, 0, 0, (C.c_int32 * 3)())
    assert lib.vif_build(V._ptr(X), 4, 2, None, 0, 2, C.byref(cv), C.byref(bad), None, C.byref(h)) == V.VIF_ERR_ARG
    assert lib.vif_last_error(None) is not None


def test_laplace_nll_stats_layout_matches_header():
    import ctypes as C
    assert C.sizeof(V.LaplaceNllStats) == 8 * 8 + 4 * 4 + 2 * 8
    assert V.LaplaceNllStats.newton_iters.offset == 64 and V.LaplaceNllStats.ms_mode.offset == 80
    assert C.sizeof(V.LaplaceGradStats) == C.sizeof(V.LaplaceNllStats) + 2 * 4 + 8
    assert V.LaplaceGradStats.pcg_iters_v.offset == C.sizeof(V.LaplaceNllStats)


def test_laplace_grad_rejects_non_vifdu_and_missing_outputs_without_a_gpu():
    """Argument checks of vif_laplace_nll_grad run before any device work."""
    import ctypes as C
    import numpy as np
    lib = V.lib()
    ls = np.array([0.2])
    cv = V.VifCov(1, 1.0, ls.ctypes.data_as(C.POINTER(C.c_double)), 1, 0.0)
    out = C.c_double()
    g = np.zeros(2)
    assert lib.vif_laplace_nll_grad(None, C.byref(cv), None, None, 1, None, 1e-2, 10, C.byref(out), V._ptr(g),
                                    None, None, None) == V.VIF_ERR_ARG


def _tridiag_reference(d, e):
    import numpy as np
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam, U = np.linalg.eigh(T)
    return float((U[0] ** 2) @ np.log(lam))


@pytest.mark.parametrize("k,kind", [(1, "random"), (2, "random"), (7, "random"), (60, "random"),
                                    (300, "random"), (40, "clustered"), (120, "lanczos-like")])
def test_tridiagonal_log_quadrature_matches_eigendecomposition(lib, k, kind):
    """The host Gauss quadrature e_1^T log(T) e_1 of the SLQ (App. D) against numpy's
    symmetric eigendecomposition (no GPU involved)."""
    import numpy as np
    rng = np.random.default_rng(k)
    if kind == "random":
        e = rng.uniform(-1.0, 1.0, k - 1)
        d = rng.uniform(0.5, 3.0, k) + np.abs(np.concatenate([e, [0]])) + np.abs(np.concatenate([[0], e]))
    elif kind == "clustered":
        # eigenvalues in two tight clusters, tridiagonalised by Householder reflections
        lam = np.concatenate([1.0 + 1e-9 * rng.standard_normal(k // 2), 5.0 + 1e-9 * rng.standard_normal(k - k // 2)])
        Qm, _ = np.linalg.qr(rng.standard_normal((k, k)))
        import scipy.linalg as sla
        H = sla.hessenberg(Qm @ np.diag(lam) @ Qm.T)
        d, e = np.diag(H).copy(), np.diag(H, -1).copy()
    else:
        # the shape CG produces: diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off sqrt(beta)/alpha
        al = rng.uniform(0.2, 2.0, k)
        be = rng.uniform(0.05, 0.9, k - 1)
        d = 1.0 / al + np.concatenate([[0.0], be / al[:-1]])
        e = np.sqrt(be) / al[:-1]
    got = V.tridiag_log_quadrature(d, e)
    ref = _tridiag_reference(d, e)
    assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (got, ref)


def test_tridiagonal_log_quadrature_rejects_an_indefinite_matrix(lib):
    import numpy as np
    with pytest.raises(V.VifError) as ei:
        V.tridiag_log_quadrature(np.array([1.0, -2.0, 1.0]), np.array([0.1, 0.1]))
    assert ei.value.status == V.VIF_ERR_NOT_PD



def test_batch_entry_points_reject_a_null_batch_without_a_gpu(lib):
    """vif_batch_run / _info / _set_shape / _factor_info check their handle before any device work."""
    import ctypes as C
    i32 = C.c_int32()
    d = C.c_double()
    assert lib.vif_batch_run(None, C.byref(d)) == V.VIF_ERR_ARG
    assert lib.vif_batch_info(None, C.byref(i32), C.byref(i32), C.byref(d)) == V.VIF_ERR_ARG
    assert lib.vif_batch_set_shape(None, 8, 1, 0) == V.VIF_ERR_ARG
    assert lib.vif_batch_factor_info(None, C.byref(i32), C.byref(i32), C.byref(i32)) == V.VIF_ERR_ARG
    lib.vif_batch_destroy(None)   # a no-op
