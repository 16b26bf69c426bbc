"""vif_nll_noalloc: the float64 likelihood for callers that cannot allocate device
memory (a framework that owns the GPU's memory, a plug-in host that forbids
allocations after start-up, a loop that cannot afford cudaMalloc's device-wide
synchronisation).  Its scratch is a static device array shared by all calls, so
this test calls it twice in a row, at two different hyperparameters, and checks
each result against vif_nll on a regular context at the float64 tolerance.

The file name makes pytest collect it last; it also passes on its own in a
fresh process (its first call then performs the one-time address lookup)."""
import numpy as np
import pytest

from paper_2507_05064_gb300 import synth
from paper_2507_05064_gb300 import vif as V

pytestmark = pytest.mark.gpu
RTOL64 = 1e-8


def test_noalloc_matches_vif_nll_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    P = synth.config1()
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64)
    N = ctx.neighbors()
    th2 = P.theta.copy()
    th2.variance, th2.lengthscale, th2.nugget = 1.4, np.array([0.06]), 0.03
    ref2 = ctx.nll(th2, P.y)
    ref1 = ctx.nll(P.theta, P.y)
    ctx.close()
    dev = torch.device("cuda")
    X = torch.from_numpy(P.X).to(dev)
    Z = torch.from_numpy(P.Z).to(dev)
    Nd = torch.from_numpy(N.astype(np.int32)).to(dev)
    y = torch.from_numpy(P.y).to(dev)
    got2 = V.nll_noalloc(X, Z, Nd, P.mv, th2, y)
    got1 = V.nll_noalloc(X, Z, Nd, P.mv, P.theta, y)
    assert got2 == pytest.approx(ref2, rel=RTOL64)
    assert got1 == pytest.approx(ref1, rel=RTOL64)


def test_noalloc_rejects_a_problem_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda")
    n, d, m, mv = 200_000, 2, 200, 10            # ~ 200k * (224 + 256) * 8 B >> 32 MiB
    X = torch.zeros((n, d), dtype=torch.float64, device=dev)
    Z = torch.zeros((m, d), dtype=torch.float64, device=dev)
    Nd = torch.full((n, mv), -1, dtype=torch.int32, device=dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    th = synth.Theta(1, 1.0, np.array([0.1]), 0.1)
    with pytest.raises(V.VifError) as ei:
        V.nll_noalloc(X, Z, Nd, mv, th, y)
    assert ei.value.status == V.VIF_ERR_ARG
    assert "maximum" in str(ei.value)


def test_noalloc_refuses_host_arrays_wrong_dtypes_and_bad_theta_before_any_launch():
    """The kernels read X, Z, N, y directly, so a host array must never reach them: the
    C ABI refuses pointers that are not device or managed memory, the binding refuses
    tensors of the wrong dtype, shape or layout, and invalid hyperparameters are refused
    exactly as vif_nll refuses them (all VIF_ERR_ARG).  A valid call afterwards still
    gives vif_nll's value."""
    import ctypes as C
    torch = pytest.importorskip("torch")
    P = synth.config1()
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64)
    N = ctx.neighbors()
    ref = ctx.nll(P.theta, P.y)
    ctx.close()
    dev = torch.device("cuda")
    X = torch.from_numpy(P.X).to(dev)
    Z = torch.from_numpy(P.Z).to(dev)
    Nd = torch.from_numpy(N.astype(np.int32)).to(dev)
    y = torch.from_numpy(P.y).to(dev)
    L = V.lib()
    n, d, m = P.X.shape[0], P.X.shape[1], P.Z.shape[0]
    cv, ls = V.make_cov(P.theta)
    out = C.c_double(-1.0)
    # host arrays straight into the C ABI (the binding's own checks bypassed)
    Xh = np.ascontiguousarray(P.X)
    yh = np.ascontiguousarray(P.y)
    for Xp, yp in ((Xh, y), (X, yh)):
        st = L.vif_nll_noalloc(V._ptr(Xp), n, d, V._ptr(Z), m, V._ptr(Nd), P.mv, C.byref(cv), V._ptr(yp),
                               None, C.byref(out))
        assert st == V.VIF_ERR_ARG
        assert "device" in L.vif_last_error(None).decode()
    assert out.value == -1.0
    # wrong dtype, layout or shape through the binding
    for bad in (dict(X=X.float()), dict(y=y.float()), dict(N=Nd.long()), dict(X=X.t().contiguous().t()),
                dict(y=y[:-1])):
        args = dict(X=X, Z=Z, N=Nd, y=y)
        args.update(bad)
        with pytest.raises(V.VifError) as ei:
            V.nll_noalloc(args["X"], args["Z"], args["N"], P.mv, P.theta, args["y"])
        assert ei.value.status == V.VIF_ERR_ARG
    # hyperparameters vif_nll rejects
    for field, val in (("variance", float("inf")), ("nugget", float("inf")), ("nugget", float("nan"))):
        th = P.theta.copy()
        setattr(th, field, val)
        with pytest.raises(V.VifError) as ei:
            V.nll_noalloc(X, Z, Nd, P.mv, th, y)
        assert ei.value.status == V.VIF_ERR_ARG
    th = P.theta.copy()
    th.lengthscale = np.array([float("inf")])
    with pytest.raises(V.VifError) as ei:
        V.nll_noalloc(X, Z, Nd, P.mv, th, y)
    assert ei.value.status == V.VIF_ERR_ARG
    assert V.nll_noalloc(X, Z, Nd, P.mv, P.theta, y) == pytest.approx(ref, rel=RTOL64)
