"""The float32 path's residual products A_N^T A_N on the tensor cores (groups of points
sharing one 128-row Gram, vif_factor_tc.cu) against the float64 oracle and against the
same float32 path with the per-point Gram on the CUDA cores.

Cases span several 32-column chunks with a ragged last one (m = 37, 130, 200), one chunk
(m = 20), the largest block the tensor-core path takes (m_v + 1 = 32), and the first
points of the order, which have fewer than m_v predecessors.  The neighbour sets come
from the oracle, so both sides factor the same structure."""
import numpy as np
import pytest

from oracle import vif_oracle as O
from paper_2507_05064_gb300 import synth
from paper_2507_05064_gb300 import vif as V
from tolerance import nll_close

pytestmark = pytest.mark.gpu
RTOL_MIXED = 1e-5

CASES = [
    # n, d, m, m_v, kind, nugget, length scale(s), seed
    (3000, 2, 37, 31, "matern52", 0.05, 0.08, 101),
    (2500, 8, 200, 20, "se", 0.01, [0.3, 0.5, 0.7, 0.9, 1.1, 1.3, 1.6, 1.9], 102),
    (2200, 5, 130, 15, "matern32", 0.1, 0.3, 103),
    (1800, 2, 20, 10, "matern12", 0.1, 0.1, 104),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}-d{c[1]}-m{c[2]}-mv{c[3]}")
def test_tensor_core_factors_match_the_oracle_and_the_simt_path(case):
    n, d, m, mv, kind, nugget, ls, seed = case
    P = synth.make_problem(n, d, m, mv, kind, 1.0, ls, nugget, seed, lloyd=3)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    ref = vif.nll(P.y)
    out = {}
    for simt in (False, True):
        ctx = V.Context(P.X, P.Z, mv, P.theta, precision=V.MIXED, neighbor_search=False, factor_path=(1 if simt else 2))
        ctx.set_neighbors(N.astype(np.int32))
        nll = ctx.nll(P.theta, P.y)
        nll2 = ctx.nll(P.theta, P.y)          # replays give the same bits
        Ac, D = ctx.factors()
        ctx.close()
        assert nll == nll2
        assert nll_close(nll, ref, n, RTOL_MIXED), (simt, nll, ref)
        rD = (D - vif.D) / vif.D
        assert np.abs(rD).max() <= 2e-3, (simt, np.abs(rD).max())
        # the tensor core's float32 accumulation truncates; drained every 64 columns, what is
        # left of that is a shift of D_i inside the spread of float32 rounding (measured: at
        # most 0.57 of the spread on the tensor cores, 0.33 on the CUDA cores)
        assert abs(rD.mean()) <= 1e-6 + 0.75 * rD.std(), (simt, rD.mean(), rD.std())
        np.testing.assert_allclose(Ac, vif.Acoef, rtol=2e-3, atol=2e-3 * np.abs(vif.Acoef).max())
        out[simt] = (nll, rD)
        print(f"simt={simt}: nll err {abs(nll - ref) / abs(ref):.2e}, D_i rel err mean {rD.mean():.2e} "
              f"std {rD.std():.2e} max {np.abs(rD).max():.2e}")
    # the tensor-core sums are no less accurate than the CUDA-core ones
    e_tc, e_simt = np.sqrt((out[False][1] ** 2).mean()), np.sqrt((out[True][1] ** 2).mean())
    assert e_tc <= 3.0 * e_simt + 1e-7, (e_tc, e_simt)


def test_tensor_core_factors_after_new_neighbor_sets():
    """vif_set_neighbors rebuilds the groups: a second structure gives its own oracle factors."""
    P = synth.make_problem(1500, 2, 60, 12, "matern32", 1.0, 0.1, 0.1, 105, lloyd=3)
    N1 = O.causal_neighbors(P.X, P.Z, P.theta, 12)
    N2 = -np.ones_like(N1)
    for i in range(1, 1500):                 # the immediately preceding points
        q = min(i, 12)
        N2[i, :q] = np.arange(i - q, i)
    ctx = V.Context(P.X, P.Z, 12, P.theta, precision=V.MIXED, neighbor_search=False)
    for N in (N1, N2):
        ctx.set_neighbors(N.astype(np.int32))
        vif = O.VIF(P.X, P.Z, P.theta, N)
        assert nll_close(ctx.nll(P.theta, P.y), vif.nll(P.y), 1500, RTOL_MIXED)
        _, D = ctx.factors()
        np.testing.assert_allclose(D, vif.D, rtol=2e-3)
    ctx.close()


def test_factor_autotuner_times_both_paths_and_keeps_the_faster():
    """factor_path = 0: the first evaluation times the CUDA-core and the tensor-core factor
    stage on its own A and keeps the faster; both give the oracle's likelihood."""
    P = synth.make_problem(2500, 8, 200, 20, "se", 1.0, [0.3, 0.5, 0.7, 0.9, 1.1, 1.3, 1.6, 1.9], 0.01, 102, lloyd=3)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 20)
    ref = O.VIF(P.X, P.Z, P.theta, N).nll(P.y)
    ctx = V.Context(P.X, P.Z, 20, P.theta, precision=V.MIXED, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    assert ctx.factor_tuning()["path"] == 0
    nll1 = ctx.nll(P.theta, P.y)
    t = ctx.factor_tuning()
    assert t["path"] in (1, 2) and t["ms_cuda_cores"] > 0 and t["ms_tensor_cores"] > 0
    assert (t["path"] == 2) == (t["ms_tensor_cores"] < t["ms_cuda_cores"])
    nll2 = ctx.nll(P.theta, P.y)
    ctx.close()
    assert nll_close(nll1, ref, 2500, RTOL_MIXED) and nll_close(nll2, ref, 2500, RTOL_MIXED)
