"""GPU (CUDA path through the C ABI) against the FP64 oracle, element by element.

Tolerances: float64 path 1e-8 relative on the likelihood; mixed path 1e-5
relative (plain relative error, except for likelihoods that cancel to below a
tenth of n/2 log 2 pi: tests/tolerance.py); neighbour sets exact up to near-ties (two candidates whose oracle keys
differ by less than TIE_TOL may be exchanged).
"""
import json
import os

import numpy as np
import pytest

from oracle import vif_oracle as O
from paper_2507_05064_gb300 import synth
from paper_2507_05064_gb300 import vif as V
from tolerance import nll_close

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TIE_TOL = 1e-9
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL64 = 1e-8
RTOL_MIXED = 1e-5


def prob(n, d, m, mv, kind, nugget, ls, seed, inducing="kmeans++"):
    return synth.make_problem(n, d, m, mv, kind, 1.0, ls, nugget, seed, inducing=inducing, lloyd=3)


def check_sets(N_gpu, N_or, keys, mv, tol=TIE_TOL):
    """Exact set equality except at near-ties; returns the number of near-tie swaps."""
    swaps = 0
    for i in range(N_or.shape[0]):
        a = set(int(j) for j in N_gpu[i] if j >= 0)
        b = set(int(j) for j in N_or[i] if j >= 0)
        if a == b:
            continue
        assert len(a) == len(b) == min(i, mv), (i, a, b)
        k = keys[i - 1] if isinstance(keys, list) and len(keys) == N_or.shape[0] - 1 else keys[i]
        ka = np.sort(k[list(a)])
        kb = np.sort(k[list(b)])
        assert np.max(np.abs(ka - kb)) <= tol, (i, sorted(a - b), sorted(b - a), ka, kb)
        swaps += 1
    return swaps


def oracle_keys_by_row(P, N):
    """Oracle neighbour sets and per-row key vectors (row i: keys against 0..i-1)."""
    Nor, keys, _ = O.causal_neighbors(P.X, P.Z, P.theta, P.mv, return_keys=True)
    return Nor, [np.zeros(0)] + keys


# --------------------------------------------------------------------------- C1: the stated small workload
@pytest.fixture(scope="module")
def c1():
    P = synth.config1()
    Nor, keys = oracle_keys_by_row(P, None)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    return P, Nor, keys, vif


def test_c1_neighbor_sets_match_oracle(c1):
    P, Nor, keys, _ = c1
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64)
    swaps = check_sets(ctx.neighbors(), Nor, keys, P.mv)
    assert swaps <= 2
    ctx.close()


@pytest.mark.parametrize("precision,rtol", [(V.FP64, RTOL64), (V.MIXED, RTOL_MIXED)])
def test_c1_nll_and_factors_with_oracle_neighbors(c1, precision, rtol):
    P, Nor, keys, vif = c1
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=precision, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    nll = ctx.nll(P.theta, P.y)
    ref = vif.nll(P.y)
    assert nll_close(nll, ref, P.X.shape[0], rtol), (nll, ref)
    Ac, D = ctx.factors()
    ftol = 1e-9 if precision == V.FP64 else 2e-3
    np.testing.assert_allclose(D, vif.D, rtol=ftol)
    np.testing.assert_allclose(Ac, vif.Acoef, rtol=ftol, atol=ftol * np.abs(vif.Acoef).max())
    ctx.close()


def test_c1_end_to_end(c1):
    P, Nor, keys, vif = c1
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64)
    assert ctx.nll(P.theta, P.y) == pytest.approx(vif.nll(P.y), rel=RTOL64)
    # a second call at other hyperparameters (neighbour sets stay fixed)
    th2 = P.theta.copy()
    th2.variance, th2.lengthscale, th2.nugget = 1.3, np.array([0.07]), 0.05
    ref2 = O.VIF(P.X, P.Z, th2, Nor).nll(P.y)
    assert ctx.nll(th2, P.y) == pytest.approx(ref2, rel=RTOL64)
    ctx.close()


def test_golden_line_neighbors():
    g = json.load(open(os.path.join(GOLD, "knn_line_m0.json")))
    X = np.array(g["x"])[:, None]
    th = synth.Theta(synth.KIND_IDS[g["kind"]], g["variance"], np.array([g["lengthscale"]]), 0.0)
    ctx = V.Context(X, None, g["mv"], th, precision=V.FP64)
    N = ctx.neighbors()
    for i, exp in enumerate(g["neighbors"]):
        assert [int(j) for j in N[i] if j >= 0] == exp
    ctx.close()


# --------------------------------------------------------------------------- special cases of Sec. 2.1
def test_full_conditioning_is_exact_gp():
    P = prob(45, 2, 8, 44, "matern32", 0.1, 0.2, 11)
    ctx = V.Context(P.X, P.Z, 44, P.theta)
    ex = O.dense_nll(O.exact_cov(P.X, P.theta), P.y)
    assert ctx.nll(P.theta, P.y) == pytest.approx(ex, rel=1e-9)
    ctx.close()


def test_zero_neighbors_is_fitc():
    P = prob(700, 2, 30, 0, "matern52", 0.1, 0.15, 12)
    N = np.zeros((700, 0), dtype=np.int64)
    ref = O.vif_nll(P.X, P.Z, P.theta, N, P.y)
    for prec, tol in [(V.FP64, RTOL64), (V.MIXED, RTOL_MIXED)]:
        ctx = V.Context(P.X, P.Z, 0, P.theta, precision=prec)
        assert nll_close(ctx.nll(P.theta, P.y), ref, 700, tol)
        ctx.close()


def test_no_inducing_points_is_classical_vecchia():
    P = prob(900, 2, 0, 8, "matern12", 0.2, 0.1, 13)
    Nor, keys = oracle_keys_by_row(P, None)
    ref = O.vif_nll(P.X, P.Z, P.theta, Nor, P.y)
    ctx = V.Context(P.X, None, 8, P.theta)
    check_sets(ctx.neighbors(), Nor, keys, 8)
    assert ctx.nll(P.theta, P.y) == pytest.approx(ref, rel=RTOL64)
    ctx.close()


# --------------------------------------------------------------------------- ragged sizes, every kernel
@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "se"])
def test_ragged_sizes_all_kernels(kind):
    ls = np.array([0.3, 0.5, 0.8]) if kind == "se" else 0.25
    P = prob(1037, 3, 45, 7, kind, 0.05, ls, 14)
    Nor, keys = oracle_keys_by_row(P, None)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    ref = vif.nll(P.y)
    ctx = V.Context(P.X, P.Z, 7, P.theta, precision=V.FP64)
    check_sets(ctx.neighbors(), Nor, keys, 7)
    assert ctx.nll(P.theta, P.y) == pytest.approx(ref, rel=RTOL64)
    ctx.close()
    ctx = V.Context(P.X, P.Z, 7, P.theta, precision=V.MIXED, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    assert nll_close(ctx.nll(P.theta, P.y), ref, 1037, RTOL_MIXED)
    ctx.close()


def test_mv30_and_k64_candidate_lists():
    """m_v = 30 uses 64-entry candidate lists and the 6x6-register factor tiles."""
    P = prob(3000, 2, 100, 30, "matern52", 0.05, 0.05, 15)
    Nor, keys = oracle_keys_by_row(P, None)
    ctx = V.Context(P.X, P.Z, 30, P.theta, precision=V.FP64)
    check_sets(ctx.neighbors(), Nor, keys, 30)
    ref = O.VIF(P.X, P.Z, P.theta, Nor).nll(P.y)
    assert ctx.nll(P.theta, P.y) == pytest.approx(ref, rel=RTOL64)
    ctx.close()


@pytest.mark.parametrize("mv", [33, 40, 47])
def test_mixed_factors_with_more_than_32_neighbours(mv):
    """Float32 factors for 32 < m_v + 1 <= 64: the register Cholesky with two rows per lane,
    including the first points of the order (fewer than 32 predecessors)."""
    P = prob(1500, 2, 90, mv, "matern32", 0.05, 0.1, 40 + mv)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, mv)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    ctx = V.Context(P.X, P.Z, mv, P.theta, precision=V.MIXED, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    assert nll_close(ctx.nll(P.theta, P.y), vif.nll(P.y), 1500, RTOL_MIXED)
    Ac, D = ctx.factors()
    ctx.close()
    np.testing.assert_allclose(D, vif.D, rtol=2e-3)
    np.testing.assert_allclose(Ac, vif.Acoef, rtol=2e-3, atol=2e-3 * np.abs(vif.Acoef).max())


# --------------------------------------------------------------------------- failure paths (host-made)
def test_nan_input_reports_not_pd():
    P = prob(300, 2, 20, 5, "matern32", 0.1, 0.2, 16)
    ctx = V.Context(P.X, P.Z, 5, P.theta, neighbor_search=False)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 5)
    ctx.set_neighbors(Nor.astype(np.int32))
    th = P.theta.copy()
    with pytest.raises(V.VifError) as ei:
        ctx.nll(th, P.y)  # fine
        Zbad = P.Z.copy()
        Zbad[3] = np.nan
        ctx2 = V.Context(P.X, Zbad, 5, P.theta, neighbor_search=False)
        ctx2.set_neighbors(Nor.astype(np.int32))
        ctx2.nll(th, P.y)
    assert ei.value.status == V.VIF_ERR_NOT_PD
    # the context stays usable after the error
    assert np.isfinite(ctx.nll(th, P.y))
    ctx.close()


def test_bad_theta_is_rejected():
    P = prob(200, 2, 10, 4, "matern32", 0.1, 0.2, 17)
    ctx = V.Context(P.X, P.Z, 4, P.theta)
    th = P.theta.copy()
    th.lengthscale = np.array([0.1, 0.2, 0.3])
    with pytest.raises(V.VifError) as ei:
        ctx.nll(th, P.y)
    assert ei.value.status == V.VIF_ERR_ARG
    ctx.close()


# --------------------------------------------------------------------------- prediction (Prop. 2.1, App. C.1)
@pytest.mark.parametrize("precision", [V.FP64, V.MIXED])
def test_c1_prediction_matches_oracle(c1, precision):
    P, Nor, keys, vif = c1
    Np = O.pred_neighbors(P.X, P.Z, P.theta, P.Xp, P.mv, vif.lowrank)
    mu_o, var_o = O.predict_appC(vif, P.y, P.Xp, Np)
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=precision, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    mu, var = ctx.predict(P.theta, P.y, P.Xp)
    np.testing.assert_allclose(mu, mu_o, rtol=RTOL64, atol=1e-10)
    np.testing.assert_allclose(var, var_o, rtol=RTOL64)
    mu_l, var_l = ctx.predict(P.theta, P.y, P.Xp, latent=True)
    np.testing.assert_allclose(mu_l, mu_o, rtol=RTOL64, atol=1e-10)
    np.testing.assert_allclose(var_l, var_o - P.theta.nugget, rtol=1e-7)
    ctx.close()


def test_prediction_with_full_conditioning_is_exact_gp():
    P = synth.make_problem(45, 2, 8, 45, "matern52", 1.0, 0.2, 0.1, 21, n_pred=30, lloyd=3)
    ctx = V.Context(P.X, P.Z, 45, P.theta)
    mu, var = ctx.predict(P.theta, P.y, P.Xp)
    mu_e, var_e = O.exact_predict(P.X, P.y, P.theta, P.Xp)
    np.testing.assert_allclose(mu, mu_e, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(var, var_e, rtol=1e-7, atol=1e-9)
    ctx.close()


def test_prediction_without_inducing_points():
    P = synth.make_problem(400, 2, 0, 8, "matern32", 1.0, 0.15, 0.1, 22, n_pred=60, lloyd=3)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 8)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    Np = O.pred_neighbors(P.X, P.Z, P.theta, P.Xp, 8, vif.lowrank)
    mu_o, var_o = O.predict_appC(vif, P.y, P.Xp, Np)
    ctx = V.Context(P.X, None, 8, P.theta, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    mu, var = ctx.predict(P.theta, P.y, P.Xp)
    np.testing.assert_allclose(mu, mu_o, rtol=RTOL64, atol=1e-10)
    np.testing.assert_allclose(var, var_o, rtol=RTOL64)
    ctx.close()


# --------------------------------------------------------------------------- Laplace (Sec. 3-4)
def bern(n, m, mv, seed, ls=0.1, d=2):
    return synth.make_problem(n, d, m, mv, "matern32", 1.0, ls, 0.0, seed, likelihood="bernoulli_logit",
                              lloyd=3)


def test_laplace_mode_matches_oracle_newton_and_pcg():
    P = bern(2000, 30, 10, 31)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 10)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    b_dense, steps_d, _ = O.laplace_mode(vif, P.y, dense=True)
    b_or, steps_o, its_o = O.laplace_mode(vif, P.y, tol=1e-6)
    ctx = V.Context(P.X, P.Z, 10, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6)
    assert np.linalg.norm(b - b_dense) <= 1e-5 * np.linalg.norm(b_dense)
    assert np.linalg.norm(b - b_or) <= 1e-5 * np.linalg.norm(b_or)
    assert abs(st["newton_iters"] - steps_o) <= 1
    assert abs(st["pcg_iters_total"] - its_o) <= 2 * steps_o, (st, its_o)
    # stationarity of the mode, with the oracle's own Sigma_dagger^{-1}
    g, _ = O.bern_grad_W(P.y, b)
    assert np.linalg.norm(g - vif.Sigma_dagger_inv(b)) <= 1e-5 * np.linalg.norm(g)
    ctx.close()


def test_vifdu_without_neighbors_takes_one_cg_step():
    P = bern(1500, 25, 0, 32)
    ctx = V.Context(P.X, P.Z, 0, P.theta, likelihood=V.BERNOULLI_LOGIT)
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8)
    assert st["pcg_iters_total"] == st["newton_iters"]
    vif = O.VIF(P.X, P.Z, P.theta, np.zeros((1500, 0), dtype=np.int64))
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    np.testing.assert_allclose(b, b_dense, rtol=1e-6, atol=1e-8)
    ctx.close()


def test_laplace_with_gpu_neighbors_and_no_inducing_points():
    P = bern(1200, 0, 8, 33)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 8)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    ctx = V.Context(P.X, None, 8, P.theta, likelihood=V.BERNOULLI_LOGIT)
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8)
    assert np.linalg.norm(b - b_dense) <= 1e-6 * np.linalg.norm(b_dense)
    ctx.close()


@pytest.mark.parametrize("shape", ["chain", "star_chain"])
def test_laplace_solves_on_deep_and_wide_dependency_graphs(shape):
    # chain (m_v = 1): N(i) = {i-1}, as many levels as rows, one row each; star_chain
    # (m_v = 2): N(i) = {0, i-1}, so row 0 has n-1 children (the whole warp and several
    # passes of terms in the B^T solve) while the rows still form one long chain
    n = 700
    mv = 1 if shape == "chain" else 2
    P = bern(n, 12, mv, 35)
    N = np.full((n, mv), -1, dtype=np.int64)
    for i in range(1, n):
        if shape == "chain":
            N[i, 0] = i - 1
        else:
            N[i, 0] = 0
            if i >= 2:
                N[i, 1] = i - 1
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    ctx = V.Context(P.X, P.Z, mv, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8)
    assert np.linalg.norm(b - b_dense) <= 1e-6 * np.linalg.norm(b_dense), st
    ctx.close()


def test_solve_waits_give_up_at_their_bound_and_the_context_recovers():
    """The sync-free triangular solves wait on values other warps write; every wait is
    bounded.  With the bound set to one poll (vif_laplace_opts.wait_polls) on the 700-level
    chain, whose rows each wait on the previous one, the waits give up, the kernels return
    and the call reports VIF_ERR_TIMEOUT; the same context then finds the dense-Newton mode
    with the default bound."""
    n = 700
    P = bern(n, 12, 1, 35)
    N = np.full((n, 1), -1, dtype=np.int64)
    N[1:, 0] = np.arange(n - 1)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    ctx = V.Context(P.X, P.Z, 1, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    with pytest.raises(V.VifError) as ei:
        ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8, wait_polls=1)
    assert ei.value.status == V.VIF_ERR_TIMEOUT, str(ei.value)
    assert "timed out" in str(ei.value)
    with pytest.raises(V.VifError) as ei:
        ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8, wait_polls=-1)
    assert ei.value.status == V.VIF_ERR_ARG
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-8)
    assert np.linalg.norm(b - b_dense) <= 1e-6 * np.linalg.norm(b_dense), st
    ctx.close()


# --------------------------------------------------------------------------- VIF-Laplace NLL with SLQ
def _vifla_case(n, m, mv, seed):
    P = bern(n, m, mv, seed)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv) if mv else np.zeros((n, 0), dtype=np.int64)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    ctx = V.Context(P.X, P.Z if m else None, mv, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    if mv:
        ctx.set_neighbors(N.astype(np.int32))
    return P, vif, b_dense, ctx


def test_vifla_nll_with_slq_matches_oracle_probe_by_probe():
    """Eq. log_det_VIFLA with the SLQ of Eq. slq_v1: same normals, same probes (Sec. 4.3), same
    PCG-Lanczos matrices, same quadratures and log-determinants as the oracle."""
    P, vif, b_dense, ctx = _vifla_case(1500, 25, 10, 41)
    eps = synth.slq_normals(6, vif.m, vif.n, seed=5)
    nll, st = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-6, rel_tol=1e-10)
    ref = O.vifla_nll_slq(vif, P.y, b_dense, eps, 1e-6)
    for key in ("neg_log_lik", "quad", "logdet_sigma"):
        assert abs(st[key] - ref[key]) <= 1e-8 * max(1.0, abs(ref[key])), (key, st[key], ref[key])
    assert abs(st["logdet_precond"] - ref["logdet_P"]) <= 1e-8 * abs(ref["logdet_P"])
    np.testing.assert_allclose(st["zPz"], ref["zPz"], rtol=1e-7)
    np.testing.assert_allclose(st["q"], ref["q"], rtol=1e-5, atol=1e-8)
    assert abs(st["pcg_iters_slq"] - int(ref["pcg_iters"].sum())) <= len(eps)
    assert abs(nll - ref["nll"]) <= 1e-7 * abs(ref["nll"]), (nll, ref["nll"])
    assert abs(st["logdet_exact_norm"] - ref["logdet_exact_norm"]) <= 1e-7 * abs(ref["logdet_exact_norm"])
    ctx.close()


@pytest.mark.parametrize("ard", [False, True])
def test_vifla_gradient_by_ste_matches_oracle_probe_by_probe(ard):
    """Sec. 4.1, App. B, App. D: the SLQ probes' CG solutions reused, the same central differences
    of the bilinear forms and log-determinants, the same control variate: s_ik, c_ik, the traces,
    c_k, tau_k and the assembled gradient agree with the oracle (isotropic and ARD ranges)."""
    P = bern(1200, 20, 8, 43)
    if ard:
        P.theta.lengthscale = np.array([0.08, 0.13])
    N = O.causal_neighbors(P.X, P.Z, P.theta, 8)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True, psi_tol=1e-14)
    ctx = V.Context(P.X, P.Z, 8, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    eps = synth.slq_normals(5, vif.m, vif.n, seed=7)
    nll, grad, st = ctx.laplace_nll_grad(P.theta, P.y, eps, slq_tol=1e-10, rel_tol=1e-10)
    ref = O.vifla_grad_ste(P.X, P.Z, P.theta, N, P.y, b_dense, eps, 1e-10, 1e-10)
    q = 1 + np.atleast_1d(P.theta.lengthscale).size
    assert grad.shape == (q,)
    terms = st["probe_terms"]
    for k in range(q):
        sc = np.abs(ref["s"][:, k]).max()
        cc = np.abs(ref["c"][:, k]).max()
        np.testing.assert_allclose(terms[:, k, 0], ref["s"][:, k], rtol=1e-6, atol=1e-7 * sc)
        np.testing.assert_allclose(terms[:, k, 1], ref["c"][:, k], rtol=1e-6, atol=1e-7 * cc)
    np.testing.assert_allclose(st["trace"][:, 2], ref["tau"], rtol=1e-6)
    np.testing.assert_allclose(st["trace"][:, 0], ref["trace_plain"], rtol=1e-6, atol=1e-7 * np.abs(ref["s"]).max())
    np.testing.assert_allclose(st["trace"][:, 1], ref["c_opt"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(st["trace"][:, 3], ref["trace"], rtol=1e-6, atol=1e-7 * np.abs(ref["s"]).max())
    np.testing.assert_allclose(grad, ref["grad"], rtol=1e-5, atol=1e-6 * np.abs(ref["grad"]).max())
    # the factors of theta are back in the context: the likelihood alone is unchanged
    nll2, _ = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-10, rel_tol=1e-10)
    assert abs(nll2 - nll) <= 1e-9 * abs(nll)
    ctx.close()


@pytest.mark.parametrize("m,mv", [(12, 0), (0, 6)])
def test_vifla_gradient_degenerate_structures_match_oracle(m, mv):
    """m_v = 0 (B = I: the VIF is FITC) and m = 0 (classical Vecchia): the same STE gradient as the
    oracle; with m_v = 0 the VIFDU preconditioner is W + Sigma_dagger^{-1} itself, so u_i = P^{-1} z_i
    and every STE sample s_ik equals its control-variate sample c_ik."""
    P, vif, b_dense, ctx = _vifla_case(700, m, mv, 45)
    N = vif.N
    eps = synth.slq_normals(4, vif.m, vif.n, seed=9)
    nll, grad, st = ctx.laplace_nll_grad(P.theta, P.y, eps, slq_tol=1e-10, rel_tol=1e-10)
    ref = O.vifla_grad_ste(P.X, P.Z, P.theta, N, P.y, b_dense, eps, 1e-10, 1e-10)
    np.testing.assert_allclose(st["probe_terms"][:, :, 0], ref["s"], rtol=1e-6, atol=1e-7 * np.abs(ref["s"]).max())
    np.testing.assert_allclose(st["trace"][:, 3], ref["trace"], rtol=1e-6, atol=1e-7 * np.abs(ref["s"]).max())
    np.testing.assert_allclose(grad, ref["grad"], rtol=1e-5, atol=1e-6 * np.abs(ref["grad"]).max())
    if mv == 0:
        pt = st["probe_terms"]
        np.testing.assert_allclose(pt[:, :, 0], pt[:, :, 1], rtol=1e-8, atol=1e-9 * np.abs(pt).max())
    ctx.close()


@pytest.mark.parametrize("ard", [False, True])
def test_vifla_gradient_fitc_form_matches_oracle_probe_by_probe(ard):
    """App. D second form (Eq. pcls2 / slq_v2): FITC probes and their CG solutions reused, bilinear
    forms of Sigma_dagger at the perturbed theta (block solves), the FITC control variate; s_ik, c_ik,
    the traces and the gradient agree with the oracle (isotropic and ARD ranges)."""
    P = bern(1200, 20, 8, 47)
    if ard:
        P.theta.lengthscale = np.array([0.08, 0.13])
    N = O.causal_neighbors(P.X, P.Z, P.theta, 8)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True, psi_tol=1e-14)
    ctx = V.Context(P.X, P.Z, 8, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    eps = synth.slq_normals(5, vif.m, vif.n, seed=7)
    nll, grad, st = ctx.laplace_nll_grad(P.theta, P.y, eps, slq_tol=1e-10, rel_tol=1e-10, precond=V.PRECOND_FITC)
    ref = O.vifla_grad_ste_fitc(P.X, P.Z, P.theta, N, P.y, b_dense, eps, 1e-10, 1e-10)
    q = 1 + np.atleast_1d(P.theta.lengthscale).size
    terms = st["probe_terms"]
    for k in range(q):
        sc = np.abs(ref["s"][:, k]).max()
        cc = np.abs(ref["c"][:, k]).max()
        np.testing.assert_allclose(terms[:, k, 0], ref["s"][:, k], rtol=1e-6, atol=1e-7 * sc)
        np.testing.assert_allclose(terms[:, k, 1], ref["c"][:, k], rtol=1e-6, atol=1e-7 * cc)
    np.testing.assert_allclose(st["trace"][:, 2], ref["tau"], rtol=1e-6)
    np.testing.assert_allclose(st["trace"][:, 3], ref["trace"], rtol=1e-6, atol=1e-7 * np.abs(ref["s"]).max())
    np.testing.assert_allclose(grad, ref["grad"], rtol=1e-5, atol=1e-6 * np.abs(ref["grad"]).max())
    ctx.close()


def test_vifla_gradient_rejects_the_learned_preconditioner():
    P, vif, b_dense, ctx = _vifla_case(300, 10, 5, 44)
    eps = synth.slq_normals(2, vif.m, vif.n, seed=8)
    cv, ls = V.make_cov(P.theta)
    import ctypes as C
    for pre in (1,):
        opts = V.LaplaceOpts(1e-6, 100, 20, pre, 0, None)
        g = np.zeros(2)
        out = C.c_double()
        rc = V.lib().vif_laplace_nll_grad(ctx.h, C.byref(cv), V._ptr(P.y), C.byref(opts), 2, V._ptr(eps), 1e-3,
                                          100, C.byref(out), V._ptr(g), None, None, None)
        assert rc == V.VIF_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("fitc", [False, True])
def test_vifla_slq_with_more_probes_than_one_block_matches_oracle(fitc):
    """70 probes: the probe CGs (VIFDU, Eq. pcls1; FITC, Eq. pcls2) run side by side in blocks of
    at most 64 columns (64 + 6), each column with its own step lengths and stopping test; every
    probe's quadrature and z^T P^{-1} z match the oracle's one-at-a-time CG."""
    P, vif, b_dense, ctx = _vifla_case(500, 12, 6, 46)
    eps = synth.slq_normals(70, vif.m, vif.n, seed=11)
    if fitc:
        nll, st = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-8, rel_tol=1e-10, precond=V.PRECOND_FITC)
        ref = O.vifla_nll_slq_fitc(vif, P.y, b_dense, eps[:, :vif.m + vif.n], 1e-8)
    else:
        nll, st = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-8, rel_tol=1e-10)
        ref = O.vifla_nll_slq(vif, P.y, b_dense, eps, 1e-8)
    np.testing.assert_allclose(st["zPz"], ref["zPz"], rtol=1e-7)
    np.testing.assert_allclose(st["q"], ref["q"], rtol=1e-5, atol=1e-8)
    assert abs(st["pcg_iters_slq"] - int(ref["pcg_iters"].sum())) <= len(eps)
    assert abs(nll - ref["nll"]) <= 1e-7 * abs(ref["nll"])
    ctx.close()


def test_vifla_nll_without_neighbours_is_exact():
    """m_v = 0: P = W + Sigma_dagger^{-1} exactly, every quadrature vanishes and the NLL is the
    dense VIF-Laplace likelihood."""
    P, vif, b_dense, ctx = _vifla_case(800, 20, 0, 42)
    eps = synth.slq_normals(3, vif.m, vif.n, seed=6)
    nll, st = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-8, rel_tol=1e-10)
    np.testing.assert_allclose(st["q"], 0.0, atol=1e-10)
    exact = -O.bern_loglik(P.y, b_dense) + 0.5 * float(b_dense @ vif.Sigma_dagger_inv(b_dense)) \
        + 0.5 * O.vifla_logdet_dense(vif, b_dense)
    assert abs(nll - exact) <= 1e-8 * abs(exact), (nll, exact)
    ctx.close()


def test_vifla_nll_untrained_learned_correction_equals_plain_vifdu():
    """An untrained network outputs c = 0, so W' = W: the learned variant of the SLQ (probes,
    preconditioner and log det P all use W') must reproduce plain VIFDU."""
    P, vif, b_dense, ctx = _vifla_case(1200, 20, 8, 43)
    eps = synth.slq_normals(4, vif.m, vif.n, seed=7)
    net = V.Network(seed=3)
    a, sa = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-6, rel_tol=1e-10)
    b, sb = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-6, rel_tol=1e-10, precond=1, mlp_weights=net)
    assert abs(a - b) <= 1e-9 * abs(a)
    np.testing.assert_allclose(sa["q"], sb["q"], rtol=1e-9, atol=1e-12)
    ctx.close()


def test_laplace_mode_with_fitc_preconditioner_matches_oracle():
    """FITC preconditioner (App. E.2) with the system form of Eq. pcls2: the mode equals the dense
    Newton mode and the CG counts follow the oracle's pcls2 PCG."""
    P, vif, b_dense, ctx = _vifla_case(1500, 25, 10, 44)
    b, st = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6, precond=V.PRECOND_FITC)
    b_or, steps_o, its_o = O.laplace_mode_fitc(vif, P.y, tol=1e-6)
    assert np.linalg.norm(b - b_dense) <= 1e-5 * np.linalg.norm(b_dense)
    assert np.linalg.norm(b - b_or) <= 1e-5 * np.linalg.norm(b_or)
    assert abs(st["newton_iters"] - steps_o) <= 1
    assert abs(st["pcg_iters_total"] - its_o) <= 2 * steps_o, (st, its_o)
    ctx.close()


def test_vifla_nll_with_fitc_slq_matches_oracle_probe_by_probe():
    """Eq. slq_v2 with the FITC preconditioner: same normals, same probes, same quadratures."""
    P, vif, b_dense, ctx = _vifla_case(1500, 25, 10, 45)
    eps = synth.slq_normals(6, vif.m, vif.n, seed=8)
    nll, st = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-6, rel_tol=1e-10, precond=V.PRECOND_FITC)
    ref = O.vifla_nll_slq_fitc(vif, P.y, b_dense, eps[:, :vif.m + vif.n], 1e-6)
    assert abs(st["logdet_precond"] - ref["logdet_P"]) <= 1e-8 * abs(ref["logdet_P"])
    np.testing.assert_allclose(st["zPz"], ref["zPz"], rtol=1e-7)
    np.testing.assert_allclose(st["q"], ref["q"], rtol=1e-5, atol=1e-8)
    assert abs(nll - ref["nll"]) <= 1e-7 * abs(ref["nll"]), (nll, ref["nll"])
    # both SLQ forms estimate the same log-determinant
    nll1, st1 = ctx.laplace_nll(P.theta, P.y, eps, slq_tol=1e-6, rel_tol=1e-10)
    assert abs(st["quad"] - st1["quad"]) <= 1e-8 * abs(st1["quad"])
    ctx.close()


def test_laplace_prediction_with_sbpv_matches_oracle():
    """Prop. 3.1 means and Alg. 1 (SBPV) variances with the same normals as the oracle; the FITC
    solves (Eq. pcls2) give the same draws z7 and so the same variances."""
    P = synth.make_problem(1500, 2, 25, 10, "matern32", 1.0, 0.1, 0.0, 46, likelihood="bernoulli_logit",
                           lloyd=3, n_pred=150)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 10)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_dense, _, _ = O.laplace_mode(vif, P.y, dense=True)
    Np = O.pred_neighbors(P.X, P.Z, P.theta, P.Xp, 10)
    eps = synth.slq_normals(8, vif.m, vif.n, seed=9)
    mu_o, var_o, _ = O.laplace_predict_sbpv(vif, P.y, b_dense, P.Xp, Np, eps, 1e-10)
    ctx = V.Context(P.X, P.Z, 10, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(N.astype(np.int32))
    mu, var, st = ctx.laplace_predict(P.theta, P.y, P.Xp, eps, cg_tol=1e-10, rel_tol=1e-10)
    np.testing.assert_allclose(mu, mu_o, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(var, var_o, rtol=1e-6, atol=1e-9)
    mu_f, var_f, _ = ctx.laplace_predict(P.theta, P.y, P.Xp, eps, cg_tol=1e-10, rel_tol=1e-10,
                                         precond=V.PRECOND_FITC)
    np.testing.assert_allclose(mu_f, mu_o, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(var_f, var_o, rtol=1e-6, atol=1e-9)
    mu_n, var_n, _ = ctx.laplace_predict(P.theta, P.y, P.Xp)
    assert var_n is None
    np.testing.assert_allclose(mu_n, mu_o, rtol=1e-5, atol=1e-7)
    ctx.close()


def test_laplace_rejects_a_nugget():
    P = bern(300, 10, 4, 34)
    ctx = V.Context(P.X, P.Z, 4, P.theta, likelihood=V.BERNOULLI_LOGIT)
    th = P.theta.copy()
    th.nugget = 0.1
    with pytest.raises(V.VifError) as ei:
        ctx.laplace_mode(th, P.y)
    assert ei.value.status == V.VIF_ERR_ARG
    ctx.close()


# --------------------------------------------------------------------------- gradient (Sec. 2.2)
def test_c1_gradient_matches_oracle(c1):
    """The reverse-mode gradient against the oracle's Sec. 2.2 / App. A form (float64 on both
    sides; a mixed context forms it from a float64 pass) and against central differences."""
    P, Nor, keys, vif = c1
    g_or = O.vif_nll_grad(P.X, P.Z, P.theta, Nor, P.y)
    g_fd = O.vif_nll_grad_fd(P.X, P.Z, P.theta, Nor, P.y)
    np.testing.assert_allclose(g_fd, g_or, rtol=1e-6, atol=1e-6 * np.abs(g_or).max())
    for prec in (V.FP64, V.MIXED):
        ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=prec, neighbor_search=False)
        ctx.set_neighbors(Nor.astype(np.int32))
        nll, g = ctx.nll(P.theta, P.y, grad=True)
        np.testing.assert_allclose(g, g_or, rtol=1e-8, atol=1e-9 * np.abs(g_or).max())
        assert nll_close(nll, vif.nll(P.y), 2000, RTOL64 if prec == V.FP64 else RTOL_MIXED)
        # the same likelihood without the gradient (float64 atomics in the triangular inverse
        # and the mixed path's autotuned factor stage may move the last bits)
        nll2 = ctx.nll(P.theta, P.y)
        assert nll2 == pytest.approx(nll, rel=1e-12 if prec == V.FP64 else RTOL_MIXED)
        ctx.close()


@pytest.mark.parametrize("m,mv,kind,ls,d", [
    (30, 12, "matern52", 0.15, 2),
    (25, 8, "se", [0.3, 0.7, 1.2], 3),
    (0, 9, "matern32", 0.2, 2),
    (20, 0, "matern12", 0.2, 2),
    (40, 36, "matern32", 0.1, 2)])
def test_gradient_matches_oracle_across_structures(m, mv, kind, ls, d):
    """ARD length scales, no inducing points (classical Vecchia), no neighbours (FITC) and
    more than 32 neighbours, all kernel families."""
    P = prob(700, d, m, mv, kind, 0.08, np.array(ls) if np.ndim(ls) else ls, 60 + mv)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, mv) if mv else -np.ones((700, 0), dtype=np.int64)
    g_or = O.vif_nll_grad(P.X, P.Z, P.theta, Nor, P.y)
    ctx = V.Context(P.X, P.Z, mv, P.theta, precision=V.FP64, neighbor_search=False)
    if mv:
        ctx.set_neighbors(Nor.astype(np.int32))
    nll, g = ctx.nll(P.theta, P.y, grad=True)
    ctx.close()
    assert g.shape == g_or.shape
    np.testing.assert_allclose(g, g_or, rtol=1e-7, atol=1e-8 * np.abs(g_or).max())
    assert nll == pytest.approx(O.vif_nll(P.X, P.Z, P.theta, Nor, P.y), rel=RTOL64)


def test_gradient_with_full_conditioning_is_the_exact_gp_gradient():
    P = synth.make_problem(45, 2, 8, 45, "matern32", 1.0, 0.2, 0.1, 41, lloyd=3)
    ctx = V.Context(P.X, P.Z, 45, P.theta)
    _, g = ctx.nll(P.theta, P.y, grad=True)
    np.testing.assert_allclose(g, O.exact_gp_grad(P.X, P.y, P.theta), rtol=1e-8, atol=1e-8)
    ctx.close()


# --------------------------------------------------------------------------- batched problems (one graph)
def test_batch_graph_replay_matches_single_problem_calls():
    torch = pytest.importorskip("torch")
    probs = synth.config5(nprob=10, n_lo=300, n_hi=2500)
    ctxs, ys, ref = [], [], []
    for k, P in enumerate(probs):
        prec = V.MIXED if k % 2 else V.FP64
        c = V.Context(P.X, P.Z, P.mv, P.theta, precision=prec)
        ctxs.append(c)
        ys.append(torch.from_numpy(P.y).cuda())
        ref.append(c.nll(P.theta, P.y))
    B = V.Batch(ctxs, [P.theta for P in probs], ys)
    for _ in range(2):
        got = B.run()
        # the triangular inverse adds its k-slices with float64 atomics, so the last bits
        # of L_m^{-1} (and of everything after it) depend on the order they land in
        np.testing.assert_allclose(got, ref, rtol=1e-10)
    info = B.info()
    assert info["branches"] in (4, 8, 16, 32) and info["best_replay_ms"] > 0
    # every float64 problem (m_v + 1 <= 49) has its factor stage in a bucket
    assert info["bucketed_problems"] >= 5 and info["factor_buckets"] >= 1
    # each shape, the bucket launches included, gives the single calls' likelihoods
    for shape in ((8, 1, 0), (8, 1, 1), (16, 2, 1), (4, 1, 2), (32, 1, 2)):
        B.set_shape(*shape)
        assert B.info()["batched_factor"] == shape[2]
        for _ in range(2):
            np.testing.assert_allclose(B.run(), ref, rtol=1e-10)
    with pytest.raises(V.VifError):
        B.set_shape(8, 1, 3)
    # float64 and mixed problems against the oracle on the GPU's neighbour sets' definition
    for k in (0, 1, 2, 3, 4, 5):
        P = probs[k]
        Nor = O.causal_neighbors(P.X, P.Z, P.theta, P.mv)
        tol = RTOL_MIXED if k % 2 else RTOL64
        assert nll_close(got[k], O.vif_nll(P.X, P.Z, P.theta, Nor, P.y), P.X.shape[0], tol), (k, got[k])
    B.close()
    for c in ctxs:
        c.close()


def test_batch_with_more_cholesky_blocks_than_fit_at_once():
    """200 problems with m = 256: the batched Cholesky's first panel launch has 3200 CTAs
    (3400 for the capacitance matrices), more than the GPU holds at once, so CTAs of one
    problem's panel start after others of it have finished.  The likelihoods equal the
    single-problem calls'."""
    torch = pytest.importorskip("torch")
    probs = [synth.make_problem(300, 2, 256, 8, "matern32", 1.0, 0.2, 0.1, 9000 + k, lloyd=1) for k in range(200)]
    ctxs, ys, ref = [], [], []
    for P in probs:
        c = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64)
        ctxs.append(c)
        ys.append(torch.from_numpy(P.y).cuda())
        ref.append(c.nll(P.theta, P.y))
    B = V.Batch(ctxs, [P.theta for P in probs], ys)
    for _ in range(2):
        np.testing.assert_allclose(B.run(), ref, rtol=1e-10)
    B.close()
    for c in ctxs:
        c.close()


# --------------------------------------------------------------------------- learned correction
from oracle import mlp_oracle as MO


def _f16(x):
    return np.asarray(x, dtype=np.float16).astype(np.float64)


def test_mlp_forward_and_backward_match_oracle():
    rng = np.random.default_rng(11)
    p = _f16(rng.normal(0, 0.3, MO.NPARAM))
    net = V.Network(params=p.astype(np.float32))
    F = rng.normal(0, 1, (3001, MO.NIN)).astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(net.forward(F), MO.forward(p, F), rtol=2e-5, atol=2e-5)
    gc = rng.normal(0, 1, 3001).astype(np.float32).astype(np.float64)
    g_gpu = net.backward(F, gc)
    g_or = MO.backward(p, F, gc)
    assert np.linalg.norm(g_gpu - g_or) <= 1e-4 * np.linalg.norm(g_or)
    np.testing.assert_allclose(net.params(), p.astype(np.float32), rtol=0, atol=0)


def test_mlp_features_match_oracle_and_untrained_network_is_plain_vifdu():
    P = bern(1500, 30, 8, 51)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 8)
    ctx = V.Context(P.X, P.Z, 8, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    b0, st0 = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6)
    _, W = O.bern_grad_W(P.y, b0)
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    F_or = MO.features(W, vif.D, vif.Acoef, Nor, 8, O.residual_neighbor_corr(P.X, P.Z, P.theta, Nor))
    F_gpu = ctx.mlp_features(W)
    np.testing.assert_allclose(F_gpu, F_or, rtol=1e-4, atol=1e-5)
    net = V.Network(seed=3)                       # zero output layer: c = 0
    b1, st1 = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6, precond=1, mlp_weights=net)
    assert st1["pcg_iters_total"] == st0["pcg_iters_total"]
    np.testing.assert_allclose(b1, b0, rtol=1e-12, atol=1e-12)
    ctx.close()


def test_trained_correction_needs_fewer_cg_iterations_on_a_held_out_problem():
    """The committed weights (trained on 5000 Newton systems of n = 2e4 Bernoulli-logit
    problems, Matern-3/2 ranges in [0.03, 0.1]) against the plain VIFDU preconditioner on a
    problem of that shape whose seed no training problem used: both reach the same mode at
    the same CG tolerance, the learned correction in fewer CG iterations."""
    p = np.load(os.path.join(ROOT, "paper_2507_05064_gb300", "weights", "vifdu_mlp.npy"))
    assert p.shape == (V.MLP_NPARAM,)
    P = synth.make_problem(20_000, 2, 200, 20, "matern32", 1.0, 0.05, 0.0, 9_100_001,
                           likelihood="bernoulli_logit", lloyd=2, rff=256)
    ctx = V.Context(P.X, P.Z, 20, P.theta, likelihood=V.BERNOULLI_LOGIT)
    net = V.Network(params=p.astype(np.float32))
    b_p, s_p = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6)
    b_l, s_l = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6, precond=1, mlp_weights=net)
    ctx.close()
    print("CG iterations plain", s_p["pcg_iters_total"], "learned", s_l["pcg_iters_total"],
          "Newton", s_p["newton_iters"], s_l["newton_iters"])
    assert np.linalg.norm(b_l - b_p) <= 1e-5 * np.linalg.norm(b_p)
    assert s_l["pcg_iters_total"] <= 0.9 * s_p["pcg_iters_total"]


def test_training_lowers_the_preconditioner_loss():
    P = bern(3000, 40, 10, 52, ls=0.05)
    Nor = O.causal_neighbors(P.X, P.Z, P.theta, 10)
    ctx = V.Context(P.X, P.Z, 10, P.theta, likelihood=V.BERNOULLI_LOGIT, neighbor_search=False)
    ctx.set_neighbors(Nor.astype(np.int32))
    net = V.Network(seed=4)
    st = ctx.mlp_train(P.theta, P.y, net, steps_per_system=15, probes=4, max_newton=3, lr=3e-3)
    assert st["systems"] == 3 and st["loss_last"] < st["loss_first"]
    b, s_l = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6, precond=1, mlp_weights=net)
    _, s_p = ctx.laplace_mode(P.theta, P.y, rel_tol=1e-6)
    print("CG iterations plain", s_p["pcg_iters_total"], "learned", s_l["pcg_iters_total"], st)
    g, _ = O.bern_grad_W(P.y, b)            # the learned preconditioner still reaches the mode
    vif = O.VIF(P.X, P.Z, P.theta, Nor)
    assert np.linalg.norm(g - vif.Sigma_dagger_inv(b)) <= 1e-5 * np.linalg.norm(g)
    ctx.close()
