"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(special cases, closed forms, library routines, invariants, hand-worked cases).
None of them re-types the oracle's own formula.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as ss
from scipy.spatial.distance import cdist

from oracle import vif_oracle as O
from paper_2507_05064_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(n=300, d=2, m=20, mv=8, kind="matern32", nugget=0.1, seed=1, ls=0.2,
                  likelihood="gaussian", n_pred=0, inducing="kmeans++"):
    return synth.make_problem(n, d, m, mv, kind, 1.0, ls, nugget, seed, likelihood=likelihood,
                              inducing=inducing, n_pred=n_pred, lloyd=3)


# --------------------------------------------------------------------------- kernels
@pytest.mark.parametrize("kind,nu", [(0, 0.5), (1, 1.5), (2, 2.5)])
def test_matern_half_integer_forms_match_bessel_definition(kind, nu):
    """General Matern: s^2 2^{1-nu}/Gamma(nu) (sqrt(2nu) r)^nu K_nu(sqrt(2nu) r)."""
    r = np.array([1e-3, 0.05, 0.3, 1.0, 2.5, 7.0])
    t = math.sqrt(2 * nu) * r
    ref = 2.0 ** (1 - nu) / ss.gamma(nu) * t ** nu * ss.kv(nu, t) * 1.7
    np.testing.assert_allclose(O.cov_of_r(r, kind, 1.7), ref, rtol=1e-12)
    assert O.cov_of_r(np.array([0.0]), kind, 1.7)[0] == pytest.approx(1.7)


def test_se_is_the_characteristic_function_of_its_spectral_density():
    """Bochner: the SE kernel exp(-r^2/2) is E[cos(w r)] with w ~ N(0,1); quadrature."""
    from scipy.integrate import quad
    r = np.array([0.05, 0.3, 1.0, 2.0])
    ref = [quad(lambda w, rr=rr: math.cos(w * rr) * math.exp(-0.5 * w * w) / math.sqrt(2 * math.pi),
                -40, 40, limit=400)[0] for rr in r]
    np.testing.assert_allclose(O.cov_of_r(r, 3, 1.0), ref, rtol=1e-10)


def test_ard_scaling_is_coordinatewise():
    th = synth.Theta(1, 1.0, np.array([0.1, 2.0]), 0.0)
    X1 = np.array([[0.1, 0.5]])
    X2 = np.array([[0.2, 0.5], [0.1, 2.5]])
    # a 0.1 shift in dim 0 (length 0.1) equals a 2.0 shift in dim 1 (length 2.0)
    k = O.cov(X1, X2, th)[0]
    assert k[0] == pytest.approx(k[1], rel=1e-14)
    assert k[0] == pytest.approx(O.cov_of_r(np.array([1.0]), 1, 1.0)[0], rel=1e-14)


# --------------------------------------------------------------------------- low rank
def test_lowrank_reproduces_sigma_when_inducing_points_are_the_data():
    """Predictive process with S* = S: Sigma^l = Sigma (Sec. 2.1), up to the jitter."""
    P = small_problem(n=60, m=0)
    th = P.theta
    lr = O.LowRank(P.X, P.X.copy(), th)
    Sl = lr.Smn.T @ lr.SinvSmn
    np.testing.assert_allclose(Sl, O.cov(P.X, P.X, th), atol=1e-8)


def test_lowrank_is_psd_and_below_sigma():
    P = small_problem(n=200, m=30)
    lr = O.LowRank(P.X, P.Z, P.theta)
    Sl = lr.Smn.T @ lr.SinvSmn
    R = O.cov(P.X, P.X, P.theta) - Sl
    assert np.linalg.eigvalsh(Sl).min() > -1e-9
    assert np.linalg.eigvalsh(R).min() > -1e-9          # Cov(b_s) is PSD
    # independent route: general LU solve instead of the Cholesky solve
    Sl2 = lr.Smn.T @ np.linalg.solve(O.sigma_m(P.Z, P.theta), lr.Smn)
    np.testing.assert_allclose(Sl, Sl2, atol=1e-9)


# --------------------------------------------------------------------------- neighbours
def test_knn_golden_line():
    g = json.load(open(os.path.join(GOLD, "knn_line_m0.json")))
    X = np.array(g["x"])[:, None]
    th = synth.Theta(synth.KIND_IDS[g["kind"]], g["variance"], np.array([g["lengthscale"]]), 0.0)
    N = O.causal_neighbors(X, np.zeros((0, 1)), th, g["mv"])
    for i, exp in enumerate(g["neighbors"]):
        got = [int(j) for j in N[i] if j >= 0]
        assert got == exp, (i, got, exp)


def test_knn_without_inducing_points_is_scaled_euclidean_knn():
    P = small_problem(n=250, d=3, m=0, mv=7, ls=np.array([0.1, 0.3, 0.9]))
    N = O.causal_neighbors(P.X, P.Z, P.theta, 7)
    Dm = cdist(P.X / P.theta.lengthscale, P.X / P.theta.lengthscale)
    for i in range(1, 250):
        q = min(i, 7)
        ref = np.sort(np.lexsort((np.arange(i), Dm[i, :i]))[:q])
        assert list(N[i, :q]) == list(ref)


def test_knn_matches_dense_residual_correlation_brute_force():
    """Brute force from the dense residual covariance Sigma - Sigma^l and d_c itself."""
    P = small_problem(n=180, m=15, mv=6, kind="matern52")
    th = P.theta
    N = O.causal_neighbors(P.X, P.Z, th, 6)
    S = O.cov(P.X, P.X, th)
    Sm = O.sigma_m(P.Z, th)
    Snm = O.cov(P.X, P.Z, th)
    R = S - Snm @ np.linalg.solve(Sm, Snm.T)
    dgl = np.diag(R)
    dc = np.sqrt(1.0 - np.minimum(np.abs(R / np.sqrt(np.outer(dgl, dgl))), 1.0))
    np.testing.assert_allclose(dc, dc.T, atol=1e-12)          # d_c is symmetric
    for i in range(1, 180):
        q = min(i, 6)
        ref = np.sort(np.lexsort((np.arange(i), dc[i, :i]))[:q])
        assert list(N[i, :q]) == list(ref), i


@pytest.mark.parametrize("m,nugget", [(15, 0.0), (0, 0.0), (15, 0.1)])
def test_residual_neighbour_correlations_from_the_dense_residual_covariance(m, nugget):
    """Inputs 8-9 of the learned correction against the dense residual covariance
    Sigma~ - Sigma^l (a dense solve, not the oracle's Cholesky route) and, without a
    nugget, against the keys the neighbour search ranked by: the chosen |rho| are the
    largest ones, so their maximum is 1 - the smallest chosen key."""
    P = small_problem(n=160, m=m, mv=6, kind="matern32", nugget=nugget, seed=7)
    th = P.theta
    N, keys, _ = O.causal_neighbors(P.X, P.Z, th, 6, return_keys=True)
    rho = O.residual_neighbor_corr(P.X, P.Z, th, N)
    R = O.cov(P.X, P.X, th) + O.residual_diag(th) * np.eye(160)
    if m:
        Snm = O.cov(P.X, P.Z, th)
        R = R - Snm @ np.linalg.solve(O.sigma_m(P.Z, th), Snm.T)
    C = np.abs(R / np.sqrt(np.outer(np.diag(R), np.diag(R))))
    assert np.all(rho[0] == 0.0)
    for i in range(1, 160):
        nb = N[i][N[i] >= 0]
        np.testing.assert_allclose(rho[i], [C[i, nb].max(), C[i, nb].mean()], rtol=1e-10, atol=1e-13)
        assert 0.0 <= rho[i, 1] <= rho[i, 0] <= 1.0
        if nugget == 0.0:
            # the residual diagonal then carries only the jitter, which moves rho by at
            # most about jitter / (smallest residual variance involved)
            kk = keys[i - 1]
            tol = 4.0 * O.residual_diag(th) / np.diag(R)[np.r_[i, nb]].min() + 1e-13
            assert abs(rho[i, 0] - (1.0 - kk[nb].min())) <= tol
            assert abs(rho[i, 1] - (1.0 - kk[nb]).mean()) <= tol
    if m == 0:                 # no inducing points: rho is the correlation function itself
        i = 100
        nb = N[i][N[i] >= 0]
        r = O.dist(O.scaled(P.X[i:i + 1], th), O.scaled(P.X[nb], th))[0]
        corr = O.cov_of_r(r, th.kind, 1.0) / (1.0 + O.residual_diag(th) / th.variance)
        np.testing.assert_allclose(rho[i], [corr.max(), corr.mean()], rtol=1e-12)


@pytest.mark.parametrize("m,kind,d", [(20, "matern32", 2), (0, "matern32", 2), (12, "se", 3)])
def test_sampled_neighbor_search_equals_the_full_brute_force(m, kind, d):
    """The streaming form used at full size (chunks of predecessors, low-rank terms of the
    queries alone) returns the sets and keys of the pinned full brute force: queries at,
    just before and just after chunk boundaries (chunk = 7), the first points (fewer than
    m_v predecessors) and the last point; m = 0 (no low-rank part) included."""
    ls = 0.2 if d == 2 else np.array([0.3, 0.6, 1.1])
    P = synth.make_problem(300, d, m, 8, kind, 1.0, ls, 0.1, 11, inducing="kmeans++", lloyd=2)
    th = P.theta
    N, keys, _ = O.causal_neighbors(P.X, P.Z, th, 8, return_keys=True)
    queries = [1, 2, 3, 6, 7, 8, 13, 14, 15, 20, 21, 22, 49, 133, 140, 141, 298, 299]
    Ns, ks = O.causal_neighbors_sample(P.X, P.Z, th, 8, queries, chunk=7)
    for a, i in enumerate(queries):
        q = min(i, 8)
        assert list(Ns[a]) == list(N[i, :q]), i
        np.testing.assert_allclose(ks[a], keys[i - 1], rtol=0, atol=1e-13)
        assert len(ks[a]) == i


# --------------------------------------------------------------------------- factors
def test_vecchia_factor_invariants():
    P = small_problem(n=300, m=25, mv=10, nugget=0.05)
    th = P.theta
    N10 = O.causal_neighbors(P.X, P.Z, th, 10)
    N4 = O.causal_neighbors(P.X, P.Z, th, 4)
    lr = O.LowRank(P.X, P.Z, th)
    _, D10 = O.vecchia_factors(P.X, P.Z, th, N10, lr)
    _, D4 = O.vecchia_factors(P.X, P.Z, th, N4, lr)
    ctilde = th.variance + th.nugget - lr.lr_diag()
    assert (D10 > 0).all() and (D10 <= ctilde + 1e-12).all()
    assert (D10 >= th.nugget - 1e-12).all()                 # noise is never explained away
    # the 4 nearest are a subset of the 10 nearest, so conditioning on more can only shrink D
    for i in range(300):
        assert set(N4[i][N4[i] >= 0]) <= set(N10[i][N10[i] >= 0])
    assert (D10 <= D4 + 1e-12).all()


@pytest.mark.parametrize("m,nugget", [(25, 0.05), (0, 0.05), (25, 0.0)])
def test_row_sampled_factors_equal_the_full_factors(m, nugget):
    """The per-row form used at full size (low-rank terms rebuilt on the rows and their
    neighbours only, indices remapped) gives the A_i, D_i of the pinned full form, for
    rows with fewer than m_v predecessors (i < m_v), rows sharing neighbours, and the last
    row; with and without inducing points and nugget."""
    P = small_problem(n=300, m=m, mv=10, nugget=nugget)
    th = P.theta
    N = O.causal_neighbors(P.X, P.Z, th, 10)
    Af, Df = O.vecchia_factors(P.X, P.Z, th, N)
    rows = np.array([0, 1, 2, 5, 9, 10, 11, 57, 58, 150, 151, 299])
    Ar, Dr = O.vecchia_factors_rows(P.X, P.Z, th, N, rows)
    np.testing.assert_allclose(Ar, Af[rows], rtol=0, atol=1e-10 * max(1.0, np.abs(Af).max()))
    np.testing.assert_allclose(Dr, Df[rows], rtol=1e-10)
    assert (Ar[0] == 0).all() and (Ar[2, 2:] == 0).all()


# --------------------------------------------------------------------------- likelihood
def test_full_conditioning_gives_the_exact_gp_likelihood():
    """m_v = n-1: the residual Vecchia is exact, so Sigma~_dagger = Sigma~ for any m, Z."""
    P = small_problem(n=120, m=15, mv=119, nugget=0.1)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 119)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    ex = O.dense_nll(O.exact_cov(P.X, P.theta), P.y)
    assert vif.nll(P.y) == pytest.approx(ex, rel=1e-10)


def test_full_conditioning_with_no_inducing_points_is_exact():
    P = small_problem(n=90, m=0, mv=89, nugget=0.2, kind="matern12")
    N = O.causal_neighbors(P.X, P.Z, P.theta, 89)
    ex = O.dense_nll(O.exact_cov(P.X, P.theta), P.y)
    assert O.vif_nll(P.X, P.Z, P.theta, N, P.y) == pytest.approx(ex, rel=1e-10)


def test_zero_neighbours_is_fitc():
    """m_v = 0: Sigma^l + diag(Sigma~ - Sigma^l) (Sec. 2.1, special case)."""
    P = small_problem(n=200, m=20, mv=0, nugget=0.1)
    th = P.theta
    N = np.zeros((200, 0), dtype=np.int64)
    Snm = O.cov(P.X, P.Z, th)
    Sl = Snm @ np.linalg.solve(O.sigma_m(P.Z, th), Snm.T)
    fitc = Sl + np.diag(th.variance + th.nugget - np.diag(Sl))
    assert O.vif_nll(P.X, P.Z, th, N, P.y) == pytest.approx(O.dense_nll(fitc, P.y), rel=1e-11)


def test_no_inducing_points_is_classical_vecchia():
    """m = 0: Vecchia of Sigma~ itself, built densely here with textbook conditionals."""
    P = small_problem(n=150, m=0, mv=6, nugget=0.1, kind="matern52")
    th = P.theta
    N = O.causal_neighbors(P.X, P.Z, th, 6)
    S = O.exact_cov(P.X, th)
    n = 150
    Bd = np.eye(n)
    Dd = np.empty(n)
    for i in range(n):
        nb = [j for j in N[i] if j >= 0]
        if nb:
            a = np.linalg.solve(S[np.ix_(nb, nb)], S[nb, i])
            Bd[i, nb] = -a
            Dd[i] = S[i, i] - S[i, nb] @ a
        else:
            Dd[i] = S[i, i]
    Sv = np.linalg.inv(Bd.T @ np.diag(1 / Dd) @ Bd)
    assert O.vif_nll(P.X, P.Z, th, N, P.y) == pytest.approx(O.dense_nll(Sv, P.y), rel=1e-10)


@pytest.mark.parametrize("m,mv,kind,nugget", [(30, 8, "matern32", 0.1), (0, 6, "matern52", 0.05),
                                              (25, 0, "se", 0.02)])
def test_whitened_evaluation_equals_the_m_form_and_the_dense_likelihood(m, mv, kind, nugget):
    """nll_whitened (the Sylvester ratio det M / det Sigma_m as det(L_m^{-1} M L_m^{-T})) gives the
    likelihood of the M form and of the explicitly formed Sigma~_dagger, with and without
    inducing points and neighbours."""
    P = small_problem(n=400, m=m, mv=mv, kind=kind, nugget=nugget, ls=0.25)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv) if mv else np.zeros((400, 0), dtype=np.int64)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    a, b = vif.nll_whitened(P.y), vif.nll(P.y)
    dense = O.dense_nll(vif.dense_Sigma_dagger(), P.y)
    assert a == pytest.approx(b, rel=1e-11)
    assert a == pytest.approx(dense, rel=1e-10)


def test_woodbury_sylvester_equals_dense_vif_likelihood():
    P = small_problem(n=250, m=25, mv=7, nugget=0.05, kind="se", ls=np.array([0.1, 0.2]))
    N = O.causal_neighbors(P.X, P.Z, P.theta, 7)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    assert vif.nll(P.y) == pytest.approx(O.dense_nll(vif.dense_Sigma_dagger(), P.y), rel=1e-10)


# --------------------------------------------------------------------------- prediction
def test_prediction_prop21_equals_appendix_c_form():
    P = small_problem(n=200, m=20, mv=8, nugget=0.1, n_pred=40)
    th = P.theta
    N = O.causal_neighbors(P.X, P.Z, th, 8)
    vif = O.VIF(P.X, P.Z, th, N)
    Np = O.pred_neighbors(P.X, P.Z, th, P.Xp, 8, vif.lowrank)
    mu1, S1 = O.predict_prop21_dense(vif, P.y, P.Xp, Np)
    mu2, v2 = O.predict_appC(vif, P.y, P.Xp, Np)
    np.testing.assert_allclose(mu1, mu2, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(np.diag(S1), v2, rtol=1e-8)


def test_prediction_with_full_conditioning_is_exact_gp_prediction():
    P = small_problem(n=100, m=12, mv=99, nugget=0.1, n_pred=15)
    th = P.theta
    N = O.causal_neighbors(P.X, P.Z, th, 99)
    vif = O.VIF(P.X, P.Z, th, N)
    Np = np.tile(np.arange(100), (15, 1))
    mu, var = O.predict_appC(vif, P.y, P.Xp, Np)
    mu_e, var_e = O.exact_predict(P.X, P.y, th, P.Xp)
    np.testing.assert_allclose(mu, mu_e, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(var, var_e, rtol=1e-7, atol=1e-9)


# --------------------------------------------------------------------------- Laplace
def test_vifdu_formula_equals_dense_definition():
    """App. E.1: the solve formula inverts P^ = B^T W B + Sigma_dagger^{-1}."""
    P = small_problem(n=120, m=12, mv=5, nugget=0.0, likelihood="bernoulli_logit")
    N = O.causal_neighbors(P.X, P.Z, P.theta, 5)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    W = np.random.default_rng(3).uniform(0.05, 0.25, 120)
    pre = O.VIFDU(vif, W)
    Pd = pre.dense(W)
    w = np.random.default_rng(4).standard_normal(120)
    np.testing.assert_allclose(pre.apply(w), np.linalg.solve(Pd, w), rtol=1e-8, atol=1e-10)


def test_vifdu_without_neighbours_is_exact_so_pcg_takes_one_step():
    P = small_problem(n=150, m=15, mv=0, nugget=0.0, likelihood="bernoulli_logit")
    N = np.zeros((150, 0), dtype=np.int64)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    W = np.random.default_rng(5).uniform(0.05, 0.25, 150)
    pre = O.VIFDU(vif, W)
    v = np.random.default_rng(6).standard_normal(150)
    _, it, rel = O.pcg(lambda w: W * w + vif.Sigma_dagger_inv(w), pre.apply, v, 1e-10, 50)
    assert it == 1 and rel < 1e-10


def test_laplace_mode_is_stationary_and_pcg_agrees_with_dense_newton():
    P = small_problem(n=200, m=15, mv=6, nugget=0.0, likelihood="bernoulli_logit",
                      kind="matern32", ls=0.15)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 6)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b_d, _, _ = O.laplace_mode(vif, P.y, dense=True)
    g, _ = O.bern_grad_W(P.y, b_d)
    stat = np.linalg.norm(g - np.linalg.solve(vif.dense_Sigma_dagger(), b_d)) / np.linalg.norm(g)
    assert stat < 1e-8
    b_p, steps, its = O.laplace_mode(vif, P.y, tol=1e-10)
    np.testing.assert_allclose(b_p, b_d, rtol=1e-6, atol=1e-8)
    assert steps < 20 and its > 0


# --------------------------------------------------------------------------- VIF-Laplace likelihood, SLQ
def _lap_problem(n=70, m=6, mv=3, seed=21):
    P = small_problem(n=n, m=m, mv=mv, nugget=0.0, likelihood="bernoulli_logit", ls=0.15, seed=seed)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv) if mv else np.zeros((n, 0), dtype=np.int64)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b, _, _ = O.laplace_mode(vif, P.y, dense=True)
    return P, vif, b


def test_vifdu_probe_recipe_has_covariance_P():
    """Sec. 4.3: the map (eps1, eps2, eps3) -> z is linear; Z Z^T must equal P^ exactly."""
    P, vif, b = _lap_problem()
    n, m = vif.n, vif.m
    _, W = O.bern_grad_W(P.y, b)
    cols = []
    for e in np.eye(m + 2 * n):
        cols.append(O.vifdu_sample(vif, W, e[:m], e[m:m + n], e[m + n:]))
    Zmap = np.column_stack(cols)
    Pd = O.VIFDU(vif, W).dense(W)
    np.testing.assert_allclose(Zmap @ Zmap.T, Pd, rtol=1e-9, atol=1e-9 * np.abs(Pd).max())


def test_vifdu_logdet_equals_dense_logdet():
    """App. E.1 (Sylvester): log det P^ = log det(W + D^-1) - log det M + log det M_3."""
    P, vif, b = _lap_problem(mv=4, seed=22)
    _, W = O.bern_grad_W(P.y, b)
    sgn, ld = np.linalg.slogdet(O.VIFDU(vif, W).dense(W))
    assert sgn > 0
    assert abs(O.vifdu_logdet(vif, W) - ld) <= 1e-9 * abs(ld)


def test_lanczos_from_pcg_coefficients_is_exact_gauss_quadrature():
    """App. D: once the Krylov space is exhausted, |P^{-1/2} z|^2 e_1^T log(T) e_1 with T from
    the PCG coefficients equals z^T P^{-1/2} log(P^{-1/2} A P^{-1/2}) P^{-1/2} z."""
    P, vif, b = _lap_problem(n=40, m=5, mv=3, seed=23)
    n = vif.n
    _, W = O.bern_grad_W(P.y, b)
    pre = O.VIFDU(vif, W)
    Amat = np.diag(W) + np.linalg.inv(vif.dense_Sigma_dagger())
    z = np.random.default_rng(7).standard_normal(n)
    _, it, rel, T, zpz = O.pcg_lanczos(lambda w: Amat @ w, pre.apply, z, 1e-14, 4 * n)
    lam, V = np.linalg.eigh(pre.dense(W))
    Ph = V @ np.diag(lam ** -0.5) @ V.T
    mu, U = np.linalg.eigh(Ph @ Amat @ Ph)
    exact = float((Ph @ z) @ (U @ (np.log(mu) * (U.T @ (Ph @ z)))))
    assert abs(zpz - float(z @ np.linalg.solve(pre.dense(W), z))) <= 1e-7 * zpz
    assert abs(zpz * O.lanczos_log_quadrature(T) - exact) <= 1e-7 * abs(exact), (it, rel)


def test_slq_without_neighbours_is_exact():
    """m_v = 0: B = I, so P^ = W + Sigma_dagger^{-1} is the system itself, every T_i = [1] and
    the estimate of Eq. slq_v1 is log det Sigma_dagger + log det P^ = log det(Sigma_dagger W + I)."""
    P, vif, b = _lap_problem(mv=0, seed=24)
    eps = np.random.default_rng(8).standard_normal((3, vif.m + 2 * vif.n))
    r = O.vifla_nll_slq(vif, P.y, b, eps, 1e-10)
    np.testing.assert_allclose(r["q"], 0.0, atol=1e-12)
    exact = O.vifla_logdet_dense(vif, b)
    assert abs(r["logdet"] - exact) <= 1e-10 * abs(exact)
    assert abs(r["nll"] - (-O.bern_loglik(P.y, b) + 0.5 * r["quad"] + 0.5 * exact)) <= 1e-10 * abs(r["nll"])


def test_slq_estimate_is_unbiased_within_its_standard_error():
    """Hutchinson over probes z ~ N(0, P^): the exactly normalised estimate averages to the dense
    log det(Sigma_dagger W + I); the paper's n/l normalisation (Eq. slq_v1) to within O(1/n)."""
    P, vif, b = _lap_problem(n=60, m=5, mv=4, seed=25)
    n, m = vif.n, vif.m
    eps = np.random.default_rng(9).standard_normal((300, m + 2 * n))
    r = O.vifla_nll_slq(vif, P.y, b, eps, 1e-12)
    exact = O.vifla_logdet_dense(vif, b)
    base = r["logdet_sigma"] + r["logdet_P"]
    terms = r["zPz"] * r["q"]
    se = terms.std(ddof=1) / math.sqrt(len(terms))
    assert abs(r["logdet_exact_norm"] - exact) <= 4.0 * se + 1e-9, (r["logdet_exact_norm"], exact, se)
    terms_n = n * r["q"]
    se_n = terms_n.std(ddof=1) / math.sqrt(len(terms_n))
    assert abs(base + terms_n.mean() - exact) <= 4.0 * se_n + 0.05 * abs(exact - base) + 1e-9


def test_fitc_preconditioner_solve_logdet_and_draws_match_its_dense_definition():
    """App. E.2: Woodbury solve = dense inverse, Sylvester log det = dense log det, and the draw
    map D_V^{1/2} eps2 + Sigma_kn^T Sigma_k^{-T/2} eps1 has covariance P^ exactly."""
    P, vif, b = _lap_problem(mv=4, seed=26)
    n, m = vif.n, vif.m
    _, W = O.bern_grad_W(P.y, b)
    pre = O.FITCPrecond(vif, W)
    Pd = pre.dense()
    w = np.random.default_rng(10).standard_normal(n)
    np.testing.assert_allclose(pre.apply(w), np.linalg.solve(Pd, w), rtol=1e-8, atol=1e-10)
    sgn, ld = np.linalg.slogdet(Pd)
    assert sgn > 0 and abs(pre.logdet() - ld) <= 1e-9 * abs(ld)
    Zmap = np.column_stack([pre.sample(e[:m], e[m:]) for e in np.eye(m + n)])
    np.testing.assert_allclose(Zmap @ Zmap.T, Pd, rtol=1e-9, atol=1e-9 * np.abs(Pd).max())
    # P^ = W^{-1} + the FITC covariance (Sigma_mn^T Sigma_m^{-1} Sigma_mn + diagonal residual)
    np.testing.assert_allclose(Pd, O.fitc_cov(P.X, P.Z, P.theta) + np.diag(1.0 / W), rtol=1e-8, atol=1e-10)


def test_pcls2_newton_with_fitc_reaches_the_dense_mode():
    """Eq. pcls2: solving (W^{-1} + Sigma_dagger)(W u) = Sigma_dagger v gives the Newton step of
    Eq. one_it_newton_mode; the mode equals the dense-Newton mode."""
    P, vif, b = _lap_problem(n=150, m=10, mv=5, seed=27)
    b_f, steps, its = O.laplace_mode_fitc(vif, P.y, tol=1e-11)
    np.testing.assert_allclose(b_f, b, rtol=1e-7, atol=1e-9)
    assert its > 0 and steps < 20


def test_slq_fitc_is_nearly_exact_when_the_vif_is_fitc_itself():
    """m_v = 0: Sigma_dagger = Sigma_mn^T Sigma_m^{-1} Sigma_mn + diag(residual + R7 jitter), so
    the FITC preconditioner equals W^{-1} + Sigma_dagger up to the 1e-10 sigma_1^2 jitter: every
    quadrature is ~0 and the estimate of Eq. slq_v2 is the dense log det."""
    P, vif, b = _lap_problem(mv=0, seed=28)
    eps = np.random.default_rng(11).standard_normal((3, vif.m + vif.n))
    r = O.vifla_nll_slq_fitc(vif, P.y, b, eps, 1e-10)
    assert np.abs(r["q"]).max() <= 1e-8
    exact = O.vifla_logdet_dense(vif, b)
    assert abs(r["logdet"] - exact) <= 1e-8 * abs(exact) + 1e-6


def test_slq_fitc_estimate_is_unbiased_within_its_standard_error():
    P, vif, b = _lap_problem(n=60, m=5, mv=4, seed=29)
    n, m = vif.n, vif.m
    eps = np.random.default_rng(12).standard_normal((300, m + n))
    r = O.vifla_nll_slq_fitc(vif, P.y, b, eps, 1e-12)
    exact = O.vifla_logdet_dense(vif, b)
    terms = r["zPz"] * r["q"]
    se = terms.std(ddof=1) / math.sqrt(len(terms))
    assert abs(r["logdet_exact_norm"] - exact) <= 4.0 * se + 1e-9, (r["logdet_exact_norm"], exact, se)
    # the two SLQ forms agree on the same log-determinant
    r1 = O.vifla_nll_slq(vif, P.y, b, np.random.default_rng(13).standard_normal((300, m + 2 * n)), 1e-12)
    t1 = r1["zPz"] * r1["q"]
    se1 = t1.std(ddof=1) / math.sqrt(len(t1))
    assert abs(r["logdet_exact_norm"] - r1["logdet_exact_norm"]) <= 4.0 * math.hypot(se, se1) + 1e-9


# --------------------------------------------------------------------------- VIF-Laplace prediction
def _gp_laplace_textbook(K, Kp, kpp, y, f):
    """Latent predictive mean and variance of the Laplace-approximated GP classifier at the mode f
    (Rasmussen & Williams, Sec. 3.4, Alg. 3.2): mean = Kp (y - sigmoid(f)), var = kpp - |v|^2 with
    v = L^{-1} W^{1/2} Kp^T, L = chol(I + W^{1/2} K W^{1/2})."""
    p = 1.0 / (1.0 + np.exp(-f))
    W = p * (1.0 - p)
    sw = np.sqrt(W)
    L = np.linalg.cholesky(np.eye(len(f)) + sw[:, None] * K * sw[None, :])
    v = sla.solve_triangular(L, sw[:, None] * Kp.T, lower=True)
    return Kp @ (y - p), kpp - (v * v).sum(0)


def test_laplace_prediction_with_full_conditioning_is_the_textbook_gp_laplace():
    """m_v = n-1 and every training point a prediction neighbour: the VIF prior is the exact GP
    (up to the 1e-10 jitter), so Prop. 3.1 must give the textbook Laplace predictive distribution."""
    P = small_problem(n=70, m=6, mv=69, nugget=0.0, likelihood="bernoulli_logit", ls=0.2, seed=30, n_pred=15)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 69)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b, _, _ = O.laplace_mode(vif, P.y, dense=True)
    Np = np.tile(np.arange(70), (15, 1))
    mu, Om = O.laplace_predict_dense(vif, P.y, b, P.Xp, Np)
    K = O.cov(P.X, P.X, P.theta)
    mu_t, var_t = _gp_laplace_textbook(K, O.cov(P.Xp, P.X, P.theta), np.full(15, P.theta.variance), P.y, b)
    np.testing.assert_allclose(mu, mu_t, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(np.diag(Om), var_t, rtol=1e-5, atol=1e-7)


def test_sbpv_is_unbiased_for_the_laplace_predictive_variances():
    """Alg. 1: the deterministic part equals the first part of Omega_p (App. C.1 = Prop. 2.1 with b for
    y) and the sample average of z8 o z8 converges to the Laplace part (Prop. 4 of the paper)."""
    P = small_problem(n=90, m=6, mv=5, nugget=0.0, likelihood="bernoulli_logit", ls=0.15, seed=31, n_pred=12)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 5)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b, _, _ = O.laplace_mode(vif, P.y, dense=True)
    Np = O.pred_neighbors(P.X, P.Z, P.theta, P.Xp, 5)
    mu_d, Om = O.laplace_predict_dense(vif, P.y, b, P.Xp, Np)
    eps = np.random.default_rng(14).standard_normal((1000, vif.m + 2 * vif.n))
    mu, var, its = O.laplace_predict_sbpv(vif, P.y, b, P.Xp, Np, eps, 1e-12)
    np.testing.assert_allclose(mu, mu_d, rtol=1e-8, atol=1e-10)
    _, var_det = O.predict_appC(vif, b, P.Xp, Np)
    part = np.diag(Om) - var_det
    assert (part > 0).all()
    # each z8_p^2 has mean part_p and variance 2 part_p^2 (z8_p is Gaussian), so the average of
    # 1000 has standard error part_p sqrt(2/1000)
    assert np.all(np.abs(var - np.diag(Om)) <= 4.0 * part * math.sqrt(2.0 / len(eps)))


# --------------------------------------------------------------------------- gradient
def _lap_grad_problem(n=70, m=6, mv=3, seed=21):
    P = small_problem(n=n, m=m, mv=mv, nugget=0.0, likelihood="bernoulli_logit", ls=0.15, seed=seed)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b, _, _ = O.laplace_mode(vif, P.y, dense=True, psi_tol=1e-14)
    return P, N, vif, b


def test_vifla_gradient_with_exact_traces_is_the_derivative_of_the_exact_likelihood():
    """App. B: explicit terms, log det derivative and the implicit term -v^T Delta_k b through the
    mode; with every trace exact the assembled gradient must equal central differences of L^VIFLA
    itself (dense Newton mode re-found at each perturbed theta, dense log-determinant)."""
    P, N, vif, b = _lap_grad_problem()
    ex = O.vifla_grad_exact(P.X, P.Z, P.theta, N, P.y, b)
    v0 = O.laplace_param_vector(P.theta)
    fd = np.empty(v0.size)
    for k in range(v0.size):
        h = 1e-4 * abs(v0[k])
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        fd[k] = (O.vifla_nll_exact(P.X, P.Z, O.laplace_theta_from_vector(P.theta, vp), N, P.y)
                 - O.vifla_nll_exact(P.X, P.Z, O.laplace_theta_from_vector(P.theta, vm), N, P.y)) / (2 * h)
    np.testing.assert_allclose(ex["grad"], fd, rtol=2e-5, atol=1e-6)


def test_ste_sums_are_exact_when_the_probes_span_the_preconditioner():
    """With eps running over the identity of R^(m+2n) the probes satisfy sum_i z_i z_i^T = P^
    exactly (Sec. 4.3 recipe), so l times each STE average of Sec. 4.1 / App. D is the exact
    trace: Tr(H^{-1} Delta_k), Tr(P^{-1} dP^/dth_k) and the diagonal (H^{-1})_jj behind dL/db.
    The recipe reproduces P^ to about 1e-7 relative (Sigma_dagger^{-1} Sigma_dagger Sigma_dagger^{-1}
    of a latent GP amplifies rounding by the conditioning of Sigma_dagger), and cond(P^) ~ 300 here,
    hence rtol 3e-4; a wrong normalisation or a dropped term is off by 7e-3 or more."""
    P, N, vif, b = _lap_grad_problem(n=40, m=5, mv=3, seed=23)
    n, m = vif.n, vif.m
    eps = np.eye(m + 2 * n)
    ell = eps.shape[0]
    r = O.vifla_grad_ste(P.X, P.Z, P.theta, N, P.y, b, eps, 1e-13, 1e-13)
    ex = O.vifla_grad_exact(P.X, P.Z, P.theta, N, P.y, b)
    np.testing.assert_allclose(ell * r["trace_plain"], ex["trace"], rtol=3e-4)
    np.testing.assert_allclose(ell * r["c"].mean(axis=0), r["tau"], rtol=3e-4)
    np.testing.assert_allclose(ell * r["g"], ex["g"], rtol=3e-4, atol=1e-9)


def test_ste_gradient_is_unbiased_and_the_control_variate_reduces_its_variance():
    """Random probes z ~ N(0, P^): the plain STE of Tr(H^{-1} Delta_k) averages to the exact trace
    and the control-variate samples c_ik to Tr(P^{-1} dP^/dth_k), within four standard errors;
    the control-variate estimate of App. D stays unbiased with a smaller spread."""
    P, N, vif, b = _lap_grad_problem()
    n, m = vif.n, vif.m
    ell = 200
    eps = np.random.default_rng(9).standard_normal((ell, m + 2 * n))
    r = O.vifla_grad_ste(P.X, P.Z, P.theta, N, P.y, b, eps, 1e-12, 1e-12)
    ex = O.vifla_grad_exact(P.X, P.Z, P.theta, N, P.y, b)
    se = r["s"].std(axis=0, ddof=1) / math.sqrt(ell)
    se_c = r["c"].std(axis=0, ddof=1) / math.sqrt(ell)
    se_cv = (r["s"] - r["c_opt"] * r["c"]).std(axis=0, ddof=1) / math.sqrt(ell)
    assert np.all(np.abs(r["trace_plain"] - ex["trace"]) <= 4 * se), (r["trace_plain"], ex["trace"], se)
    assert np.all(np.abs(r["c"].mean(axis=0) - r["tau"]) <= 4 * se_c), (r["c"].mean(axis=0), r["tau"], se_c)
    assert np.all(np.abs(r["trace"] - ex["trace"]) <= 4 * se_cv), (r["trace"], ex["trace"], se_cv)
    assert np.all(se_cv < 0.5 * se), (se_cv, se)


def _gp_laplace_gradient_textbook(X, y, theta):
    """Gradient of -log q(y | X, theta) of the exact-GP Laplace approximation for Bernoulli-logit
    responses in the K form of Rasmussen & Williams (2006): the mode by the Newton step of Alg. 3.1,
    the gradient with the structure of Alg. 5.1, i.e. the explicit part 1/2 a^T C a -
    1/2 tr((W^{-1} + K)^{-1} C) (a = grad log p at the mode, C = dK/dth) plus s2^T df/dth with
    df/dth = (I + K W)^{-1} C grad log p and s2_i = dlog q/df_i = -1/2 dlog|I + K W|/df_i
    = 1/2 [(K^{-1} + W)^{-1}]_ii d^3 log p/df_i^3 (dW/df = -d^3 log p/df^3)."""
    n = len(y)
    K = O.exact_cov(X, theta)
    f = np.zeros(n)
    for _ in range(100):
        p = 1.0 / (1.0 + np.exp(-f))
        W = p * (1 - p)
        g = y - p
        f_new = K @ np.linalg.solve(np.eye(n) + W[:, None] * K, W * f + g)
        if np.max(np.abs(f_new - f)) < 1e-13:
            f = f_new
            break
        f = f_new
    p = 1.0 / (1.0 + np.exp(-f))
    W = p * (1 - p)
    g = y - p
    d3 = -W * (1 - 2 * p)                                      # third derivative of log p
    R = np.linalg.inv(np.diag(1.0 / W) + K)                     # (W^{-1} + K)^{-1}
    Sig = np.linalg.inv(np.linalg.inv(K) + np.diag(W))          # (K^{-1} + W)^{-1}
    s2 = 0.5 * np.diag(Sig) * d3
    Xs = O.scaled(X, theta)
    r = O.dist(Xs, Xs)
    dK = O.dcov_of_r(r, theta.kind, theta.variance)
    lam = float(np.atleast_1d(theta.lengthscale)[0])
    mats = [O.cov_of_r(r, theta.kind, theta.variance) / theta.variance, -dK * r / lam]
    grad = []
    for C in mats:
        s1 = 0.5 * g @ C @ g - 0.5 * np.sum(R * C)
        b = C @ g
        s3 = b - K @ (R @ b)
        grad.append(-(s1 + s2 @ s3))
    return np.array(grad)


def test_vifla_gradient_with_full_conditioning_is_the_textbook_gp_laplace_gradient():
    """With m_v = n - 1 the VIF is the exact GP (Sigma_dagger = Sigma), so the App. B gradient with exact
    traces must be the textbook GP-Laplace gradient (Rasmussen & Williams Alg. 5.1, a different
    derivation: K form, its own Newton mode)."""
    n = 40
    P = small_problem(n=n, m=5, mv=n - 1, nugget=0.0, likelihood="bernoulli_logit", ls=0.2, seed=27)
    N = O.causal_neighbors(P.X, P.Z, P.theta, n - 1)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    b, _, _ = O.laplace_mode(vif, P.y, dense=True, psi_tol=1e-14)
    ex = O.vifla_grad_exact(P.X, P.Z, P.theta, N, P.y, b)
    tb = _gp_laplace_gradient_textbook(P.X, P.y, P.theta)
    np.testing.assert_allclose(ex["grad"], tb, rtol=1e-5, atol=1e-7)


def test_fitc_form_gradient_with_exact_traces_equals_the_vifdu_form():
    """App. B / App. D second form: through Sigma_dagger and H_F = W^{-1} + Sigma_dagger (Eq. pcls2) the
    assembled gradient is the same derivative of L^VIFLA as through Sigma_dagger^{-1} (pinned above to
    finite differences of the likelihood)."""
    P, N, vif, b = _lap_grad_problem()
    ex = O.vifla_grad_exact(P.X, P.Z, P.theta, N, P.y, b)
    exf = O.vifla_grad_exact_fitc(P.X, P.Z, P.theta, N, P.y, b)
    np.testing.assert_allclose(exf["grad"], ex["grad"], rtol=2e-5, atol=1e-6)


def test_fitc_ste_sums_are_exact_when_the_probes_span_the_preconditioner():
    """FITC probes z = D_V^{1/2} eps2 + Sigma_mn^T L_m^{-T} eps1 with eps over the identity of R^(m+n):
    sum z z^T = P exactly, so l times each STE average is the exact trace Tr(H_F^{-1} dSigma_k),
    Tr(P^{-1} dP/dth_k) and diagonal (H_F^{-1})_jj."""
    P, N, vif, b = _lap_grad_problem(n=40, m=5, mv=3, seed=23)
    n, m = vif.n, vif.m
    eps = np.eye(m + n)
    ell = eps.shape[0]
    r = O.vifla_grad_ste_fitc(P.X, P.Z, P.theta, N, P.y, b, eps, 1e-13, 1e-13)
    exf = O.vifla_grad_exact_fitc(P.X, P.Z, P.theta, N, P.y, b)
    np.testing.assert_allclose(ell * r["trace_plain"], exf["trace"], rtol=1e-8)
    np.testing.assert_allclose(ell * r["c"].mean(axis=0), r["tau"], rtol=1e-8)
    np.testing.assert_allclose(ell * r["dhat"], exf["dHF"], rtol=1e-9)


def test_fitc_ste_gradient_is_unbiased_and_the_control_variate_reduces_its_variance():
    P, N, vif, b = _lap_grad_problem()
    n, m = vif.n, vif.m
    ell = 200
    eps = np.random.default_rng(9).standard_normal((ell, m + 2 * n))
    r = O.vifla_grad_ste_fitc(P.X, P.Z, P.theta, N, P.y, b, eps, 1e-12, 1e-12)
    exf = O.vifla_grad_exact_fitc(P.X, P.Z, P.theta, N, P.y, b)
    se = r["s"].std(axis=0, ddof=1) / math.sqrt(ell)
    se_c = r["c"].std(axis=0, ddof=1) / math.sqrt(ell)
    se_cv = (r["s"] - r["c_opt"] * r["c"]).std(axis=0, ddof=1) / math.sqrt(ell)
    assert np.all(np.abs(r["trace_plain"] - exf["trace"]) <= 4 * se), (r["trace_plain"], exf["trace"], se)
    assert np.all(np.abs(r["c"].mean(axis=0) - r["tau"]) <= 4 * se_c)
    assert np.all(np.abs(r["trace"] - exf["trace"]) <= 4 * se_cv), (r["trace"], exf["trace"], se_cv)
    assert np.all(se_cv < 0.75 * se), (se_cv, se)


def test_fd_gradient_with_full_conditioning_is_the_exact_gp_gradient():
    """m_v = n-1 makes the VIF likelihood the exact one, whose gradient is analytic."""
    P = small_problem(n=60, m=8, mv=59, nugget=0.1, kind="matern32", ls=0.2)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 59)
    g_fd = O.vif_nll_grad_fd(P.X, P.Z, P.theta, N, P.y)
    g_ex = O.exact_gp_grad(P.X, P.y, P.theta)
    np.testing.assert_allclose(g_fd, g_ex, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("m,mv,kind,ls,step,tol", [
    (20, 8, "matern32", 0.2, 1e-4, 1e-6),
    (0, 5, "matern52", 0.3, 1e-4, 1e-6),
    (12, 0, "matern12", 0.2, 1e-4, 1e-6),
    (15, 6, "se", np.array([0.3, 0.6]), 3e-4, 2e-6)])
def test_analytic_gradient_matches_central_differences_of_the_likelihood(m, mv, kind, ls, step, tol):
    """The Sec. 2.2 / App. A gradient against central differences of the oracle's own NLL
    (a different route: no derivative algebra).  The SE case is ill-conditioned (Sigma_m
    jitter 1e-8), so its differences take a larger step to stay above rounding."""
    P = small_problem(n=220, d=2, m=m, mv=mv, kind=kind, ls=ls, nugget=0.1, seed=3)
    N = O.causal_neighbors(P.X, P.Z, P.theta, mv) if mv else -np.ones((220, 0), dtype=np.int64)
    g = O.vif_nll_grad(P.X, P.Z, P.theta, N, P.y)
    g_fd = O.vif_nll_grad_fd(P.X, P.Z, P.theta, N, P.y, rel_step=step)
    np.testing.assert_allclose(g, g_fd, rtol=0, atol=tol * np.abs(g_fd).max())


def test_analytic_gradient_with_full_conditioning_is_the_exact_gp_gradient():
    P = small_problem(n=60, m=8, mv=59, nugget=0.1, kind="matern32", ls=0.2)
    N = O.causal_neighbors(P.X, P.Z, P.theta, 59)
    np.testing.assert_allclose(O.vif_nll_grad(P.X, P.Z, P.theta, N, P.y),
                               O.exact_gp_grad(P.X, P.y, P.theta), rtol=1e-9, atol=1e-10)


def test_analytic_gradient_of_the_independent_model_is_closed_form():
    """m = 0 and m_v = 0: Sigma~_dagger = (sigma1^2 + sigma^2) I, so the NLL is
    n/2 log(2 pi s) + |y|^2 / (2 s) with s = sigma1^2 + sigma^2, and the length scale has no
    effect."""
    P = small_problem(n=50, m=0, mv=0, nugget=0.3, kind="matern32", ls=0.2)
    N = -np.ones((50, 0), dtype=np.int64)
    s2 = P.theta.variance + P.theta.nugget
    ds = 0.5 * 50 / s2 - 0.5 * (P.y @ P.y) / s2 ** 2
    np.testing.assert_allclose(O.vif_nll_grad(P.X, P.Z, P.theta, N, P.y), [ds, 0.0, ds], rtol=1e-12, atol=1e-12)


def test_exact_gp_gradient_ard_matches_its_own_finite_differences():
    P = small_problem(n=40, m=0, mv=0, nugget=0.05, kind="se", ls=np.array([0.2, 0.4]))
    g = O.exact_gp_grad(P.X, P.y, P.theta)
    v0 = O.theta_vector(P.theta)
    for k in range(v0.size):
        h = 1e-5 * v0[k]
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        fp = O.dense_nll(O.exact_cov(P.X, O.theta_from_vector(P.theta, vp)), P.y)
        fm = O.dense_nll(O.exact_cov(P.X, O.theta_from_vector(P.theta, vm)), P.y)
        assert (fp - fm) / (2 * h) == pytest.approx(g[k], rel=1e-5, abs=1e-6)


# --------------------------------------------------------------------------- learned correction (oracle side)
from oracle import mlp_oracle as M


def test_mlp_forward_closed_form_special_case():
    p = np.zeros(M.NPARAM)
    W1, b1, W2, b2, w3, b3 = M.unpack(p)      # views into p
    W1[0, 0] = 1.0
    W2[...] = np.eye(M.NH)
    w3[0] = 2.0
    F = np.array([[0.3] + [5.0] * (M.NIN - 1), [-1.2] + [0.0] * (M.NIN - 1)])
    o = 2.0 * np.tanh(np.tanh(F[:, 0]))
    np.testing.assert_allclose(M.forward(p, F), 4.0 * np.tanh(o / 4.0), rtol=1e-14)
    assert np.all(M.forward(M.init_params(3), F) == 0.0)     # zero output layer: plain VIFDU


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 0.3, M.NPARAM)
    F = rng.normal(0, 1, (7, M.NIN))
    gc = rng.normal(0, 1, 7)
    g = M.backward(p, F, gc)
    for k in rng.choice(M.NPARAM, 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (gc @ M.forward(pp, F) - gc @ M.forward(pm, F)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-9)


def test_preconditioner_loss_gradient_formula_matches_dense_finite_differences():
    """dL/dd_j = -2 (B P^-1 r)_j (B u)_j for L = ||P(d)^-1 A z - z||^2, P(d) = B^T diag(d) B + Sigma_dagger^-1."""
    P = small_problem(n=70, m=8, mv=4, nugget=0.0, likelihood="bernoulli_logit")
    N = O.causal_neighbors(P.X, P.Z, P.theta, 4)
    vif = O.VIF(P.X, P.Z, P.theta, N)
    rng = np.random.default_rng(7)
    W = rng.uniform(0.05, 0.25, 70)
    d = W * np.exp(rng.normal(0, 0.5, 70))
    Sdi = np.column_stack([vif.Sigma_dagger_inv(e) for e in np.eye(70)])
    A = np.diag(W) + Sdi
    B = vif.B.toarray()
    z = rng.choice([-1.0, 1.0], 70)

    def loss(dd):
        Pm = B.T @ np.diag(dd) @ B + Sdi
        r = np.linalg.solve(Pm, A @ z) - z
        return r @ r
    Pm = B.T @ np.diag(d) @ B + Sdi
    u = np.linalg.solve(Pm, A @ z)
    r = u - z
    g = -2.0 * (B @ np.linalg.solve(Pm, r)) * (B @ u)
    for j in (0, 5, 33, 69):
        h = 1e-4 * d[j]
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        assert (loss(dp) - loss(dm)) / (2 * h) == pytest.approx(g[j], rel=1e-5, abs=1e-9)


def test_features_hand_example():
    # three points: 1 conditions on 0 (A=0.5), 2 conditions on 0 and 1 (A = 0.2, -0.4)
    W = np.array([0.2, 0.1, 0.25])
    D = np.array([1.0, 0.5, 0.25])
    Ac = np.array([[0.0, 0.0], [0.5, 0.0], [0.2, -0.4]])
    N = np.array([[-1, -1], [0, -1], [0, 1]])
    F = M.features(W, D, Ac, N, 2)
    assert F[0, 5] == pytest.approx(0.25 + 0.04)                  # A_1[0]^2 + A_2[0]^2
    assert F[1, 5] == pytest.approx(0.16)
    assert F[2, 4] == pytest.approx(0.04 + 0.16)
    assert F[2, 6] == pytest.approx(np.log(0.15 / 0.25))            # mean W over {0, 1} / W_2
    assert F[0, 7] == pytest.approx(np.log1p((0.1 * 0.25 + 0.25 * 0.04) / 0.2))
    assert F[1, 3] == pytest.approx(0.5) and F[0, 3] == 0.0
