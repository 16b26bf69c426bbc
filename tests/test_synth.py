"""The seeded input generators shared by the oracle and the CUDA path (synth.py hold none of the
method's arithmetic): determinism, shapes and ranges of the recipe, and the random-Fourier-feature
latent field having the stated covariance (its spectral densities: Gaussian for SE, Student-t with
2 nu degrees of freedom for Matern-nu)."""
import math

import numpy as np
import pytest

from oracle import vif_oracle as O
from paper_2507_05064_gb300 import synth


def test_make_problem_is_deterministic_and_within_the_recipe():
    a = synth.make_problem(3000, 3, 40, 8, "matern52", 1.0, 0.2, 0.05, 123)
    b = synth.make_problem(3000, 3, 40, 8, "matern52", 1.0, 0.2, 0.05, 123)
    for x, y in ((a.X, b.X), (a.y, b.y), (a.Z, b.Z)):
        np.testing.assert_array_equal(x, y)
    c = synth.make_problem(3000, 3, 40, 8, "matern52", 1.0, 0.2, 0.05, 124)
    assert not np.array_equal(a.X, c.X)
    assert a.X.shape == (3000, 3) and a.Z.shape == (40, 3) and a.y.shape == (3000,)
    assert a.X.min() >= 0.0 and a.X.max() <= 1.0
    assert a.Z.min() >= 0.0 and a.Z.max() <= 1.0          # k-means++ centres lie in the hull of X


def test_bernoulli_responses_and_subset_inducing_points():
    P = synth.make_problem(2000, 2, 30, 5, "matern32", 1.0, 0.1, 0.0, 7, likelihood="bernoulli_logit",
                           inducing="subset")
    assert set(np.unique(P.y)) <= {0.0, 1.0}
    assert 0.2 < P.y.mean() < 0.8
    rows = {tuple(r) for r in P.X}
    assert all(tuple(z) in rows for z in P.Z)
    assert P.theta.nugget == 0.0


@pytest.mark.parametrize("kind", ["matern12", "matern32", "matern52", "se"])
def test_random_fourier_field_has_the_stated_covariance(kind):
    """E[f(x) f(x')] = sigma1^2 E cos(w.(x - x')) = k(x, x') when w follows the kernel's spectral
    density; averaged over independent draws at three separations (four standard errors)."""
    theta = synth.Theta(synth.KIND_IDS[kind], 1.7, np.array([0.3]), 0.0)
    X = np.array([[0.0, 0.0], [0.1, 0.05], [0.3, 0.2], [0.0, 0.0]])
    rng = np.random.Generator(np.random.PCG64(5))
    draws = np.array([synth.latent_rff(X, theta, rng, R=256) for _ in range(3000)])
    K = O.cov(X[:3], X[:3], theta)
    for j in range(3):
        prod = draws[:, 0] * draws[:, j]
        se = prod.std(ddof=1) / math.sqrt(len(prod))
        assert abs(prod.mean() - K[0, j]) <= 4 * se + 1e-3, (kind, j, prod.mean(), K[0, j], se)


def test_config_recipes():
    ls = synth.config3_lengthscales()
    assert ls.shape == (8,) and ls.min() >= 0.2 and ls.max() <= 2.0
    np.testing.assert_array_equal(ls, synth.config3_lengthscales())
    P1 = synth.config1(n=400, n_pred=50)
    assert P1.X.shape == (400, 2) and P1.Z.shape == (50, 2) and P1.mv == 10 and P1.Xp.shape == (50, 2)
    assert P1.theta.nugget == pytest.approx(0.1) and P1.theta.kind == synth.KIND_IDS["matern32"]
    P4 = synth.config4(n=3000, lloyd=1)
    assert P4.likelihood == "bernoulli_logit" and P4.Z.shape == (200, 2) and P4.mv == 20
    probs = synth.config5(nprob=6, n_lo=2000, n_hi=3000)
    for P in probs:
        d = P.X.shape[1]
        assert 2000 <= P.X.shape[0] <= 3000 and d in (2, 5)
        assert 64 <= P.Z.shape[0] <= 256 and 10 <= P.mv <= 40
        assert 0.02 <= float(P.theta.lengthscale[0]) <= 0.3 and 0.01 <= P.theta.nugget <= 0.1


def test_slq_normals():
    e = synth.slq_normals(7, 5, 300, seed=3)
    assert e.shape == (7, 5 + 600)
    np.testing.assert_array_equal(e, synth.slq_normals(7, 5, 300, seed=3))
    assert abs(e.mean()) < 0.05 and abs(e.std() - 1.0) < 0.05
