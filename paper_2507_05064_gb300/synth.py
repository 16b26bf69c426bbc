"""Seeded synthetic inputs shaped like the paper's simulated experiments (Sec. 7).

This module holds no arithmetic of the VIF method itself: it only draws inputs
(locations, responses, inducing points, hyperparameters).  Both the CUDA path
and the CPU oracle take their inputs from here.

* Locations are i.i.d. uniform on the unit hypercube [0,1]^d (Sec. 7).
* The latent GP is drawn with random Fourier features (Rahimi & Recht, 2007):
  f(s) = sqrt(2 sigma1^2 / R) * sum_r cos(w_r . s/lambda + b_r), with w_r from
  the kernel's spectral density (standard normal for the squared-exponential
  kernel, multivariate Student-t with 2 nu degrees of freedom for Matern-nu).
  The likelihood cost does not depend on y, and parity feeds the same y to
  both sides, so an approximate draw is enough.
* Gaussian responses add N(0, sigma^2) noise; Bernoulli responses draw
  y ~ Bernoulli(sigmoid(f)) (Sec. 3, logit link).
* Inducing points come from k-means++ seeding plus Lloyd steps in the
  ARD-scaled space s/lambda (Sec. 6), or from a random subset of the inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KIND_IDS = {"matern12": 0, "matern32": 1, "matern52": 2, "se": 3}
NU = {0: 0.5, 1: 1.5, 2: 2.5, 3: math.inf}


@dataclasses.dataclass
class Theta:
    """Covariance hyperparameters: kernel kind, marginal variance sigma1^2,
    length scale(s) lambda (one value, or one per input dimension), and the
    nugget sigma^2 (0 for latent-GP / Laplace problems)."""

    kind: int
    variance: float
    lengthscale: np.ndarray
    nugget: float

    def copy(self) -> "Theta":
        return Theta(self.kind, float(self.variance), np.array(self.lengthscale, dtype=np.float64),
                     float(self.nugget))


@dataclasses.dataclass
class Problem:
    X: np.ndarray          # n x d, float64
    y: np.ndarray          # n, float64
    Z: np.ndarray          # m x d, float64
    theta: Theta
    mv: int
    likelihood: str        # "gaussian" or "bernoulli_logit"
    Xp: np.ndarray | None = None   # prediction inputs (n_p x d)
    name: str = ""


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def latent_rff(X: np.ndarray, theta: Theta, rng: np.random.Generator, R: int = 2048,
               chunk: int = 65536) -> np.ndarray:
    """Approximate zero-mean GP draw at X with random Fourier features."""
    n, d = X.shape
    ls = np.broadcast_to(np.asarray(theta.lengthscale, dtype=np.float64), (d,))
    g = rng.standard_normal((R, d))
    nu = NU[theta.kind]
    if math.isinf(nu):
        W = g
    else:
        u = rng.chisquare(2.0 * nu, size=R)
        W = g * np.sqrt(2.0 * nu / u)[:, None]
    b = rng.uniform(0.0, 2.0 * math.pi, size=R)
    amp = math.sqrt(2.0 * theta.variance / R)
    f = np.empty(n)
    Wt = (W / ls[None, :]).T
    for s in range(0, n, chunk):
        f[s:s + chunk] = amp * np.cos(X[s:s + chunk] @ Wt + b).sum(axis=1)
    return f


def kmeanspp(Xs: np.ndarray, m: int, rng: np.random.Generator, lloyd: int = 10) -> np.ndarray:
    """k-means++ seeding (Arthur & Vassilvitskii, 2007) plus `lloyd` Lloyd steps.
    Works on whatever coordinates it is given (the caller passes s/lambda)."""
    n, d = Xs.shape
    C = np.empty((m, d))
    C[0] = Xs[rng.integers(n)]
    d2 = ((Xs - C[0]) ** 2).sum(1)
    for k in range(1, m):
        tot = d2.sum()
        if tot <= 0:
            C[k] = Xs[rng.integers(n)]
        else:
            i = int(np.searchsorted(np.cumsum(d2), rng.uniform(0.0, tot)))
            C[k] = Xs[min(i, n - 1)]
        d2 = np.minimum(d2, ((Xs - C[k]) ** 2).sum(1))
    xx = (Xs ** 2).sum(1)
    for _ in range(lloyd):
        lab = np.empty(n, dtype=np.int64)
        cc = (C ** 2).sum(1)
        for s in range(0, n, 65536):
            dd = cc[None, :] - 2.0 * Xs[s:s + 65536] @ C.T
            lab[s:s + 65536] = dd.argmin(1)
        cnt = np.bincount(lab, minlength=m)
        for j in range(d):
            sj = np.bincount(lab, weights=Xs[:, j], minlength=m)
            C[cnt > 0, j] = sj[cnt > 0] / cnt[cnt > 0]
    del xx
    return C


def make_problem(n: int, d: int, m: int, mv: int, kind: str, variance: float,
                 lengthscale, nugget: float, seed: int, likelihood: str = "gaussian",
                 inducing: str = "kmeans++", n_pred: int = 0, lloyd: int = 10,
                 name: str = "", rff: int | None = None) -> Problem:
    rng = _rng(seed)
    X = rng.uniform(size=(n, d))
    ls = np.atleast_1d(np.asarray(lengthscale, dtype=np.float64))
    theta = Theta(KIND_IDS[kind], float(variance), ls, float(nugget))
    f = latent_rff(X, theta, rng, R=rff or (2048 if n <= 100_000 else 512))
    if likelihood == "gaussian":
        y = f + math.sqrt(nugget) * rng.standard_normal(n)
    else:
        p = 1.0 / (1.0 + np.exp(-f))
        y = (rng.uniform(size=n) < p).astype(np.float64)
    if m == 0:
        Z = np.zeros((0, d))
    elif inducing == "subset":
        Z = X[np.sort(rng.choice(n, size=m, replace=False))].copy()
    else:
        lsd = np.broadcast_to(ls, (d,))
        Z = kmeanspp(X / lsd, m, rng, lloyd=lloyd) * lsd
    Xp = rng.uniform(size=(n_pred, d)) if n_pred > 0 else None
    return Problem(X, y, Z, theta, mv, likelihood, Xp, name)


# The five workloads, with the sizes stated for them.  Seeds: 20250707 + id.
def config1(n=2000, n_pred=500) -> Problem:
    """n=2000 on [0,1]^2, Matern-3/2 (variance 1, range 0.1) plus N(0,0.1) noise,
    m=50 inducing points as a random subset of the inputs, m_v=10."""
    return make_problem(n, 2, 50, 10, "matern32", 1.0, 0.1, 0.1, 20250708,
                        inducing="subset", n_pred=n_pred, name="matern32-n2000-d2-m50-mv10")


def config2(n=100_000, lloyd=10) -> Problem:
    """n=1e5 on [0,1]^2, Matern-5/2 (variance 1, range 0.05, nugget 0.05),
    m=200 by k-means++, m_v=30."""
    return make_problem(n, 2, 200, 30, "matern52", 1.0, 0.05, 0.05, 20250709, lloyd=lloyd,
                        name=f"matern52-n{n}-d2-m200-mv30")


def config3_lengthscales() -> np.ndarray:
    rng = _rng(20250710 + 1000)
    return np.exp(rng.uniform(math.log(0.2), math.log(2.0), size=8))


def config3(n=500_000, m=500, mv=20, lloyd=3) -> Problem:
    """n=5e5 on [0,1]^8, ARD squared-exponential with length scales log-uniform
    in [0.2, 2], variance 1, nugget 0.01; m=500, m_v=20."""
    return make_problem(n, 8, m, mv, "se", 1.0, config3_lengthscales(), 0.01, 20250710,
                        lloyd=lloyd, name=f"se-ard-n{n}-d8-m{m}-mv{mv}")


def config4(n=200_000, lloyd=5) -> Problem:
    """Bernoulli-logit, n=2e5 on [0,1]^2, Matern-3/2 (variance 1, range 0.05),
    m=200, m_v=20."""
    return make_problem(n, 2, 200, 20, "matern32", 1.0, 0.05, 0.0, 20250711,
                        likelihood="bernoulli_logit", lloyd=lloyd,
                        name=f"bernoulli-matern32-n{n}-d2-m200-mv20")


def config5(nprob=256, n_lo=2_000, n_hi=50_000, seed=20250712, lloyd=2):
    """256 independent Gaussian problems: n log-uniform in [2e3, 5e4], d in {2, 5},
    m uniform in [64, 256], m_v uniform in [10, 40], Matern-3/2 or 5/2 with range
    uniform in [0.02, 0.3], nugget uniform in [0.01, 0.1], k-means++ inducing points."""
    rng = _rng(seed)
    out = []
    for k in range(nprob):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice([2, 5]))
        m = int(rng.integers(64, 257))
        mv = int(rng.integers(10, 41))
        kind = "matern32" if rng.uniform() < 0.5 else "matern52"
        rng_range = float(rng.uniform(0.02, 0.3))
        nug = float(rng.uniform(0.01, 0.1))
        out.append(make_problem(n, d, m, mv, kind, 1.0, rng_range, nug, seed * 1000 + k, lloyd=lloyd,
                                rff=256, name=f"c5-{k}"))
    return out


def slq_normals(nprobe: int, m: int, n: int, seed: int = 20250714) -> np.ndarray:
    """Standard normal numbers of nprobe SLQ probes, row i = (eps1 (m), eps2 (n), eps3 (n)):
    the random draws of the probe recipe, generated here so that every implementation
    receives the same ones."""
    return _rng(seed).standard_normal((nprobe, m + 2 * n))
