"""FP64 CPU oracle of the VIF approximation (Gyger, Furrer & Sigrist, 2025).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  The CUDA library never calls it,
and it shares no code with the CUDA library.

Every function follows the paper's formulas in the paper's own algebra, written
out in numpy/scipy float64, with library primitives (Cholesky, triangular and
dense solves, sparse products, sorting) as the only building blocks:

* covariance functions: the half-integer Matern forms and the Gaussian (SE)
  kernel, r = ||(s - s')/lambda|| (Sec. 2 and Eq. cov_trans_iso of Sec. 6);
* the predictive-process low-rank part  Sigma_mn^T Sigma_m^{-1} Sigma_mn  (Sec. 2.1);
* correlation-based causal neighbour sets with the distance d_c (Sec. 6);
* the residual Vecchia factors A_i, D_i of Eq. D_A_Vecchia (Sec. 2.1);
* the negative log-likelihood through M (Eq. def_M) with Woodbury and
  Sylvester (Sec. 2.2), and the dense definitions used as pins;
* predictive means and variances (Prop. 2.1, App. C.1);
* Laplace mode finding for a Bernoulli-logit likelihood (Eq. one_it_newton_mode)
  with preconditioned CG (Eq. pcls1) and the VIFDU preconditioner (Sec. 4.3, App. E.1);
* the VIF-Laplace likelihood (Eq. log_det_VIFLA) with the preconditioned SLQ
  log-determinant (Eq. slq_v1, App. D), probes drawn by the recipe of Sec. 4.3;
* the FITC preconditioner (Sec. 4.3, App. E.2) with the system form of Eq. pcls2 and
  the SLQ form of Eq. slq_v2;
* VIF-Laplace predictive distributions (Prop. 3.1) and their variances by Alg. 1 (SBPV);
* the analytic gradient of the Gaussian VIF likelihood (Sec. 2.2 trace formula, App. A
  derivatives of B and D), pinned against central differences and the exact GP;
* the VIF-Laplace gradient by stochastic trace estimation with the preconditioner control
  variate (Sec. 4.1, App. B, App. D), in the VIFDU (Eq. pcls1) and the FITC (Eq. pcls2) form.

Readings of points the paper leaves open (all shared with the CUDA path):
  R1 kernel forms of Rasmussen & Williams; "range" = length scale lambda.
  R3 points are ordered as given; prediction points come after all training points.
  R4 d_c uses Sigma without the nugget; if c_r(i,i) or c_r(j,j) <= TAU_V*sigma1^2 the
     correlation is taken as 0; |rho| is clamped to 1; ranking key = 1 - |rho|.
  R5 ties are broken by ascending index.
  R7 Sigma_m += eps*sigma1^2*I (eps = 1e-8 SE, 1e-10 Matern); residual Vecchia blocks
     get +1e-10*sigma1^2 on the diagonal when there is no nugget (latent GP).
  R9 prediction points condition on training points only (B_p = I); their
     neighbours are the m_v nearest training points by d_c (non-causal).
  R10 Newton from b=0; PCG from x=0 stops at ||v - A x||_2/||v||_2 <= tol.
  R17 App. A's derivative of D_i is read as the product rule of D_i = c~_ii - A_i c_Ni: its
      printed term in dA_i multiplies the cross covariance c_Ni (the printed c_ii is garbled).
  R16 derivatives in theta of Sigma_dagger^{-1}, log det Sigma_dagger, log det P^ and B^T W B are
      central differences (relative step 1e-4) with N, Z, W and the mode fixed; the control
      variate is applied to the theta traces, the traces for dL/db use the plain estimate.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SQRT3 = math.sqrt(3.0)
SQRT5 = math.sqrt(5.0)
TAU_V = 1e-6          # R4: residual variances below TAU_V*sigma1^2 count as zero
LOG2PI = math.log(2.0 * math.pi)


# ----------------------------------------------------------------------------
# Covariance functions (Sec. 2, Eq. cov_trans_iso; reading R1)
# ----------------------------------------------------------------------------
def jitter_eps(theta) -> float:
    """R7: relative jitter added to Sigma_m."""
    return 1e-8 if theta.kind == 3 else 1e-10


def residual_diag(theta) -> float:
    """Diagonal added to residual Vecchia blocks: the nugget sigma^2 in the
    Gaussian case (Sigma-tilde of Eq. cov_mat_gauss), else the R7 jitter."""
    return theta.nugget if theta.nugget > 0 else 1e-10 * theta.variance


def cov_of_r(r: np.ndarray, kind: int, variance: float) -> np.ndarray:
    """c(r) for Matern-1/2, 3/2, 5/2 and the squared-exponential kernel (R1)."""
    if kind == 0:
        return variance * np.exp(-r)
    if kind == 1:
        t = SQRT3 * r
        return variance * (1.0 + t) * np.exp(-t)
    if kind == 2:
        t = SQRT5 * r
        return variance * (1.0 + t + t * t / 3.0) * np.exp(-t)
    if kind == 3:
        return variance * np.exp(-0.5 * r * r)
    raise ValueError(kind)


def scaled(X: np.ndarray, theta) -> np.ndarray:
    """q_lambda(s) = s / lambda (Sec. 6, ARD transform)."""
    ls = np.broadcast_to(np.asarray(theta.lengthscale, dtype=np.float64), (X.shape[1],))
    return X / ls


def dist(X1: np.ndarray, X2: np.ndarray) -> np.ndarray:
    """Euclidean distances, computed from coordinate differences (in blocks of X2
    rows so that the temporary stays below ~128 MB)."""
    n1, n2, d = X1.shape[0], X2.shape[0], X1.shape[1]
    out = np.empty((n1, n2))
    blk = max(1, (1 << 24) // max(1, n1 * d))
    for s in range(0, n2, blk):
        diff = X1[:, None, :] - X2[None, s:s + blk, :]
        out[:, s:s + blk] = np.sqrt((diff * diff).sum(-1))
    return out


def cov(X1: np.ndarray, X2: np.ndarray, theta) -> np.ndarray:
    """Cross-covariance matrix [c_theta(s_i, s'_j)] without the nugget."""
    return cov_of_r(dist(scaled(X1, theta), scaled(X2, theta)), theta.kind, theta.variance)


def sigma_m(Z: np.ndarray, theta) -> np.ndarray:
    """Sigma_m with the R7 jitter."""
    S = cov(Z, Z, theta)
    return S + jitter_eps(theta) * theta.variance * np.eye(Z.shape[0])


# ----------------------------------------------------------------------------
# Low-rank part (Sec. 2.1, Eq. def_b_low)
# ----------------------------------------------------------------------------
class LowRank:
    """Holds Sigma_m, its Cholesky factor and Sigma_m^{-1} Sigma_mn for the data.

    lr(i, j) = Sigma_mi^T Sigma_m^{-1} Sigma_mj  (the low-rank covariance Sigma^l),
    computed through a Cholesky solve with Sigma_m itself (the paper's algebra).
    """

    def __init__(self, X: np.ndarray, Z: np.ndarray, theta):
        self.theta = theta
        self.m = Z.shape[0]
        if self.m == 0:
            self.Smn = np.zeros((0, X.shape[0]))
            self.SinvSmn = self.Smn
            self.Sm = np.zeros((0, 0))
            self.cf = None
            return
        self.Sm = sigma_m(Z, theta)
        self.cf = sla.cho_factor(self.Sm, lower=True)
        self.Smn = cov(Z, X, theta)                          # m x n
        self.SinvSmn = sla.cho_solve(self.cf, self.Smn)      # Sigma_m^{-1} Sigma_mn

    def lr(self, idx_a, idx_b) -> np.ndarray:
        return self.Smn[:, idx_a].T @ self.SinvSmn[:, idx_b]

    def lr_diag(self) -> np.ndarray:
        return np.einsum("ij,ij->j", self.Smn, self.SinvSmn)

    def logdet_Sm(self) -> float:
        return 2.0 * float(np.log(np.diag(self.cf[0])).sum()) if self.m else 0.0


# ----------------------------------------------------------------------------
# Correlation-based neighbour selection (Sec. 6, distance d_c; R4, R5)
# ----------------------------------------------------------------------------
def residual_var(X, lowrank: LowRank, theta) -> np.ndarray:
    """c_r(i,i) = Sigma_ii - Sigma_mi^T Sigma_m^{-1} Sigma_mi (no nugget)."""
    return theta.variance - lowrank.lr_diag() if lowrank.m else np.full(X.shape[0], theta.variance)


def corr_keys(q_x: np.ndarray, q_cr: float, X_c: np.ndarray, cr_c: np.ndarray, theta,
              lr_cross: np.ndarray) -> np.ndarray:
    """Ranking key 1 - |rho| of one query against candidates (R4).

    rho = c_r(q,j) / sqrt(c_r(q,q) c_r(j,j)), c_r(q,j) = Sigma_qj - lr(q,j).
    Since d_c = sqrt(1-|rho|) is monotone in the key, ranking by the key gives
    the same order as ranking by d_c.
    """
    K = cov(q_x[None, :], X_c, theta)[0]
    c = K - lr_cross
    tv = TAU_V * theta.variance
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = c / np.sqrt(q_cr * cr_c)
    rho = np.where((q_cr <= tv) | (cr_c <= tv), 0.0, rho)
    rho = np.clip(np.abs(rho), 0.0, 1.0)
    return 1.0 - rho


def causal_neighbors(X, Z, theta, mv: int, return_keys: bool = False):
    """N(i): the min(i, m_v) predecessors j < i with the smallest (key, j)
    (Sec. 2.1 neighbour rule; Sec. 6 distance), stored in ascending index order,
    padded with -1.  Brute force over all j < i."""
    n = X.shape[0]
    lowrank = LowRank(X, Z, theta)
    cr = residual_var(X, lowrank, theta)
    N = -np.ones((n, mv), dtype=np.int64)
    keys = [] if return_keys else None
    for i in range(1, n):
        if lowrank.m:
            lr = lowrank.Smn[:, :i].T @ lowrank.SinvSmn[:, i]
        else:
            lr = np.zeros(i)
        k = corr_keys(X[i], cr[i], X[:i], cr[:i], theta, lr)
        q = min(i, mv)
        order = np.lexsort((np.arange(i), k))[:q]
        N[i, :q] = np.sort(order)
        if return_keys:
            keys.append(k)
    if return_keys:
        return N, keys, cr
    return N


def causal_neighbors_sample(X, Z, theta, mv: int, queries, chunk: int = 65536):
    """N(i) and all keys of selected queries only, streaming over the predecessors
    in chunks (the same definition as causal_neighbors, for full-size checks)."""
    queries = np.asarray(queries, dtype=np.int64)
    m = Z.shape[0]
    tv = TAU_V * theta.variance
    if m:
        cf = sla.cho_factor(sigma_m(Z, theta), lower=True)
        Sq = cov(Z, X[queries], theta)
        Wq = sla.cho_solve(cf, Sq)
        crq = theta.variance - (Sq * Wq).sum(0)
    else:
        crq = np.full(len(queries), theta.variance)
    imax = int(queries.max())
    keys = [np.empty(int(i)) for i in queries]
    for s0 in range(0, imax, chunk):
        s1 = min(imax, s0 + chunk)
        Xc = X[s0:s1]
        if m:
            Sc = cov(Z, Xc, theta)
            crc = theta.variance - (Sc * sla.cho_solve(cf, Sc)).sum(0)
            LR = Wq.T @ Sc
        else:
            crc = np.full(s1 - s0, theta.variance)
            LR = np.zeros((len(queries), s1 - s0))
        K = cov(X[queries], Xc, theta)
        for a, i in enumerate(queries):
            e = min(int(i), s1)
            if e <= s0:
                continue
            c = K[a, :e - s0] - LR[a, :e - s0]
            with np.errstate(divide="ignore", invalid="ignore"):
                rho = c / np.sqrt(crq[a] * crc[:e - s0])
            rho = np.where((crq[a] <= tv) | (crc[:e - s0] <= tv), 0.0, rho)
            keys[a][s0:e] = 1.0 - np.clip(np.abs(rho), 0.0, 1.0)
    Ns = []
    for a, i in enumerate(queries):
        q = min(int(i), mv)
        order = np.lexsort((np.arange(int(i)), keys[a]))[:q]
        Ns.append(np.sort(order))
    return Ns, keys


def vecchia_factors_rows(X, Z, theta, N, rows):
    """A_i and D_i (Eq. D_A_Vecchia) for selected rows only: the low-rank terms
    are formed on the selected points and their neighbours alone."""
    rows = np.asarray(rows, dtype=np.int64)
    need = np.unique(np.concatenate([rows, N[rows][N[rows] >= 0].ravel()]))
    pos = {int(j): k for k, j in enumerate(need)}
    Nsub = -np.ones((len(rows), N.shape[1]), dtype=np.int64)
    Xsub = np.concatenate([X[need]])
    # points of the reduced problem: the needed ones; rows refer into it
    lr = LowRank(Xsub, Z, theta)
    tdiag = residual_diag(theta)
    out_A = np.zeros((len(rows), N.shape[1]))
    out_D = np.empty(len(rows))
    for a, i in enumerate(rows):
        nb = [pos[int(j)] for j in N[i] if j >= 0]
        ii = pos[int(i)]
        q = len(nb)
        dii = theta.variance + tdiag - (lr.lr(ii, ii) if lr.m else 0.0)
        if q == 0:
            out_D[a] = dii
            continue
        S_iN = cov(Xsub[ii:ii + 1], Xsub[nb], theta)[0]
        S_NN = cov(Xsub[nb], Xsub[nb], theta) + tdiag * np.eye(q)
        if lr.m:
            S_iN_l = S_iN - lr.lr([ii], nb)[0]
            S_NN_l = S_NN - lr.lr(nb, nb)
        else:
            S_iN_l, S_NN_l = S_iN, S_NN
        Ai = np.linalg.solve(S_NN_l, S_iN_l)
        out_A[a, :q] = Ai
        out_D[a] = dii - Ai @ S_iN_l
    return out_A, out_D


# ----------------------------------------------------------------------------
# Residual Vecchia factors (Sec. 2.1, Eq. D_A_Vecchia)
# ----------------------------------------------------------------------------
def vecchia_factors(X, Z, theta, N, lowrank: LowRank | None = None):
    """Returns (Acoef, D): Acoef[i, :q_i] = A_i (row of -B on N(i)), D[i] = D_i.

    A_i = (Sigma_iN - Sigma_mi^T Sigma_m^{-1} Sigma_mN)(Sigma~_N - Sigma_mN^T Sigma_m^{-1} Sigma_mN)^{-1}
    D_i = Sigma~_ii - Sigma_mi^T Sigma_m^{-1} Sigma_mi - A_i (Sigma_iN^T - Sigma_mN^T Sigma_m^{-1} Sigma_mi)
    Sigma~ carries the nugget (Gaussian) or the R7 jitter (latent GP).
    Points with the same neighbour count are processed as one batch of solves.
    """
    n = X.shape[0]
    mv = N.shape[1]
    lowrank = lowrank or LowRank(X, Z, theta)
    tdiag = residual_diag(theta)
    Acoef = np.zeros((n, mv))
    D = np.empty(n)
    q_of = (N >= 0).sum(1)
    Xs = scaled(X, theta)
    for q in np.unique(q_of):
        I = np.nonzero(q_of == q)[0]
        for s in range(0, len(I), 4096):
            Ib = I[s:s + 4096]
            dii = theta.variance + tdiag
            lrii = (lowrank.Smn[:, Ib] * lowrank.SinvSmn[:, Ib]).sum(0) if lowrank.m else 0.0
            if q == 0:
                D[Ib] = dii - lrii
                continue
            Nb = N[Ib, :q]                                        # b x q
            xi = Xs[Ib]                                           # b x d
            xn = Xs[Nb]                                           # b x q x d
            r_iN = np.sqrt(((xi[:, None, :] - xn) ** 2).sum(-1))
            S_iN = cov_of_r(r_iN, theta.kind, theta.variance)     # b x q
            r_NN = np.sqrt(((xn[:, :, None, :] - xn[:, None, :, :]) ** 2).sum(-1))
            S_NN = cov_of_r(r_NN, theta.kind, theta.variance) + tdiag * np.eye(q)
            if lowrank.m:
                Smi = lowrank.Smn[:, Ib].T                        # b x m
                Wi = lowrank.SinvSmn[:, Ib].T                     # b x m
                SmN = lowrank.Smn[:, Nb].transpose(1, 2, 0)       # b x q x m
                WN = lowrank.SinvSmn[:, Nb].transpose(1, 2, 0)    # b x q x m
                lr_iN = np.matmul(WN, Smi[:, :, None])[:, :, 0]        # Sigma_mi^T Sigma_m^-1 Sigma_mN
                lr_NN = np.matmul(SmN, WN.transpose(0, 2, 1))
                lr_Ni = np.matmul(SmN, Wi[:, :, None])[:, :, 0]
            else:
                lr_iN = lr_Ni = 0.0
                lr_NN = 0.0
            left = S_iN - lr_iN
            Mat = S_NN - lr_NN
            Ai = np.linalg.solve(Mat, left[:, :, None])[:, :, 0]   # Mat symmetric
            Acoef[Ib, :q] = Ai
            D[Ib] = dii - lrii - (Ai * (S_iN - lr_Ni)).sum(1)
    return Acoef, D


def residual_neighbor_corr(X, Z, theta, N) -> np.ndarray:
    """Per point i: the largest and the mean |rho(i, j)| over its neighbours j in N(i), rho
    the correlation of the residual process whose covariance the residual Vecchia blocks
    hold (Sec. 2.1: Sigma~ - Sigma_mn^T Sigma_m^{-1} Sigma_mn, the nugget or the R7 jitter on
    the diagonal); zeros for points without neighbours.  Inputs 8 and 9 of the learned
    preconditioner correction."""
    n = X.shape[0]
    lowrank = LowRank(X, Z, theta)
    tdiag = residual_diag(theta)
    cdiag = theta.variance + tdiag - (lowrank.lr_diag() if lowrank.m else np.zeros(n))
    out = np.zeros((n, 2))
    for i in range(n):
        nb = N[i][N[i] >= 0]
        if len(nb) == 0:
            continue
        c = cov(X[i:i + 1], X[nb], theta)[0]
        if lowrank.m:
            c = c - lowrank.lr([i], nb)[0]
        r = np.abs(c / np.sqrt(cdiag[i] * cdiag[nb]))
        out[i] = r.max(), r.mean()
    return out


def B_matrix(N, Acoef) -> sp.csr_matrix:
    """Unit lower-triangular B with B_{i,N(i)} = -A_i (Sec. 2.1)."""
    n, mv = N.shape
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.ones(n)]
    mask = N >= 0
    r = np.repeat(np.arange(n)[:, None], mv, 1)[mask]
    rows.append(r)
    cols.append(N[mask])
    vals.append(-Acoef[mask])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


# ----------------------------------------------------------------------------
# Negative log-likelihood (Sec. 2.1-2.2)
# ----------------------------------------------------------------------------
class VIF:
    """All factors of one VIF approximation: Sigma_m, Sigma_mn, B, D, M."""

    def __init__(self, X, Z, theta, N):
        self.X, self.Z, self.theta, self.N = X, Z, theta, N
        self.n = X.shape[0]
        self.m = Z.shape[0]
        self.lowrank = LowRank(X, Z, theta)
        self.Acoef, self.D = vecchia_factors(X, Z, theta, N, self.lowrank)
        self.B = B_matrix(N, self.Acoef)
        self.Dinv = 1.0 / self.D
        if self.m:
            Smn = self.lowrank.Smn
            # Q Sigma_mn^T with Q = B^T D^{-1} B, then M of Eq. def_M
            self.QSnm = self.Q(Smn.T)
            self.M = self.lowrank.Sm + Smn @ self.QSnm
            self.Mcf = sla.cho_factor(self.M, lower=True)

    def Q(self, V):
        """Q V = B^T D^{-1} B V."""
        BV = self.B @ V
        if BV.ndim == 1:
            return self.B.T @ (self.Dinv * BV)
        return self.B.T @ (self.Dinv[:, None] * BV)

    def Sigma_dagger_inv(self, v):
        """Woodbury: Q v - Q Sigma_mn^T M^{-1} Sigma_mn Q v (Sec. 2.2)."""
        Qv = self.Q(v)
        if not self.m:
            return Qv
        return Qv - self.QSnm @ sla.cho_solve(self.Mcf, self.lowrank.Smn @ Qv)

    def logdet(self) -> float:
        """Sylvester: log det M - log det Sigma_m + log det D (Sec. 2.2)."""
        ld = float(np.log(self.D).sum())
        if self.m:
            ld += 2.0 * float(np.log(np.diag(self.Mcf[0])).sum()) - self.lowrank.logdet_Sm()
        return ld

    def nll(self, y) -> float:
        quad = float(y @ self.Sigma_dagger_inv(y))
        return 0.5 * (self.n * LOG2PI + self.logdet() + quad)

    def nll_whitened(self, y) -> float:
        """The same likelihood (Woodbury and Sylvester, Sec. 2.2) evaluated in the basis that the
        Cholesky factor L_m of Sigma_m whitens: with W = L_m^{-1} Sigma_mn (triangular solve),
        F = D^{-1/2} B W^T, z = D^{-1/2} B y and u = F^T z,
            log det M - log det Sigma_m = log det(I + F^T F)        (L_m^{-1} M L_m^{-T} = I + F^T F)
            y^T Q y - (Sigma_mn Q y)^T M^{-1} Sigma_mn Q y = z^T z - u^T (I + F^T F)^{-1} u.
        M itself has eigenvalues from those of Sigma_m (1e-4 at n = 5e5, d = 8, m = 500) up to
        the data's weight (1e7), so its float64 Cholesky carries an error of ~1e-8 of the
        likelihood at that size (two float64 platforms disagree by that much on the M form);
        I + F^T F has eigenvalues >= 1.  Used as the reference for large problems, and pinned to
        the M form and the dense definition on small ones."""
        ld = float(np.log(self.D).sum())
        rs = 1.0 / np.sqrt(self.D)
        z = rs * (self.B @ y)
        quad = float(z @ z)
        if self.m:
            W = sla.solve_triangular(self.lowrank.cf[0], self.lowrank.Smn, lower=True)   # m x n
            F = (self.B @ W.T) * rs[:, None]                                            # n x m
            C = np.eye(self.m) + F.T @ F
            Lc = np.linalg.cholesky(C)
            w = sla.solve_triangular(Lc, F.T @ z, lower=True)
            ld += 2.0 * float(np.log(np.diag(Lc)).sum())
            quad -= float(w @ w)
        return 0.5 * (self.n * LOG2PI + ld + quad)

    def dense_Sigma_dagger(self) -> np.ndarray:
        """Sigma~_dagger = Sigma^l + (B^T D^{-1} B)^{-1}, formed explicitly (small n)."""
        Binv = np.linalg.inv(self.B.toarray())
        S = Binv @ np.diag(self.D) @ Binv.T
        if self.m:
            S = S + self.lowrank.Smn.T @ self.lowrank.SinvSmn
        return S


def vif_nll(X, Z, theta, N, y) -> float:
    return VIF(X, Z, theta, N).nll(y)


def dense_nll(S: np.ndarray, y: np.ndarray) -> float:
    """-log N(y; 0, S) by a dense Cholesky (Sec. 2, first display)."""
    L = np.linalg.cholesky(S)
    a = sla.solve_triangular(L, y, lower=True)
    return 0.5 * (len(y) * LOG2PI + 2.0 * np.log(np.diag(L)).sum() + a @ a)


def exact_cov(X, theta) -> np.ndarray:
    """Sigma~ = Sigma + sigma^2 I (Eq. cov_mat_gauss)."""
    return cov(X, X, theta) + theta.nugget * np.eye(X.shape[0])


def fitc_cov(X, Z, theta) -> np.ndarray:
    """FITC covariance: Sigma^l + diag(Sigma~ - Sigma^l) (Sec. 2.1, m_v = 0)."""
    lr = LowRank(X, Z, theta)
    Sl = lr.Smn.T @ lr.SinvSmn
    Sf = exact_cov(X, theta)
    return Sl + np.diag(np.diag(Sf) - np.diag(Sl))


# ----------------------------------------------------------------------------
# Prediction (Prop. 2.1, proof, App. C.1; reading R9)
# ----------------------------------------------------------------------------
def pred_neighbors(X, Z, theta, Xp, mv: int, lowrank: LowRank | None = None):
    """N_p(j): the m_v training points with the smallest d_c to prediction point j."""
    lowrank = lowrank or LowRank(X, Z, theta)
    n = X.shape[0]
    cr = residual_var(X, lowrank, theta)
    lrp = LowRank(Xp, Z, theta)
    crp = residual_var(Xp, lrp, theta)
    Np = np.empty((Xp.shape[0], mv), dtype=np.int64)
    for p in range(Xp.shape[0]):
        lr = (lowrank.Smn.T @ lrp.SinvSmn[:, p]) if lowrank.m else np.zeros(n)
        k = corr_keys(Xp[p], crp[p], X, cr, theta, lr)
        order = np.lexsort((np.arange(n), k))[:mv]
        Np[p] = np.sort(order)
    return Np


def pred_factors(X, Z, theta, Xp, Np, lowrank: LowRank):
    """Rows of B_po (coefficients A_p on N_p) and D_p for the joint residual
    Vecchia approximation of Eq. vecchia_pred with B_p = I (R9)."""
    npred, mv = Np.shape
    tdiag = residual_diag(theta)
    lrp = LowRank(Xp, Z, theta)
    Ap = np.zeros((npred, mv))
    Dp = np.empty(npred)
    for p in range(npred):
        Nn = Np[p]
        S_pN = cov(Xp[p:p + 1], X[Nn], theta)[0]
        S_NN = cov(X[Nn], X[Nn], theta) + tdiag * np.eye(mv)
        if lowrank.m:
            lr_pN = lrp.Smn[:, p] @ lowrank.SinvSmn[:, Nn]
            lr_NN = lowrank.Smn[:, Nn].T @ lowrank.SinvSmn[:, Nn]
            lr_pp = lrp.Smn[:, p] @ lrp.SinvSmn[:, p]
        else:
            lr_pN, lr_NN, lr_pp = np.zeros(mv), 0.0, 0.0
        c = S_pN - lr_pN
        a = np.linalg.solve(S_NN - lr_NN, c)
        Ap[p] = a
        Dp[p] = theta.variance + tdiag - lr_pp - a @ c
    return Ap, Dp, lrp


def predict_prop21_dense(vif: VIF, y, Xp, Np):
    """Predictive mean and covariance of Prop. 2.1 evaluated literally with
    dense matrices (small n only).  Returns (mean, Sigma^p) for the response."""
    X, Z, theta = vif.X, vif.Z, vif.theta
    n = vif.n
    Ap, Dp, lrp = pred_factors(X, Z, theta, Xp, Np, vif.lowrank)
    npred = Xp.shape[0]
    Bpo = np.zeros((npred, n))
    for p in range(npred):
        Bpo[p, Np[p]] = -Ap[p]
    Bp_inv = np.eye(npred)
    Bd = vif.B.toarray()
    Prec = Bd.T @ np.diag(vif.Dinv) @ Bd            # B^T D^{-1} B
    PrecInv = np.linalg.inv(Prec)
    if vif.m:
        Smn, Smnp = vif.lowrank.Smn, lrp.Smn
        SmInv = np.linalg.inv(vif.lowrank.Sm)
        LRpn = Smnp.T @ SmInv @ Smn                   # Sigma_mnp^T Sigma_m^-1 Sigma_mn
        LRpp = Smnp.T @ SmInv @ Smnp
        Minv = np.linalg.inv(vif.M)
        SMS = Smn.T @ Minv @ Smn                      # Sigma_mn^T M^-1 Sigma_mn
    else:
        LRpn = np.zeros((npred, n))
        LRpp = np.zeros((npred, npred))
        SMS = np.zeros((n, n))
    mu = (-Bp_inv @ Bpo @ y + LRpn @ Prec @ y - LRpn @ Prec @ SMS @ Prec @ y
          + Bp_inv @ Bpo @ SMS @ Prec @ y)
    Sd_inv = Prec - Prec @ SMS @ Prec                  # Sigma~_dagger^{-1}
    left = LRpn - Bp_inv @ Bpo @ PrecInv
    Sig = (Bp_inv @ np.diag(Dp) @ Bp_inv.T + Bp_inv @ Bpo @ PrecInv @ Bpo.T @ Bp_inv.T + LRpp
           - left @ Sd_inv @ left.T)
    return mu, Sig


def predict_appC(vif: VIF, y, Xp, Np):
    """Predictive mean (Prop. 2.1) and variances via the expansion of App. C.1,
    using only sparse products and m x m solves.  Returns (mean, var) for the
    response y^p; subtract the nugget for the latent process."""
    X, Z, theta = vif.X, vif.Z, vif.theta
    Ap, Dp, lrp = pred_factors(X, Z, theta, Xp, Np, vif.lowrank)
    npred = Xp.shape[0]
    rows = np.repeat(np.arange(npred), Np.shape[1])
    Bpo = sp.csr_matrix((-Ap.ravel(), (rows, Np.ravel())), shape=(npred, vif.n))
    Qy = vif.Q(y)
    if not vif.m:
        mu = -(Bpo @ y)
        # (B^T D^-1 B)^-1 B_po^T rows are needed only for the cancelled term
        return mu, Dp.copy()
    Smn, Smnp = vif.lowrank.Smn, lrp.Smn
    cfS, cfM = vif.lowrank.cf, vif.Mcf
    SmInvSmnp = sla.cho_solve(cfS, Smnp)               # Sigma_m^-1 Sigma_mnp  (m x np)
    SmnQy = Smn @ Qy
    MinvSmnQy = sla.cho_solve(cfM, SmnQy)
    # mean, Prop. 2.1 (B_p = I)
    mu = (-(Bpo @ y) + SmInvSmnp.T @ SmnQy - SmInvSmnp.T @ (Smn @ vif.Q(Smn.T @ MinvSmnQy))
          + Bpo @ (Smn.T @ MinvSmnQy))
    # variances, App. C.1 (diagonal of each term)
    T = Smn @ vif.QSnm                                  # Sigma_mn B^T D^-1 B Sigma_mn^T  (m x m)
    U = Smn @ Bpo.T.toarray()                           # Sigma_mn B_po^T (m x np)
    V = SmInvSmnp                                       # Sigma_m^-1 Sigma_mnp
    MinvU = sla.cho_solve(cfM, U)
    MinvTV = sla.cho_solve(cfM, T @ V)
    t1 = Dp
    t2 = (Smnp * V).sum(0)                              # Sigma_mnp^T Sigma_m^-1 Sigma_mnp
    t3 = -(V * (T @ V)).sum(0)
    t4 = (V * U).sum(0)                                 # Sigma_mnp^T Sigma_m^-1 Sigma_mn B_po^T
    t5 = t4
    t6 = (U * MinvU).sum(0)                             # B_po Sigma_mn^T M^-1 Sigma_mn B_po^T
    t7 = -(U * MinvTV).sum(0)
    t8 = t7
    t9 = ((T @ V) * MinvTV).sum(0)
    var = t1 + t2 + t3 + t4 + t5 + t6 + t7 + t8 + t9
    return mu, var


def exact_predict(X, y, theta, Xp):
    """Exact GP predictive mean and variance of y^p (Sec. 2, second paragraph)."""
    S = exact_cov(X, theta)
    Snp = cov(X, Xp, theta)
    L = np.linalg.cholesky(S)
    alpha = sla.cho_solve((L, True), y)
    mu = Snp.T @ alpha
    Vv = sla.solve_triangular(L, Snp, lower=True)
    var = theta.variance + theta.nugget - (Vv * Vv).sum(0)
    return mu, var


# ----------------------------------------------------------------------------
# Laplace approximation for Bernoulli-logit (Sec. 3, Sec. 4)
# ----------------------------------------------------------------------------
def bern_grad_W(y, b):
    """d log p(y|b)/db = y - sigmoid(b);  W_ii = sigmoid(b)(1 - sigmoid(b)) (Eq. W_diag)."""
    p = 1.0 / (1.0 + np.exp(-b))
    return y - p, p * (1.0 - p)


def bern_loglik(y, b) -> float:
    return float((y * b - np.logaddexp(0.0, b)).sum())


class VIFDU:
    """VIFDU preconditioner P^ = B^T W B + Sigma_dagger^{-1} applied with the
    formula of App. E.1: B^{-1}[(W+D^{-1})^{-1} + (W+D^{-1})^{-1} D^{-1} B Sigma_mn^T
    M_3^{-1} Sigma_mn B^T D^{-1} (W+D^{-1})^{-1}] B^{-T},
    M_3 = M - Sigma_mn B^T D^{-1} (W+D^{-1})^{-1} D^{-1} B Sigma_mn^T."""

    def __init__(self, vif: VIF, W):
        self.vif = vif
        self.Ginv = 1.0 / (W + vif.Dinv)
        self.Bcsr = vif.B.tocsr()
        self.BTcsr = vif.B.T.tocsr()
        if vif.m:
            DBS = vif.Dinv[:, None] * (vif.B @ vif.lowrank.Smn.T)     # D^-1 B Sigma_mn^T
            self.DBS = DBS
            self.M3 = vif.M - DBS.T @ (self.Ginv[:, None] * DBS)
            self.M3cf = sla.cho_factor(self.M3, lower=True)

    def apply(self, w):
        x = spla.spsolve_triangular(self.BTcsr, w, lower=False)          # B^{-T} w
        g = self.Ginv * x
        if self.vif.m:
            g = g + self.Ginv * (self.DBS @ sla.cho_solve(self.M3cf, self.DBS.T @ g))
        return spla.spsolve_triangular(self.Bcsr, g, lower=True)          # B^{-1} (.)

    def dense(self, W) -> np.ndarray:
        B = self.vif.B.toarray()
        n = self.vif.n
        Sdi = np.column_stack([self.vif.Sigma_dagger_inv(e) for e in np.eye(n)])
        return B.T @ np.diag(W) @ B + Sdi


def pcg(matvec, precond, v, tol: float, max_iter: int):
    """Preconditioned CG from x=0 on (W + Sigma_dagger^{-1}) x = v (Eq. pcls1);
    stops when ||r||_2/||v||_2 <= tol (R10).  Returns (x, iterations, rel_res)."""
    x = np.zeros_like(v)
    r = v.copy()
    nv = np.linalg.norm(v)
    if nv == 0:
        return x, 0, 0.0
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        Ap = matvec(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rel = np.linalg.norm(r) / nv
        if rel <= tol:
            return x, it, rel
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, rel


def laplace_mode(vif: VIF, y, tol=1e-6, max_pcg=1000, max_newton=50, psi_tol=1e-10,
                 dense: bool = False):
    """Newton iterations of Eq. one_it_newton_mode from b=0 (R10); each linear
    solve uses PCG with the VIFDU preconditioner, or a dense solve if `dense`.
    Returns (mode, newton_steps, total_pcg_iterations)."""
    n = vif.n
    b = np.zeros(n)
    psi_old = None
    tot = 0
    Sdi_dense = None
    if dense:
        Sdi_dense = np.linalg.inv(vif.dense_Sigma_dagger())
    for t in range(1, max_newton + 1):
        g, W = bern_grad_W(y, b)
        v = W * b + g
        if dense:
            b = np.linalg.solve(np.diag(W) + Sdi_dense, v)
        else:
            pre = VIFDU(vif, W)
            b, it, _ = pcg(lambda w: W * w + vif.Sigma_dagger_inv(w), pre.apply, v, tol, max_pcg)
            tot += it
        psi = bern_loglik(y, b) - 0.5 * float(b @ vif.Sigma_dagger_inv(b))
        if psi_old is not None and abs(psi - psi_old) <= psi_tol * abs(psi):
            return b, t, tot
        psi_old = psi
    return b, max_newton, tot


# ----------------------------------------------------------------------------
# VIF-Laplace negative log-marginal likelihood (Eq. log_det_VIFLA) with the
# preconditioned stochastic Lanczos quadrature of Eq. slq_v1 (Sec. 4.1, App. D)
# ----------------------------------------------------------------------------
def vifdu_logdet(vif: VIF, W) -> float:
    """log det P^ = log det(W + D^{-1}) - log det M + log det M_3 (App. E.1, Sylvester)."""
    ld = float(np.log(W + vif.Dinv).sum())
    if vif.m:
        pre = VIFDU(vif, W)
        ld += 2.0 * float(np.log(np.diag(pre.M3cf[0])).sum()) - 2.0 * float(np.log(np.diag(vif.Mcf[0])).sum())
    return ld


def vifdu_sample(vif: VIF, W, eps1, eps2, eps3):
    """A draw from N(0, P^) by the recipe of Sec. 4.3:
    B^T W^{1/2} eps3 + Sigma_dagger^{-1} (B^{-1} D^{1/2} eps2 + Sigma_mn^T Sigma_m^{-T/2} eps1),
    Sigma_m = L L^T (L lower) and Sigma_m^{-T/2} = L^{-T}, so that the bracket has covariance
    Sigma_dagger (reading of the paper's Sigma_m^{-1/2}).  eps1 (m), eps2, eps3 (n) are standard
    normal vectors supplied by the caller."""
    s = spla.spsolve_triangular(vif.B.tocsr(), np.sqrt(vif.D) * eps2, lower=True)
    if vif.m:
        s = s + vif.lowrank.Smn.T @ sla.solve_triangular(vif.lowrank.cf[0], eps1, lower=True, trans="T")
    return vif.B.T @ (np.sqrt(W) * eps3) + vif.Sigma_dagger_inv(s)


def pcg_lanczos(matvec, precond, v, tol: float, max_iter: int):
    """The PCG of `pcg` (Eq. pcls1, R10 stopping rule), also returning the Lanczos
    tridiagonal matrix of the preconditioned operator that its coefficients define
    (App. D, after Saad): with step lengths alpha_j and direction updates
    beta_j = r_{j+1}^T z_{j+1} / r_j^T z_j,
        T[0,0] = 1/alpha_0,  T[j,j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},
        T[j,j-1] = T[j-1,j] = sqrt(beta_{j-1})/alpha_{j-1},
    and the starting vector's squared length v^T P^{-1} v.
    Returns (x, iterations, rel_res, T, v^T P^{-1} v)."""
    x = np.zeros_like(v)
    r = v.copy()
    nv = np.linalg.norm(v)
    z = precond(r)
    p = z.copy()
    rz = r @ z
    rz0 = rz
    alphas, betas = [], []
    it, rel = 0, 0.0
    for it in range(1, max_iter + 1):
        Ap = matvec(p)
        alpha = rz / (p @ Ap)
        alphas.append(alpha)
        x += alpha * p
        r -= alpha * Ap
        rel = np.linalg.norm(r) / nv
        if rel <= tol:
            break
        z = precond(r)
        rz_new = r @ z
        betas.append(rz_new / rz)
        p = z + betas[-1] * p
        rz = rz_new
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j > 0:
            T[j, j - 1] = T[j - 1, j] = math.sqrt(betas[j - 1]) / alphas[j - 1]
    return x, it, rel, T, float(rz0)


def lanczos_log_quadrature(T) -> float:
    """e_1^T log(T) e_1: Gauss quadrature of log with the eigenvalues of T as nodes
    and the squared first eigenvector components as weights (App. D)."""
    lam, V = np.linalg.eigh(T)
    return float((V[0, :] ** 2) @ np.log(lam))


def vifla_nll_slq(vif: VIF, y, b, eps, tol: float, max_iter: int = 1000):
    """L^VIFLA of Eq. log_det_VIFLA at the mode b, the log-determinant by Eq. slq_v1:
        log det(Sigma_dagger W + I) ~ log det Sigma_dagger + (n/l) sum_i e_1^T log(T_i) e_1 + log det P^,
    T_i from PCG on (W + Sigma_dagger^{-1}) x = z_i with the VIFDU preconditioner P^ and
    z_i ~ N(0, P^) drawn from eps[i] = (eps1 (m), eps2 (n), eps3 (n)).  Returns a dict with
    the NLL and its parts, the per-probe quadratures q_i, z_i^T P^{-1} z_i and PCG counts."""
    n, m = vif.n, vif.m
    g, W = bern_grad_W(y, b)
    pre = VIFDU(vif, W)
    A = lambda w: W * w + vif.Sigma_dagger_inv(w)
    q, zpz, its = [], [], []
    for e in np.atleast_2d(eps):
        z = vifdu_sample(vif, W, e[:m], e[m:m + n], e[m + n:m + 2 * n])
        _, it, _, T, zz = pcg_lanczos(A, pre.apply, z, tol, max_iter)
        q.append(lanczos_log_quadrature(T))
        zpz.append(zz)
        its.append(it)
    q, zpz = np.array(q), np.array(zpz)
    ld_sigma = vif.logdet()
    ld_P = vifdu_logdet(vif, W)
    slq = n / len(q) * float(q.sum())
    logdet = ld_sigma + slq + ld_P
    nll_lik = -bern_loglik(y, b)
    quad = float(b @ vif.Sigma_dagger_inv(b))
    return dict(nll=nll_lik + 0.5 * quad + 0.5 * logdet, neg_log_lik=nll_lik, quad=quad,
                logdet_sigma=ld_sigma, logdet_P=ld_P, slq_term=slq, logdet=logdet,
                logdet_exact_norm=ld_sigma + float((zpz * q).mean()) + ld_P,
                q=q, zPz=zpz, pcg_iters=np.array(its))


class FITCPrecond:
    """FITC preconditioner P^ = D_V + Sigma_kn^T Sigma_k^{-1} Sigma_kn with
    D_V = diag(Sigma - Sigma_kn^T Sigma_k^{-1} Sigma_kn) + W^{-1} (Sec. 4.3, App. E.2), its
    inducing points being those of the VIF approximation (k = m).  Solves by Woodbury with
    M_V = Sigma_k + Sigma_kn D_V^{-1} Sigma_kn^T; log det by Sylvester; draws by
    D_V^{1/2} eps2 + Sigma_kn^T Sigma_k^{-T/2} eps1 (Sigma_k = L L^T, L lower)."""

    def __init__(self, vif: VIF, W):
        self.vif = vif
        lr = vif.lowrank
        self.DV = vif.theta.variance - (lr.lr_diag() if vif.m else 0.0) + 1.0 / W
        if vif.m:
            self.MV = lr.Sm + lr.Smn @ (lr.Smn.T / self.DV[:, None])
            self.MVcf = sla.cho_factor(self.MV, lower=True)

    def apply(self, w):
        g = w / self.DV
        if self.vif.m:
            lr = self.vif.lowrank
            g = g - (lr.Smn.T @ sla.cho_solve(self.MVcf, lr.Smn @ g)) / self.DV
        return g

    def logdet(self) -> float:
        ld = float(np.log(self.DV).sum())
        if self.vif.m:
            ld += 2.0 * float(np.log(np.diag(self.MVcf[0])).sum()) - self.vif.lowrank.logdet_Sm()
        return ld

    def sample(self, eps1, eps2):
        z = np.sqrt(self.DV) * eps2
        if self.vif.m:
            lr = self.vif.lowrank
            z = z + lr.Smn.T @ sla.solve_triangular(lr.cf[0], eps1, lower=True, trans="T")
        return z

    def dense(self) -> np.ndarray:
        S = np.diag(self.DV)
        if self.vif.m:
            S = S + self.vif.lowrank.Smn.T @ self.vif.lowrank.SinvSmn
        return S


def Sigma_dagger_matvec(vif: VIF, x):
    """Sigma_dagger x = B^{-1} D B^{-T} x + Sigma_mn^T Sigma_m^{-1} Sigma_mn x (Sec. 2.1)."""
    t = spla.spsolve_triangular(vif.B.T.tocsr(), x, lower=False)
    out = spla.spsolve_triangular(vif.B.tocsr(), vif.D * t, lower=True)
    if vif.m:
        out = out + vif.lowrank.Smn.T @ (vif.lowrank.SinvSmn @ x)
    return out


def laplace_mode_fitc(vif: VIF, y, tol=1e-6, max_pcg=1000, max_newton=50, psi_tol=1e-10):
    """Newton iterations of Eq. one_it_newton_mode from b = 0 (R10), each system solved in the
    form of Eq. pcls2, (W^{-1} + Sigma_dagger)(W u) = Sigma_dagger v, by PCG with the FITC
    preconditioner.  Returns (mode, newton_steps, total_pcg_iterations)."""
    n = vif.n
    b = np.zeros(n)
    psi_old = None
    tot = 0
    for t in range(1, max_newton + 1):
        g, W = bern_grad_W(y, b)
        v = W * b + g
        pre = FITCPrecond(vif, W)
        rhs = Sigma_dagger_matvec(vif, v)
        yw, it, _ = pcg(lambda w: w / W + Sigma_dagger_matvec(vif, w), pre.apply, rhs, tol, max_pcg)
        b = yw / W
        tot += it
        psi = bern_loglik(y, b) - 0.5 * float(b @ vif.Sigma_dagger_inv(b))
        if psi_old is not None and abs(psi - psi_old) <= psi_tol * abs(psi):
            return b, t, tot
        psi_old = psi
    return b, max_newton, tot


def vifla_nll_slq_fitc(vif: VIF, y, b, eps, tol: float, max_iter: int = 1000):
    """L^VIFLA of Eq. log_det_VIFLA at the mode b, the log-determinant by Eq. slq_v2:
        log det(Sigma_dagger W + I) ~ log det W + (n/l) sum_i e_1^T log(T_i) e_1 + log det P^,
    T_i from PCG on (W^{-1} + Sigma_dagger) x = z_i with the FITC preconditioner P^ and
    z_i ~ N(0, P^) drawn from eps[i] = (eps1 (m), eps2 (n))."""
    n, m = vif.n, vif.m
    g, W = bern_grad_W(y, b)
    pre = FITCPrecond(vif, W)
    A = lambda w: w / W + Sigma_dagger_matvec(vif, w)
    q, zpz, its = [], [], []
    for e in np.atleast_2d(eps):
        z = pre.sample(e[:m], e[m:m + n])
        _, it, _, T, zz = pcg_lanczos(A, pre.apply, z, tol, max_iter)
        q.append(lanczos_log_quadrature(T))
        zpz.append(zz)
        its.append(it)
    q, zpz = np.array(q), np.array(zpz)
    ld_W = float(np.log(W).sum())
    ld_P = pre.logdet()
    slq = n / len(q) * float(q.sum())
    logdet = ld_W + slq + ld_P
    nll_lik = -bern_loglik(y, b)
    quad = float(b @ vif.Sigma_dagger_inv(b))
    return dict(nll=nll_lik + 0.5 * quad + 0.5 * logdet, neg_log_lik=nll_lik, quad=quad,
                logdet_W=ld_W, logdet_P=ld_P, slq_term=slq, logdet=logdet,
                logdet_exact_norm=ld_W + float((zpz * q).mean()) + ld_P,
                q=q, zPz=zpz, pcg_iters=np.array(its))


def laplace_predict_dense(vif: VIF, y, b, Xp, Np):
    """Prop. 3.1 with dense matrices (small n): the latent predictive mean omega_p and covariance
    Omega_p at the mode b.  The first part of Omega_p and omega_p have the algebra of Prop. 2.1
    with y replaced by b (predict_prop21_dense); the Laplace part adds
    K_p Sigma_dagger^{-1} (W + Sigma_dagger^{-1})^{-1} Sigma_dagger^{-1} K_p^T with
    K_p = Sigma_mnp^T Sigma_m^{-1} Sigma_mn - B_p^{-1} B_po (B^T D^{-1} B)^{-1}."""
    mu, Sig = predict_prop21_dense(vif, b, Xp, Np)
    X, Z, theta = vif.X, vif.Z, vif.theta
    n = vif.n
    Ap, Dp, lrp = pred_factors(X, Z, theta, Xp, Np, vif.lowrank)
    npred = Xp.shape[0]
    Bpo = np.zeros((npred, n))
    for p in range(npred):
        Bpo[p, Np[p]] = -Ap[p]
    Bd = vif.B.toarray()
    PrecInv = np.linalg.inv(Bd.T @ np.diag(vif.Dinv) @ Bd)
    LRpn = lrp.Smn.T @ np.linalg.inv(vif.lowrank.Sm) @ vif.lowrank.Smn if vif.m else np.zeros((npred, n))
    Kp = LRpn - Bpo @ PrecInv
    Sdi = np.linalg.inv(vif.dense_Sigma_dagger())
    _, W = bern_grad_W(y, b)
    H = Sdi @ np.linalg.solve(np.diag(W) + Sdi, Sdi)
    return mu, Sig + Kp @ H @ Kp.T


def laplace_predict_sbpv(vif: VIF, y, b, Xp, Np, eps, tol: float, max_iter: int = 1000):
    """Latent predictive means (Prop. 3.1) and variances by Alg. 1 (SBPV) at the mode b, the
    variance diagonal version: the deterministic part is the latent variance of Prop. 2.1 /
    App. C.1 with b for y, the stochastic part (1/l) sum_i z8_i o z8_i with, for each row
    eps[i] = (z3 (m), z1 (n), z2 (n)):
        z4 = Sigma_mn^T L_m^{-T} z3 + B^{-1} D^{1/2} z1        ~ N(0, Sigma_dagger)
        z5 = Sigma_dagger^{-1} z4                               ~ N(0, Sigma_dagger^{-1})
        z6 = z5 + W^{1/2} z2                                    ~ N(0, Sigma_dagger^{-1} + W)
        z7 = (Sigma_dagger^{-1} + W)^{-1} z6  (PCG with VIFDU)  ~ N(0, (Sigma_dagger^{-1} + W)^{-1})
        z8 = K_p Sigma_dagger^{-1} z7  (the predictive-mean operator applied to z7).
    Returns (mean, var, per-sample PCG iterations)."""
    n, m = vif.n, vif.m
    mu, var_det = predict_appC(vif, b, Xp, Np)
    _, W = bern_grad_W(y, b)
    pre = VIFDU(vif, W)
    acc = np.zeros(Xp.shape[0])
    its = []
    for e in np.atleast_2d(eps):
        z3, z1, z2 = e[:m], e[m:m + n], e[m + n:m + 2 * n]
        z4 = spla.spsolve_triangular(vif.B.tocsr(), np.sqrt(vif.D) * z1, lower=True)
        if m:
            z4 = z4 + vif.lowrank.Smn.T @ sla.solve_triangular(vif.lowrank.cf[0], z3, lower=True, trans="T")
        z6 = vif.Sigma_dagger_inv(z4) + np.sqrt(W) * z2
        z7, it, _ = pcg(lambda w: W * w + vif.Sigma_dagger_inv(w), pre.apply, z6, tol, max_iter)
        z8, _ = predict_appC(vif, z7, Xp, Np)
        acc += z8 * z8
        its.append(it)
    return mu, var_det + acc / len(its), np.array(its)


def vifla_logdet_dense(vif: VIF, b) -> float:
    """log det(Sigma_dagger W + I) from the dense Sigma_dagger (small n): the exact value
    the SLQ estimate targets."""
    _, W = bern_grad_W(np.zeros_like(b), b)
    S = vif.dense_Sigma_dagger()
    sgn, ld = np.linalg.slogdet(S * W[None, :] + np.eye(vif.n))
    return float(ld)


# ----------------------------------------------------------------------------
# Gradient of the VIF-Laplace likelihood by stochastic trace estimation
# (Sec. 4.1 after Eq. slq_v2, App. B "Gradients", App. D control variate)
# ----------------------------------------------------------------------------
def laplace_param_vector(theta) -> np.ndarray:
    """Parameter order of the VIF-Laplace gradient: (sigma1^2, lambda_1..lambda_k); a latent
    GP has no nugget."""
    return np.concatenate([[theta.variance], np.atleast_1d(theta.lengthscale)])


def laplace_theta_from_vector(theta, v):
    t = theta.copy()
    t.variance = float(v[0])
    t.lengthscale = np.array(v[1:], dtype=np.float64)
    return t


def bern_dW(b):
    """dW_ii/db_i for the Bernoulli-logit W_ii = p(1-p), p = sigmoid(b_i):  p(1-p)(1-2p)."""
    p = 1.0 / (1.0 + np.exp(-b))
    return p * (1.0 - p) * (1.0 - 2.0 * p)


def _perturbed(X, Z, theta, N, rel_step):
    """For each parameter k: (h_k, VIF at theta + h_k e_k, VIF at theta - h_k e_k), N and Z
    fixed (R16)."""
    v0 = laplace_param_vector(theta)
    out = []
    for k in range(v0.size):
        h = rel_step * abs(v0[k])
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        out.append((h, VIF(X, Z, laplace_theta_from_vector(theta, vp), N),
                    VIF(X, Z, laplace_theta_from_vector(theta, vm), N)))
    return out


def vifla_grad_ste(X, Z, theta, N, y, b, eps, tol: float, solve_tol: float, max_iter: int = 1000,
                   rel_step: float = 1e-4):
    """Gradient of L^VIFLA (Eq. log_det_VIFLA) with respect to (sigma1^2, lambda) at the mode b,
    VIFDU form (Eq. pcls1 / slq_v1), assembled as in App. B:

        dL/dth_k = 1/2 b^T Delta_k b + 1/2 dlogdet(Sigma_dagger W + I)/dth_k + (dL/db)^T db/dth_k,
        dlogdet(Sigma_dagger W + I)/dth_k = dlogdet(Sigma_dagger)/dth_k + Tr(H^{-1} Delta_k),
        db/dth_k = -H^{-1} Delta_k b,   dL/db_i = 1/2 Tr(H^{-1} dW/db_i),

    with H = W + Sigma_dagger^{-1} and Delta_k = dSigma_dagger^{-1}/dth_k.  Both traces are
    stochastic trace estimates (Sec. 4.1) from the SLQ probes z_i ~ N(0, P^) (recipe of
    Sec. 4.3): with u_i = H^{-1} z_i (the PCG solves of the SLQ, tolerance `tol`) and
    y_i = P^{-1} z_i,
        Tr(H^{-1} dW/db_j) ~ (1/l) sum_i u_ij dW_jj/db_j y_ij,
        Tr(H^{-1} Delta_k) ~ (1/l) sum_i s_ik,  s_ik = u_i^T Delta_k y_i,
    the latter with the control variate of App. D built from P^ = B^T W B + Sigma_dagger^{-1}:
        c_ik = y_i^T (dP^/dth_k) y_i,  tau_k = Tr(P^{-1} dP^/dth_k) = dlogdet(P^)/dth_k,
        c_opt = sum_i (s_ik - mean s_k)(c_ik - tau_k) / sum_i (c_ik - tau_k)^2,
        T_k = (1/l) sum_i (s_ik - c_opt c_ik) + c_opt tau_k.
    The implicit term is -v^T Delta_k b with v = H^{-1} (dL/db) (PCG, tolerance `solve_tol`).
    Every derivative of a theta-dependent quantity (the bilinear forms x^T Sigma_dagger^{-1} y,
    (B y)^T W (B y), log det Sigma_dagger, log det P^) is a central difference in th_k with step
    rel_step * th_k, holding N, Z, W and b fixed (R16).
    eps: l x (m + 2n) standard normals as in vifla_nll_slq.  Returns a dict with grad, s, c
    (l x q), trace_plain, c_opt, tau, trace (q) and the vectors g = dL/db, v."""
    vif = VIF(X, Z, theta, N)
    n, m = vif.n, vif.m
    _, W = bern_grad_W(y, b)
    pre = VIFDU(vif, W)
    H = lambda w: W * w + vif.Sigma_dagger_inv(w)
    U, Yp = [], []
    for e in np.atleast_2d(eps):
        z = vifdu_sample(vif, W, e[:m], e[m:m + n], e[m + n:m + 2 * n])
        u, _, _, _, _ = pcg_lanczos(H, pre.apply, z, tol, max_iter)
        U.append(u)
        Yp.append(pre.apply(z))
    U, Yp = np.array(U), np.array(Yp)
    ell = U.shape[0]
    g = 0.5 * bern_dW(b) * (U * Yp).mean(axis=0)
    v, _, _ = pcg(H, pre.apply, g, solve_tol, max_iter)

    def forms(vf):
        sdb = vf.Sigma_dagger_inv(b)
        sdy = np.array([vf.Sigma_dagger_inv(yi) for yi in Yp])
        By = np.array([vf.B @ yi for yi in Yp])
        return dict(ldS=vf.logdet(), ldP=vifdu_logdet(vf, W), bb=float(b @ sdb), vb=float(v @ sdb),
                    uy=(U * sdy).sum(axis=1), yy=(Yp * sdy).sum(axis=1), bwb=(By * (W * By)).sum(axis=1))

    q = laplace_param_vector(theta).size
    grad = np.empty(q)
    S = np.empty((ell, q))
    C = np.empty((ell, q))
    tr_plain, c_opt, tau, trace = (np.empty(q) for _ in range(4))
    for k, (h, vp, vm) in enumerate(_perturbed(X, Z, theta, N, rel_step)):
        fp, fm = forms(vp), forms(vm)
        d = {key: (fp[key] - fm[key]) / (2.0 * h) for key in fp}
        S[:, k] = d["uy"]
        C[:, k] = d["bwb"] + d["yy"]
        tau[k] = d["ldP"]
        tr_plain[k] = S[:, k].mean()
        dc = C[:, k] - tau[k]
        den = float(dc @ dc)
        c_opt[k] = float((S[:, k] - tr_plain[k]) @ dc) / den if den > 0 else 0.0
        trace[k] = float((S[:, k] - c_opt[k] * C[:, k]).mean()) + c_opt[k] * tau[k]
        grad[k] = 0.5 * d["bb"] + 0.5 * (d["ldS"] + trace[k]) - d["vb"]
    return dict(grad=grad, s=S, c=C, trace_plain=tr_plain, c_opt=c_opt, tau=tau, trace=trace, g=g, v=v)


def vifla_grad_ste_fitc(X, Z, theta, N, y, b, eps, tol: float, solve_tol: float, max_iter: int = 1000,
                        rel_step: float = 1e-4):
    """The gradient of vifla_grad_ste in the FITC form (Eq. pcls2 / slq_v2, App. D second form):
    with H_F = W^{-1} + Sigma_dagger, log det(Sigma_dagger W + I) = log det W + log det H_F, so

        dL/dth_k = -1/2 a^T dSigma_k a + av^T dSigma_k a + 1/2 Tr(H_F^{-1} dSigma_k),
        dL/db_j  = 1/2 (dW_jj/db_j / W_jj - dW_jj/db_j / W_jj^2 (H_F^{-1})_jj),

    dSigma_k = dSigma_dagger/dth_k, a = Sigma_dagger^{-1} b (so that b^T Delta_k b = -a^T dSigma_k a) and
    av = Sigma_dagger^{-1} v, v = (W + Sigma_dagger^{-1})^{-1} dL/db = W^{-1} H_F^{-1} Sigma_dagger dL/db (CG on
    Eq. pcls2, tolerance `solve_tol`).  The traces are the STE of Sec. 4.1 with the FITC probes
    z_i ~ N(0, P) (App. E.2), u_i = H_F^{-1} z_i (the SLQ's CG solves, tolerance `tol`), y_i = P^{-1} z_i:
        (H_F^{-1})_jj ~ (1/l) sum_i u_ij y_ij,   s_ik = u_i^T dSigma_k y_i,
    with the control variate of App. D: c_ik = y_i^T (dP/dth_k) y_i, tau_k = dlog det P/dth_k
    (P = D_V + Sigma_mn^T Sigma_m^{-1} Sigma_mn, W fixed).  Derivatives in theta are central differences
    (R16).  eps: l x (m + n) (or wider; the first m + n entries are used).  Returns the dict of
    vifla_grad_ste plus dhat (the diagonal estimate)."""
    vif = VIF(X, Z, theta, N)
    n, m = vif.n, vif.m
    _, W = bern_grad_W(y, b)
    pre = FITCPrecond(vif, W)
    HF = lambda w: w / W + Sigma_dagger_matvec(vif, w)
    U, Yp = [], []
    for e in np.atleast_2d(eps):
        z = pre.sample(e[:m], e[m:m + n])
        u, _, _, _, _ = pcg_lanczos(HF, pre.apply, z, tol, max_iter)
        U.append(u)
        Yp.append(pre.apply(z))
    U, Yp = np.array(U), np.array(Yp)
    ell = U.shape[0]
    dW = bern_dW(b)
    dhat = (U * Yp).mean(axis=0)
    g = 0.5 * (dW / W - dW / W ** 2 * dhat)
    sv, _, _ = pcg(HF, pre.apply, Sigma_dagger_matvec(vif, g), solve_tol, max_iter)
    v = sv / W
    a = vif.Sigma_dagger_inv(b)
    av = vif.Sigma_dagger_inv(v)

    def forms(vf):
        Sa = Sigma_dagger_matvec(vf, a)
        SY = np.array([Sigma_dagger_matvec(vf, yi) for yi in Yp])
        pf = FITCPrecond(vf, W)
        if vf.m:
            lr = vf.lowrank
            AY = Yp @ lr.Smn.T                        # rows Sigma_mn y_i
            low = (AY * (Yp @ lr.SinvSmn.T)).sum(axis=1)
        else:
            low = np.zeros(ell)
        return dict(aa=float(a @ Sa), va=float(av @ Sa), uy=(U * SY).sum(axis=1),
                    yPy=(Yp * Yp * pf.DV[None, :]).sum(axis=1) + low, ldP=pf.logdet())

    q = laplace_param_vector(theta).size
    grad = np.empty(q)
    S = np.empty((ell, q))
    C = np.empty((ell, q))
    tr_plain, c_opt, tau, trace = (np.empty(q) for _ in range(4))
    for k, (h, vp, vm) in enumerate(_perturbed(X, Z, theta, N, rel_step)):
        fp, fm = forms(vp), forms(vm)
        d = {key: (fp[key] - fm[key]) / (2.0 * h) for key in fp}
        S[:, k] = d["uy"]
        C[:, k] = d["yPy"]
        tau[k] = d["ldP"]
        tr_plain[k] = S[:, k].mean()
        dc = C[:, k] - tau[k]
        den = float(dc @ dc)
        c_opt[k] = float((S[:, k] - tr_plain[k]) @ dc) / den if den > 0 else 0.0
        trace[k] = float((S[:, k] - c_opt[k] * C[:, k]).mean()) + c_opt[k] * tau[k]
        grad[k] = -0.5 * d["aa"] + d["va"] + 0.5 * trace[k]
    return dict(grad=grad, s=S, c=C, trace_plain=tr_plain, c_opt=c_opt, tau=tau, trace=trace, g=g, v=v,
                dhat=dhat)


def vifla_grad_exact_fitc(X, Z, theta, N, y, b, rel_step: float = 1e-4):
    """vifla_grad_ste_fitc with every trace exact from dense matrices (small n): H_F^{-1} dense and
    dSigma_k the central difference of the dense Sigma_dagger.  Equals vifla_grad_exact (the same
    gradient through Sigma_dagger instead of its inverse)."""
    vif = VIF(X, Z, theta, N)
    _, W = bern_grad_W(y, b)
    Sd = vif.dense_Sigma_dagger()
    HFinv = np.linalg.inv(np.diag(1.0 / W) + Sd)
    dW = bern_dW(b)
    g = 0.5 * (dW / W - dW / W ** 2 * np.diag(HFinv))
    v = (HFinv @ (Sd @ g)) / W
    a = vif.Sigma_dagger_inv(b)
    av = vif.Sigma_dagger_inv(v)
    q = laplace_param_vector(theta).size
    grad, trace = np.empty(q), np.empty(q)
    for k, (h, vp, vm) in enumerate(_perturbed(X, Z, theta, N, rel_step)):
        Dk = (vp.dense_Sigma_dagger() - vm.dense_Sigma_dagger()) / (2.0 * h)
        trace[k] = float(np.sum(HFinv * Dk))
        grad[k] = -0.5 * a @ Dk @ a + av @ Dk @ a + 0.5 * trace[k]
    return dict(grad=grad, trace=trace, dHF=np.diag(HFinv), g=g, v=v)


def dense_Sigma_dagger_inv(vif: VIF) -> np.ndarray:
    """Sigma_dagger^{-1} column by column through the Woodbury form (Sec. 2.2); inverting the dense
    Sigma_dagger of a latent GP (no nugget) loses digits to its conditioning."""
    return np.column_stack([vif.Sigma_dagger_inv(e) for e in np.eye(vif.n)])


def vifla_grad_exact(X, Z, theta, N, y, b, rel_step: float = 1e-4):
    """The gradient of vifla_grad_ste with every trace taken exactly from dense matrices (small n):
    Tr(H^{-1} Delta_k) with Delta_k the central difference of the dense Sigma_dagger^{-1}, and
    dL/db_j = 1/2 (H^{-1})_jj dW_jj/db_j.  The value the stochastic estimate targets."""
    vif = VIF(X, Z, theta, N)
    _, W = bern_grad_W(y, b)
    Hinv = np.linalg.inv(np.diag(W) + dense_Sigma_dagger_inv(vif))
    g = 0.5 * bern_dW(b) * np.diag(Hinv)
    v = Hinv @ g
    q = laplace_param_vector(theta).size
    grad, trace = np.empty(q), np.empty(q)
    for k, (h, vp, vm) in enumerate(_perturbed(X, Z, theta, N, rel_step)):
        Dk = (dense_Sigma_dagger_inv(vp) - dense_Sigma_dagger_inv(vm)) / (2.0 * h)
        dldS = (vp.logdet() - vm.logdet()) / (2.0 * h)
        trace[k] = float(np.sum(Hinv * Dk))
        grad[k] = 0.5 * b @ Dk @ b + 0.5 * (dldS + trace[k]) - v @ Dk @ b
    return dict(grad=grad, trace=trace, g=g, v=v)


def vifla_nll_exact(X, Z, theta, N, y) -> float:
    """L^VIFLA (Eq. log_det_VIFLA) with the exact (dense Newton) mode and the dense
    log det(Sigma_dagger W + I) (small n)."""
    vif = VIF(X, Z, theta, N)
    b, _, _ = laplace_mode(vif, y, dense=True, psi_tol=1e-14)
    return -bern_loglik(y, b) + 0.5 * float(b @ vif.Sigma_dagger_inv(b)) + 0.5 * vifla_logdet_dense(vif, b)


# ----------------------------------------------------------------------------
# Gradient of the negative log-likelihood (Sec. 2.2)
# ----------------------------------------------------------------------------
def theta_vector(theta) -> np.ndarray:
    """Parameter order of the gradient: (sigma1^2, lambda_1..lambda_k, sigma^2)."""
    return np.concatenate([[theta.variance], np.atleast_1d(theta.lengthscale), [theta.nugget]])


def theta_from_vector(theta, v):
    t = theta.copy()
    k = np.atleast_1d(theta.lengthscale).size
    t.variance = float(v[0])
    t.lengthscale = np.array(v[1:1 + k], dtype=np.float64)
    t.nugget = float(v[1 + k])
    return t


def vif_nll_grad_fd(X, Z, theta, N, y, rel_step=1e-4):
    """Central differences of the VIF NLL with N and Z held fixed (R11): step
    h_k = rel_step * theta_k in each parameter."""
    v0 = theta_vector(theta)
    g = np.empty_like(v0)
    for k in range(v0.size):
        h = rel_step * abs(v0[k]) if v0[k] != 0 else rel_step
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        g[k] = (vif_nll(X, Z, theta_from_vector(theta, vp), N, y)
                - vif_nll(X, Z, theta_from_vector(theta, vm), N, y)) / (2 * h)
    return g


def dcov_of_r(r, kind, variance):
    """dc/dr for the kernels of cov_of_r."""
    if kind == 0:
        return -variance * np.exp(-r)
    if kind == 1:
        return -3.0 * variance * r * np.exp(-SQRT3 * r)
    if kind == 2:
        return -(5.0 / 3.0) * variance * r * (1.0 + SQRT5 * r) * np.exp(-SQRT5 * r)
    return -variance * r * np.exp(-0.5 * r * r)


def exact_gp_grad(X, y, theta) -> np.ndarray:
    """Analytic gradient of the exact GP NLL (Sec. 2 first display):
    dL/dth = 1/2 tr(Sigma~^{-1} dSigma~) - 1/2 alpha^T dSigma~ alpha, alpha = Sigma~^{-1} y,
    for (sigma1^2, lambda (one or per dimension), sigma^2)."""
    S = exact_cov(X, theta)
    L = np.linalg.cholesky(S)
    Sinv = sla.cho_solve((L, True), np.eye(len(y)))
    alpha = Sinv @ y
    ls = np.atleast_1d(theta.lengthscale)
    Xs = scaled(X, theta)
    r = dist(Xs, Xs)
    K = cov_of_r(r, theta.kind, theta.variance)
    dK = dcov_of_r(r, theta.kind, theta.variance)
    mats = [K / theta.variance]
    with np.errstate(divide="ignore", invalid="ignore"):
        if ls.size == 1:
            mats.append(np.where(r > 0, -dK * r / ls[0], 0.0))
        else:
            for k in range(ls.size):
                dk2 = (X[:, None, k] - X[None, :, k]) ** 2 / ls[k] ** 3
                mats.append(np.where(r > 0, -dK * dk2 / r, 0.0))
    mats.append(np.eye(len(y)))
    return np.array([0.5 * np.sum(Sinv * M) - 0.5 * alpha @ M @ alpha for M in mats])



def dcov(X1, X2, theta) -> list:
    """Derivatives of the cross covariance cov(X1, X2) (no nugget) with respect to
    (sigma1^2, lambda_1..lambda_k, sigma^2), in the order of theta_vector."""
    ls = np.atleast_1d(theta.lengthscale)
    r = dist(scaled(X1, theta), scaled(X2, theta))
    K = cov_of_r(r, theta.kind, theta.variance)
    dK = dcov_of_r(r, theta.kind, theta.variance)
    mats = [K / theta.variance]
    with np.errstate(divide="ignore", invalid="ignore"):
        if ls.size == 1:
            mats.append(np.where(r > 0, -dK * r / ls[0], 0.0))     # dr/dlambda = -r / lambda
        else:
            for t in range(ls.size):
                dk2 = (X1[:, None, t] - X2[None, :, t]) ** 2 / ls[t] ** 3
                mats.append(np.where(r > 0, -dK * dk2 / r, 0.0))
    mats.append(np.zeros_like(K))
    return mats


def vif_nll_grad(X, Z, theta, N, y) -> np.ndarray:
    """Analytic gradient of the VIF NLL in (sigma1^2, lambda_1..lambda_k, sigma^2) with N and Z
    fixed, as Sec. 2.2 writes it: 1/2 Tr(Sigma~_dagger^{-1} dSigma~_dagger) - 1/2 alpha^T
    dSigma~_dagger alpha (alpha = Sigma~_dagger^{-1} y), dSigma~_dagger = dSigma~^s + dSigma^l with
      dSigma^l = dSigma_mn^T Sigma_m^{-1} Sigma_mn + Sigma_mn^T Sigma_m^{-1} dSigma_mn
                 - Sigma_mn^T Sigma_m^{-1} dSigma_m Sigma_m^{-1} Sigma_mn,
      dSigma~^s = B^{-1} dD B^{-T} - B^{-1} dB B^{-1} D B^{-T} - B^{-1} D B^{-T} dB^T B^{-T},
    and dB, dD per point from App. A (D_i = c~_ii - A_i c_Ni differentiated by the product
    rule, reading R17).  Sigma_m carries the R7 jitter eps sigma1^2 (derivative Sigma_m /
    sigma1^2 in sigma1^2); the residual blocks' diagonal carries the nugget.  Dense n x n
    algebra: small n only."""
    n, mv = N.shape
    m = Z.shape[0]
    vif = VIF(X, Z, theta, N)
    q_par = theta_vector(theta).size
    Kx = dcov(X, X, theta)
    tdiag = residual_diag(theta)
    dtdiag = np.zeros(q_par)
    if theta.nugget > 0:
        dtdiag[-1] = 1.0
    else:
        dtdiag[0] = tdiag / theta.variance
    if m:
        Smn = vif.lowrank.Smn
        W = vif.lowrank.SinvSmn                                   # Sigma_m^{-1} Sigma_mn
        dSmn = dcov(Z, X, theta)
        dSm = dcov(Z, Z, theta)
        dSm[0] = sigma_m(Z, theta) / theta.variance               # jitter scales with sigma1^2
        dLR = [dSmn[k].T @ W + W.T @ dSmn[k] - W.T @ dSm[k] @ W for k in range(q_par)]
        LR = Smn.T @ W
    else:
        dLR = [np.zeros((n, n)) for _ in range(q_par)]
        LR = np.zeros((n, n))
    S_full = cov(X, X, theta)
    Binv = np.linalg.inv(vif.B.toarray())
    Ss = Binv @ np.diag(vif.D) @ Binv.T
    Sdag = vif.dense_Sigma_dagger()
    cf = sla.cho_factor(Sdag, lower=True)
    Sdinv = sla.cho_solve(cf, np.eye(n))
    alpha = Sdinv @ y
    g = np.empty(q_par)
    for k in range(q_par):
        dB = np.zeros((n, n))
        dD = np.zeros(n)
        for i in range(n):
            Ni = N[i][N[i] >= 0]
            c_ii = theta.variance + tdiag - LR[i, i]
            dc_ii = Kx[k][i, i] + dtdiag[k] - dLR[k][i, i]
            if len(Ni) == 0:
                dD[i] = dc_ii
                continue
            Mat = S_full[np.ix_(Ni, Ni)] + tdiag * np.eye(len(Ni)) - LR[np.ix_(Ni, Ni)]
            dMat = Kx[k][np.ix_(Ni, Ni)] + dtdiag[k] * np.eye(len(Ni)) - dLR[k][np.ix_(Ni, Ni)]
            c_iN = S_full[i, Ni] - LR[i, Ni]
            dc_iN = Kx[k][i, Ni] - dLR[k][i, Ni]
            Ai = np.linalg.solve(Mat, c_iN)
            dAi = np.linalg.solve(Mat, dc_iN - dMat @ Ai)
            dB[i, Ni] = -dAi
            dD[i] = dc_ii - dAi @ c_iN - Ai @ dc_iN
        dSs = Binv @ np.diag(dD) @ Binv.T - Binv @ dB @ Ss - Ss @ dB.T @ Binv.T
        dS = dSs + dLR[k]
        g[k] = 0.5 * np.sum(Sdinv * dS) - 0.5 * alpha @ dS @ alpha
    return g