"""FP64 CPU oracle of the learned diagonal correction of the VIFDU preconditioner.

TEST INFRASTRUCTURE ONLY (see vif_oracle).  The paper has no learned part; this
module states, in plain numpy, what the CUDA network computes:

  features f_i (10 per point, from the Laplace weight W, the residual Vecchia
  factors A_i, D_i of the current Newton iterate and the residual correlations of
  each point with its neighbours) -> h1 = tanh(W1 f + b1) ->
  h2 = tanh(W2 h1 + b2) -> o = w3 . h2 + b3 -> c_i = 4 tanh(o / 4),

and the preconditioner uses W'_i = W_i exp(c_i) in P = B^T W' B + Sigma_dagger^{-1}.
Parameters are packed as W1 (64x10, row-major), b1 (64), W2 (64x64), b2 (64), w3 (64), b3 (1).

The training loss is the Hutchinson estimate of ||P^{-1} A - I||_F^2 with
A = W + Sigma_dagger^{-1}: L = mean_k ||P^{-1} A z_k - z_k||^2 over Rademacher z_k,
whose gradient with respect to d = W' is
  dL/dd_j = -2 (B P^{-1} r)_j (B u)_j,  u = P^{-1} A z, r = u - z,
because dP/dd_j = b_j b_j^T with b_j the j-th row of B.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 10, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(p: np.ndarray):
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    w3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Correction c for feature rows F (n x 10)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(F @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ w3 + b3
    return 4.0 * np.tanh(o / 4.0)


def backward(p: np.ndarray, F: np.ndarray, gc: np.ndarray) -> np.ndarray:
    """Gradient of sum_i gc_i c_i with respect to the packed parameters."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(F @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ w3 + b3
    do = gc * (1.0 - np.tanh(o / 4.0) ** 2)
    dw3 = h2.T @ do
    db3 = do.sum()
    da2 = (do[:, None] * w3[None, :]) * (1.0 - h2 ** 2)
    dW2 = da2.T @ h1
    db2 = da2.sum(0)
    da1 = (da2 @ W2) * (1.0 - h1 ** 2)
    dW1 = da1.T @ F
    db1 = da1.sum(0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])


def features(W, D, Acoef, N, mv: int, rho=None) -> np.ndarray:
    """Per-point network inputs (each a fixed affine map of a local quantity):
      0 log W_i            1 log D_i             2 log(1 + W_i D_i)
      3 |N(i)| / m_v       4 sum_k A_i[k]^2      5 sum over the points j that condition on i
                                                   of A_j[k]^2
      6 log(mean_{k} W_{N_k(i)} / W_i)           7 log(1 + sum_{j: N_k(j)=i} W_j A_j[k]^2 / W_i)
      8 max_k |rho(i, N_k(i))|                   9 mean_k |rho(i, N_k(i))|
    with rho (n x 2: the largest and the mean) from vif_oracle.residual_neighbor_corr.
    """
    n = W.shape[0]
    F = np.zeros((n, NIN))
    q = (N >= 0).sum(1) if mv > 0 else np.zeros(n, dtype=int)
    s_own = (Acoef ** 2).sum(1) if mv > 0 else np.zeros(n)
    s_ch = np.zeros(n)
    s_chw = np.zeros(n)
    mW = np.zeros(n)
    for i in range(n):
        for k in range(mv):
            j = N[i, k]
            if j >= 0:
                s_ch[j] += Acoef[i, k] ** 2
                s_chw[j] += W[i] * Acoef[i, k] ** 2
                mW[i] += W[j]
    F[:, 0] = (np.log(W) + 3.0) * 0.5
    F[:, 1] = (np.log(D) + 3.0) * 0.5
    F[:, 2] = np.log1p(W * D)
    F[:, 3] = q / max(mv, 1)
    F[:, 4] = s_own
    F[:, 5] = s_ch
    F[:, 6] = np.where(q > 0, np.log(np.where(q > 0, mW / np.maximum(q, 1), 1.0) / W), 0.0)
    F[:, 7] = np.log1p(s_chw / W)
    if rho is not None:
        F[:, 8] = rho[:, 0]
        F[:, 9] = rho[:, 1]
    return F


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform hidden layers, zero output layer (c = 0: the plain preconditioner)."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (NH, NIN)) * np.sqrt(6.0 / (NIN + NH))
    W2 = rng.uniform(-1, 1, (NH, NH)) * np.sqrt(6.0 / (2 * NH))
    return np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), np.zeros(NH), [0.0]])
