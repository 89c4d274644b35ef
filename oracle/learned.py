"""Learned row proposal for skeletonization, in plain FP64 (test infrastructure only).

The paper samples the block K_{[1:N] alpha} "using nearest-neighbor information"
(Sec. II-B).  This project adds a learned proposal: a small MLP scores candidate
rows of a node and the best-scored rows form the sample.  Everything here is the
reference the GPU kernels are checked against; none of it is in the paper.

* ``candidate_features``: 8 features per (node, candidate row) from the node's
  column subset (at most 32 evenly spaced columns of the ID), the candidate's kNN
  hit count, the node's level and size.
* ``mlp_forward`` / ``mlp_backward``: a 3-layer MLP F -> 128 -> 128 -> 1 with ReLU,
  loss = mean squared error.
* ``adam_step``: Adam (Kingma & Ba 2015) with bias correction.
* ``ridge_leverage``: label of a row b of a block B: b^T (B^T B + mu I)^{-1} b, the
  ridge leverage score, large for rows that carry the block's dominant directions.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

from .kernel import gaussian_kernel

NFEAT = 8
WIDTH = 128
COL_SUBSET = 32


def column_subset(cols: np.ndarray) -> np.ndarray:
    """At most 32 evenly spaced entries of the ID's column list: cols[floor(j n_c / k)]."""
    nc = cols.size
    k = min(COL_SUBSET, nc)
    return cols[(np.arange(k) * nc) // k]


def candidate_features(Xp: np.ndarray, cand: np.ndarray, hits: np.ndarray, cols: np.ndarray,
                       h: float, level: int, L: int, n: int, N: int, kappa: int) -> np.ndarray:
    """Features of candidate rows (permuted positions) for a node with ID columns ``cols``.

    f0 log(1 + hits) / log(1 + kappa)        f4 level / L
    f1 ||x_c - mu|| / h                       f5 log2(n) / log2(N)
    f2 max_j K(x_c, y_j)                      f6 ||x_c - mu|| / r  (r: largest ||y_j - mu||)
    f3 mean_j K(x_c, y_j)                     f7 0
    with y_j the column subset and mu its mean.
    """
    Y = Xp[column_subset(cols)]
    mu = Y.mean(axis=0)
    r = float(np.sqrt(((Y - mu) ** 2).sum(axis=1)).max())
    Xc = Xp[cand]
    dmu = np.sqrt(((Xc - mu) ** 2).sum(axis=1))
    K = gaussian_kernel(Xc, Y, h)
    F = np.zeros((cand.size, NFEAT))
    F[:, 0] = np.log1p(hits) / math.log1p(kappa)
    F[:, 1] = dmu / h
    F[:, 2] = K.max(axis=1)
    F[:, 3] = K.mean(axis=1)
    F[:, 4] = level / max(L, 1)
    F[:, 5] = math.log2(n) / math.log2(N)
    F[:, 6] = np.minimum(dmu / max(r, 1e-30), 1e3)
    return F


Params = Dict[str, np.ndarray]


def mlp_init(seed: int = 0, fin: int = NFEAT, width: int = WIDTH) -> Params:
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    lim1 = math.sqrt(6.0 / fin)
    lim2 = math.sqrt(6.0 / width)
    return {
        "W1": rng.uniform(-lim1, lim1, (width, fin)), "b1": np.zeros(width),
        "W2": rng.uniform(-lim2, lim2, (width, width)), "b2": np.zeros(width),
        "w3": rng.uniform(-lim2, lim2, width), "b3": np.zeros(1),
    }


def mlp_forward(p: Params, X: np.ndarray) -> Tuple[np.ndarray, tuple]:
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for every row x of X."""
    A1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(A2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, (X, H1, H2)


def mse_loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def mlp_backward(p: Params, cache: tuple, y: np.ndarray, t: np.ndarray) -> Params:
    """Gradients of the mean squared error with respect to every parameter."""
    X, H1, H2 = cache
    B = y.size
    dy = 2.0 * (y - t) / B
    g = {"w3": H2.T @ dy, "b3": np.array([dy.sum()])}
    dA2 = np.outer(dy, p["w3"]) * (H2 > 0)
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(axis=0)
    dA1 = (dA2 @ p["W2"]) * (H1 > 0)
    g["W1"] = dA1.T @ X
    g["b1"] = dA1.sum(axis=0)
    return g


def adam_step(p: Params, g: Params, state: dict, lr: float = 1e-3, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; ``state`` holds t, m and v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)


def ridge_leverage(B_rows: np.ndarray, G: np.ndarray, mu: float) -> np.ndarray:
    """l_i = b_i^T (G + mu I)^{-1} b_i for the rows b_i of B_rows, G a Gram matrix."""
    M = np.linalg.solve(G + mu * np.eye(G.shape[0]), B_rows.T)
    return np.einsum("ij,ji->i", B_rows, M)
