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


# ---------------------------------------------------------------------------
# Learned sampling inside skeletonization.  For a non-root node alpha owning the
# permuted positions [o, o + n) of a problem of N points (complement size N - n) with
# n_samp = min(samp_factor s_max, N - n) rows to sample:
#
# * candidates (n_samp < N - n only): n_cand = min(cand_factor n_samp, N - n) rows.
#   First, at most n_cand // 2 of the node's kNN candidates in the plain sampling order
#   (hits descending, position ascending) with their hit counts; then uniform draws
#   without replacement from the complement on the node's LEARN stream until n_cand
#   rows are held (their hits feature is 0).
# * selection: the n_samp candidates of largest key (ties to the lower position),
#   returned in ascending position order; the key is the MLP score plus temp times a
#   Gumbel draw of the node's GUMBEL stream (temp = 0: the score itself), which makes
#   the selection a sample without replacement with probabilities ~ exp(score / temp).
# * row strata: the complement of alpha splits into its sibling (whose rows use alpha's
#   skeletons directly, and hold most of the kernel mass) and the points outside the
#   parent.  A stratified draw of `count` rows takes c_s = count // 2 rows uniformly with
#   replacement from the sibling and the rest from outside the parent (all from the
#   sibling when the parent is the root); a row of stratum t weighs |t| / (its draws).
# * judge: NHOLD stratified rows H (weights w) on the node's HOLD stream; the held-out
#   ID error of a skeleton set S with interpolation matrix P is
#   sum_h w_h ||K(h, cols) - K(h, S) P||^2 / sum_h w_h ||K(h, cols)||^2; the learned ID
#   is kept when its error is <= the plain sample's, otherwise the node falls back.
# * labels (training): NGRAM stratified rows on the GRAM stream give
#   G = B^T diag(w) B, B = K(gram rows, cols), mu = tol^2 trace(G) (tol = 1e-6 for fixed
#   ranks); the label of candidate c is the ridge leverage b_c^T (G + mu I)^{-1} b_c with
#   b_c = K(x_c, cols), and the training target its logarithm standardized over the
#   node's candidates.
# Each auxiliary stream is SplitMix64 with state s0 = splitmix64(splitmix64(seed ^ salt)
# ^ uid) and draw q equal to splitmix64(s0 + q gamma); a draw r is mapped to the sibling
# position sib_o + r mod |sib|, or to j = r mod (N - |parent|) taken as j (j < parent
# offset) or j + |parent|; the candidates' uniform part maps j = r mod (N - n) around
# alpha itself, as the plain uniform fill does.
# ---------------------------------------------------------------------------
from .sampling import GAMMA, MASK64, splitmix64  # noqa: E402

LEARN_SALT = 0x4C4541524E
HOLD_SALT = 0x484F4C44
GRAM_SALT = 0x4752414D
GUMBEL_SALT = 0x47554D42
NHOLD = 64
NGRAM = 4096
CAND_FACTOR = 8


def stream_state(seed: int, salt: int, uid: int) -> int:
    return splitmix64(splitmix64((seed ^ salt) & MASK64) ^ uid)


def stream_position(s0: int, q: int, o: int, n: int, N: int) -> int:
    j = splitmix64((s0 + q * GAMMA) & MASK64) % (N - n)
    return j if j < o else j + n


def knn_ranked(knn_pos: np.ndarray, o: int, n: int):
    """The node's kNN candidates outside [o, o + n) with hit counts, hits descending then
    position ascending (the plain sampling order)."""
    cand = knn_pos.ravel()
    cand = cand[(cand < o) | (cand >= o + n)]
    if cand.size == 0:
        return np.empty(0, dtype=np.int64), np.empty(0, dtype=np.int64)
    vals, counts = np.unique(cand, return_counts=True)
    order = np.lexsort((vals, -counts))
    return vals[order].astype(np.int64), counts[order].astype(np.int64)


def learned_candidates(knn_pos: np.ndarray, o: int, n: int, N: int, n_samp: int, seed: int,
                       uid: int, cand_factor: int = CAND_FACTOR):
    """(candidate positions, hit counts) of the node, kNN part first, then the draws."""
    comp = N - n
    n_samp = min(n_samp, comp)
    n_cand = min(cand_factor * n_samp, comp)
    vals, counts = knn_ranked(knn_pos, o, n)
    k = min(vals.size, n_cand // 2)
    cand = [int(v) for v in vals[:k]]
    hits = [int(c) for c in counts[:k]]
    taken = set(cand)
    s0 = stream_state(seed, LEARN_SALT, uid)
    q = 0
    while len(cand) < n_cand:
        pos = stream_position(s0, q, o, n, N)
        if pos not in taken:
            taken.add(pos)
            cand.append(pos)
            hits.append(0)
        q += 1
    return np.array(cand, dtype=np.int64), np.array(hits, dtype=np.int64)


def uniform_rows(o: int, n: int, N: int, count: int, seed: int, salt: int, uid: int) -> np.ndarray:
    """``count`` positions of the complement drawn with replacement on a node stream."""
    s0 = stream_state(seed, salt, uid)
    return np.array([stream_position(s0, q, o, n, N) for q in range(count)], dtype=np.int64)


def stratified_rows(sib_o: int, sib_n: int, par_o: int, par_n: int, N: int, count: int,
                    seed: int, salt: int, uid: int):
    """(positions, weights) of a stratified draw: sibling rows first, then rows outside
    the parent."""
    s0 = stream_state(seed, salt, uid)
    far = N - par_n
    cs = count if far == 0 else count // 2
    rows = np.empty(count, dtype=np.int64)
    wts = np.empty(count)
    for q in range(count):
        r = splitmix64((s0 + q * GAMMA) & MASK64)
        if q < cs:
            rows[q] = sib_o + r % sib_n
            wts[q] = sib_n / cs
        else:
            j = r % far
            rows[q] = j if j < par_o else j + par_n
            wts[q] = far / (count - cs)
    return rows, wts


def gumbel_keys(scores: np.ndarray, seed: int, uid: int, temp: float) -> np.ndarray:
    """scores + temp * g with Gumbel draws g_c = -log(-log(u_c)), u_c = ((r_c >> 11) + 1/2)
    2^-53 from draw c of the node's GUMBEL stream, rounded to FP32.  The top n of the
    keys are a sample without replacement with probabilities ~ exp(score / temp)."""
    s0 = stream_state(seed, GUMBEL_SALT, uid)
    u = np.array([((splitmix64((s0 + c * GAMMA) & MASK64) >> 11) + 0.5) * 2.0 ** -53
                  for c in range(len(scores))])
    return (np.asarray(scores, dtype=np.float64) + temp * -np.log(-np.log(u))).astype(np.float32)


def select_top(scores: np.ndarray, cand: np.ndarray, n_samp: int) -> np.ndarray:
    """The n_samp candidates of largest score (ties: lower position first), ascending."""
    order = np.lexsort((cand, -np.asarray(scores, dtype=np.float64)))
    return np.sort(cand[order[:n_samp]])


def heldout_error(Xp: np.ndarray, H: np.ndarray, wts: np.ndarray, cols: np.ndarray,
                  skel: np.ndarray, P: np.ndarray, h: float) -> float:
    """sum_h w_h ||K(h, cols) - K(h, skel) P||^2 / sum_h w_h ||K(h, cols)||^2."""
    A = gaussian_kernel(Xp[H], Xp[cols], h)
    E = A - gaussian_kernel(Xp[H], Xp[skel], h) @ P
    den = float(wts @ (A * A).sum(axis=1))
    return float(wts @ (E * E).sum(axis=1)) / den if den > 0 else 0.0


def leverage_labels(Xp: np.ndarray, cand: np.ndarray, cols: np.ndarray, gram: np.ndarray,
                    wts: np.ndarray, h: float, tol: float):
    """(ridge leverage of each candidate against G = B^T diag(w) B, standardized log)."""
    B = gaussian_kernel(Xp[gram], Xp[cols], h)
    G = B.T @ (wts[:, None] * B)
    t = tol if tol > 0 else 1e-6
    mu = t * t * float(np.trace(G))
    lev = ridge_leverage(gaussian_kernel(Xp[cand], Xp[cols], h), G, mu)
    z = np.log(np.maximum(lev, 1e-300))
    sd = z.std()
    target = (z - z.mean()) / sd if sd > 1e-12 else np.zeros_like(z)
    return lev, target
