"""ASKIT's hierarchical approximation K~ = D + UV (Sec. II-B) in plain FP64.

Part of the oracle (test infrastructure only).

* ``skeletonize``: the w-independent part of Skeletonize (Sec. II-B), bottom-up.
  Leaves take the ID of K(samples, leaf points); an internal node alpha takes the
  ID of K(samples, [l~ r~]) over its children's skeletons, so its skeletons are a
  subset of theirs and only the nested P_{a~[l~ r~]} (s_a x (s_l + s_r)) is kept.
  The root is not skeletonized (it has no sibling).
* ``full_P``: P_{a~ a} from eq. (innerid), P_{a~[l~ r~]} blockdiag(P_{l~ l}, P_{r~ r}),
  formed by matrix products.
* ``dense_Ktilde``: the definition of K~ with the i-not-in-alpha separation
  (eqs. offdiag-askit, uv-askit): K~_aa = blockdiag(K~_ll, K~_rr) +
  [[0, K_{l r~} P_{r~ r}], [K_{r l~} P_{l~ l}, 0]], and K~_aa = K_aa at a leaf.
* ``matvec``: the fast MatVec u = (lambda I + K~) w by Skeletonize (its steps that
  depend on w: w~ = P w up the tree) and Evaluate (u_i = K_{i a~} w~_a for every
  node a separated from i, exact leaf interactions otherwise).

All quantities live in the tree's permuted order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Tuple

import numpy as np

from .kernel import kernel_matrix
from .linalg import cpqr_id
from .sampling import sample_rows
from .tree import Tree

Node = Tuple[int, int]


@dataclass
class Skeletons:
    tree: Tree
    Xp: np.ndarray                      # points in permuted order
    h: float
    samp: Dict[Node, np.ndarray] = field(default_factory=dict)
    cols: Dict[Node, np.ndarray] = field(default_factory=dict)
    piv: Dict[Node, np.ndarray] = field(default_factory=dict)
    P: Dict[Node, np.ndarray] = field(default_factory=dict)     # nested P (s x n_cols)
    skel: Dict[Node, np.ndarray] = field(default_factory=dict)  # permuted positions, pivot order
    margin: Dict[Node, float] = field(default_factory=dict)

    def rank(self, node: Node) -> int:
        return int(self.skel[node].size)


def skeletonize(X: np.ndarray, tree: Tree, knn: np.ndarray, h: float, s_max: int,
                tol: float, samp_factor: int = 2, seed: int = 0) -> Skeletons:
    """Skeletons and nested P for every non-root node, leaves first (Sec. II-B)."""
    Xp = np.asarray(X, dtype=np.float64)[tree.perm]
    knn_pos = tree.iperm[knn[tree.perm]]          # row = permuted position, entries = positions
    sk = Skeletons(tree=tree, Xp=Xp, h=h)
    N = tree.N
    for l in range(tree.L, 0, -1):
        for i in range(1 << l):
            o, e = tree.node_range(l, i)
            n = e - o
            samp = sample_rows(knn_pos[o:e], o, n, N, samp_factor * s_max, seed, (1 << l) + i)
            if l == tree.L:
                cols = np.arange(o, e, dtype=np.int64)
            else:
                cols = np.concatenate([sk.skel[(l + 1, 2 * i)], sk.skel[(l + 1, 2 * i + 1)]])
            A = kernel_matrix(Xp[samp], Xp[cols], h)
            piv, s, P, _, margin = cpqr_id(A, s_max, tol)
            node = (l, i)
            sk.samp[node] = samp
            sk.cols[node] = cols
            sk.piv[node] = piv
            sk.P[node] = P
            sk.skel[node] = cols[piv[:s]]
            sk.margin[node] = margin
    return sk


def full_P(sk: Skeletons, node: Node, cache: Dict[Node, np.ndarray] = None) -> np.ndarray:
    """P_{a~ a} (s_a x |a|) by eq. (innerid); the leaf P is the ID's own."""
    if cache is not None and node in cache:
        return cache[node]
    l, i = node
    if l == sk.tree.L:
        out = sk.P[node]
    else:
        Pl = full_P(sk, (l + 1, 2 * i), cache)
        Pr = full_P(sk, (l + 1, 2 * i + 1), cache)
        sl, nl = Pl.shape
        sr, nr = Pr.shape
        B = np.zeros((sl + sr, nl + nr))
        B[:sl, :nl] = Pl
        B[sl:, nl:] = Pr
        out = sk.P[node] @ B
    if cache is not None:
        cache[node] = out
    return out


def dense_Ktilde(sk: Skeletons) -> np.ndarray:
    """K~ assembled densely in permuted order from its recursive definition."""
    tree, Xp, h = sk.tree, sk.Xp, sk.h
    cache: Dict[Node, np.ndarray] = {}

    def block(l: int, i: int) -> np.ndarray:
        o, e = tree.node_range(l, i)
        if l == tree.L:
            return kernel_matrix(Xp[o:e], Xp[o:e], h)
        left, right = (l + 1, 2 * i), (l + 1, 2 * i + 1)
        ol, el = tree.node_range(*left)
        orr, er = tree.node_range(*right)
        Kll = block(*left)
        Krr = block(*right)
        Klr = kernel_matrix(Xp[ol:el], Xp[sk.skel[right]], h) @ full_P(sk, right, cache)
        Krl = kernel_matrix(Xp[orr:er], Xp[sk.skel[left]], h) @ full_P(sk, left, cache)
        return np.block([[Kll, Klr], [Krl, Krr]])

    return block(0, 0)


def matvec(sk: Skeletons, lam: float, w: np.ndarray) -> np.ndarray:
    """u = (lambda I + K~) w, permuted order, by Skeletonize + Evaluate (Sec. II-B)."""
    tree, Xp, h = sk.tree, sk.Xp, sk.h
    w = np.asarray(w, dtype=np.float64)
    vec = w.ndim == 1
    W = w[:, None] if vec else w
    wt: Dict[Node, np.ndarray] = {}
    for l in range(tree.L, 0, -1):                       # Skeletonize: w~ = P w upward
        for i in range(1 << l):
            o, e = tree.node_range(l, i)
            if l == tree.L:
                wt[(l, i)] = sk.P[(l, i)] @ W[o:e]
            else:
                wt[(l, i)] = sk.P[(l, i)] @ np.vstack([wt[(l + 1, 2 * i)], wt[(l + 1, 2 * i + 1)]])
    U = lam * W.copy()
    for l in range(tree.L):                              # Evaluate: separated siblings
        for i in range(1 << l):
            left, right = (l + 1, 2 * i), (l + 1, 2 * i + 1)
            ol, el = tree.node_range(*left)
            orr, er = tree.node_range(*right)
            U[ol:el] += kernel_matrix(Xp[ol:el], Xp[sk.skel[right]], h) @ wt[right]
            U[orr:er] += kernel_matrix(Xp[orr:er], Xp[sk.skel[left]], h) @ wt[left]
    for i in range(1 << tree.L):                         # Evaluate: leaf self-interaction
        o, e = tree.node_range(tree.L, i)
        U[o:e] += kernel_matrix(Xp[o:e], Xp[o:e], h) @ W[o:e]
    return U[:, 0] if vec else U
