"""kNN-separated ASKIT: the near-field correction S of eq. (askit), K ~ K~ + S.

Part of the oracle (test infrastructure only).

Sec. II-B gives ASKIT a second separation rule: a target i is separated from a node
alpha only when none of i's nearest neighbours lies in alpha.  The paper keeps the
hierarchical matrix of eq. (offdiag-askit) and, for a target i whose nearest
neighbours reach into a node alpha that the first rule (i not in alpha) evaluates
through its skeletons, replaces that skeleton evaluation u_i += K_{i a~} w~_a of the
Evaluate step by the exact u_i += K_{i a} w_a.  Reading taken here: the nodes concerned
are the ones the Evaluate step reaches for i under the first rule, i.e. the siblings of
the ancestors of i's leaf (one per level); such a node is evaluated exactly over all its
points when it holds at least one of i's kappa nearest neighbours (i itself is not in
its own list).  The matrix applied is then lambda I + K~ + S with
S_{i a} = K_{i a} - K_{i a~} P_{a~ a} on those (i, alpha) pairs and zero elsewhere;
S = 0 when every neighbour list stays inside its point's leaf.

* ``interaction_node(tree, p, q)``: the node of p's list that contains position q, or
  None when p and q share a leaf.
* ``matvec_knn``: u = (lambda I + K~ + S) w by Skeletonize and the Evaluate recursion
  MatVec(i, alpha) with the replaced skeleton evaluation, target by target.
* ``dense_Ktilde_knn``: the same matrix entry by entry from its definition: K_ij when j
  shares i's leaf or lies in a node of i's list holding a neighbour of i, K~_ij
  (``askit.dense_Ktilde``) elsewhere.

All quantities live in the tree's permuted order; ``knn_pos`` holds, per position, the
positions of its nearest neighbours.
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from .askit import Node, Skeletons, dense_Ktilde, full_P
from .kernel import kernel_matrix
from .tree import Tree


def interaction_node(tree: Tree, p: int, q: int) -> Optional[Node]:
    """The sibling of an ancestor of p's leaf that contains q (None: same leaf)."""
    l, i = 0, 0
    while l < tree.L:
        lo, hi = tree.node_range(l + 1, 2 * i)
        cp = 2 * i if lo <= p < hi else 2 * i + 1
        cq = 2 * i if lo <= q < hi else 2 * i + 1
        if cp != cq:
            return (l + 1, cq)
        l, i = l + 1, cp
    return None


def near_nodes(tree: Tree, p: int, knn_pos: np.ndarray) -> set:
    """Nodes of p's list holding at least one of p's nearest neighbours."""
    out = set()
    for q in np.asarray(knn_pos[p]).ravel():
        a = interaction_node(tree, p, int(q))
        if a is not None:
            out.add(a)
    return out


def matvec_knn(sk: Skeletons, lam: float, w: np.ndarray, knn_pos: np.ndarray) -> np.ndarray:
    """u = (lambda I + K~ + S) w in permuted order (Skeletonize, then Evaluate per target
    with the exact evaluation of the nodes that hold a neighbour of the target)."""
    tree, Xp, h = sk.tree, sk.Xp, sk.h
    w = np.asarray(w, dtype=np.float64)
    vec = w.ndim == 1
    W = w[:, None] if vec else w
    wt: Dict[Node, np.ndarray] = {}
    for l in range(tree.L, 0, -1):                       # Skeletonize: w~ = P w upward
        for i in range(1 << l):
            if l == tree.L:
                o, e = tree.node_range(l, i)
                wt[(l, i)] = sk.P[(l, i)] @ W[o:e]
            else:
                wt[(l, i)] = sk.P[(l, i)] @ np.vstack([wt[(l + 1, 2 * i)], wt[(l + 1, 2 * i + 1)]])
    U = lam * W.copy()
    for t in range(tree.N):
        near = near_nodes(tree, t, knn_pos)
        xt = Xp[t:t + 1]

        def visit(l: int, i: int) -> None:               # MatVec(t, alpha)
            o, e = tree.node_range(l, i)
            if not (o <= t < e):                         # separated under t not in alpha
                if (l, i) in near:                       # ... but holds a neighbour: exact
                    U[t] += (kernel_matrix(xt, Xp[o:e], h) @ W[o:e])[0]
                else:
                    U[t] += (kernel_matrix(xt, Xp[sk.skel[(l, i)]], h) @ wt[(l, i)])[0]
            elif l == tree.L:                            # t's own leaf: exact
                U[t] += (kernel_matrix(xt, Xp[o:e], h) @ W[o:e])[0]
            else:
                visit(l + 1, 2 * i)
                visit(l + 1, 2 * i + 1)

        visit(0, 0)
    return U[:, 0] if vec else U


def dense_Ktilde_knn(sk: Skeletons, knn_pos: np.ndarray) -> np.ndarray:
    """K~ + S assembled entry by entry (permuted order)."""
    tree, Xp, h = sk.tree, sk.Xp, sk.h
    K = kernel_matrix(Xp, Xp, h)
    Kt = dense_Ktilde(sk)
    out = Kt.copy()
    for i in range(tree.N):
        near = near_nodes(tree, i, knn_pos)
        for j in range(tree.N):
            a = interaction_node(tree, i, j)
            if a is None or a in near:
                out[i, j] = K[i, j]
    return out


def S_block(sk: Skeletons, i: int, node: Node) -> np.ndarray:
    """S_{i a} = K_{i a} - K_{i a~} P_{a~ a} for one target and one node of its list."""
    o, e = sk.tree.node_range(*node)
    xi = sk.Xp[i:i + 1]
    return (kernel_matrix(xi, sk.Xp[o:e], sk.h)
            - kernel_matrix(xi, sk.Xp[sk.skel[node]], sk.h) @ full_P(sk, node))[0]
