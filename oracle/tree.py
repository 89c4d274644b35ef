"""Binary space partition (Sec. II-A) and exact kNN lists (Sec. II-B).

Part of the oracle (test infrastructure only).

Tree (Sec. II-A: leaves hold at most m points, levels l = 0 at the root to
l = log2(N/m) at the leaves; the paper's ball tree is replaced by a median split):

* depth L is the smallest l with ceil(N / 2^l) <= m, and every node above level L
  is split, so all leaves sit at level L;
* a node of n points gets a left child of floor(n/2) points and a right child of
  the remaining n - floor(n/2); node sizes therefore depend on N only;
* the split coordinate c is the one of largest spread max - min over the node's
  points, ties to the lowest coordinate;
* the left child takes the floor(n/2) points that come first in ascending order of
  the key (x_c, original index);
* inside every node the points are kept in ascending original index.

``perm[pos]`` is the original index of the point at permuted position ``pos``;
node (l, i) owns positions [off[l][i], off[l][i+1]).

kNN (the input that drives ASKIT's sampling, Sec. II-B): for every point the kappa
nearest other points in ascending (squared distance, original index), with the
squared distance of ``kernel.sqdist``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from .kernel import sqdist


def tree_depth(N: int, m: int) -> int:
    """Smallest L with ceil(N / 2^L) <= m."""
    L = 0
    while -(-N // (1 << L)) > m:
        L += 1
    return L


def node_sizes(N: int, L: int) -> List[np.ndarray]:
    """Sizes of the nodes of every level: level l+1 interleaves (floor(n/2), n - floor(n/2))."""
    sizes = [np.array([N], dtype=np.int64)]
    for _ in range(L):
        prev = sizes[-1]
        nxt = np.empty(2 * prev.size, dtype=np.int64)
        nxt[0::2] = prev // 2
        nxt[1::2] = prev - prev // 2
        sizes.append(nxt)
    return sizes


@dataclass
class Tree:
    N: int
    d: int
    m: int
    L: int
    perm: np.ndarray                     # perm[pos] = original index
    iperm: np.ndarray                    # iperm[orig] = pos
    off: List[np.ndarray] = field(default_factory=list)   # off[l] has 2^l + 1 entries
    split_dim: List[np.ndarray] = field(default_factory=list)  # per level < L

    def node_range(self, l: int, i: int):
        return int(self.off[l][i]), int(self.off[l][i + 1])

    def is_leaf(self, l: int) -> bool:
        return l == self.L


def build_tree(X: np.ndarray, m: int) -> Tree:
    """Median split on the coordinate of largest spread, level by level (Sec. II-A)."""
    X = np.asarray(X, dtype=np.float64)
    N, d = X.shape
    L = tree_depth(N, m)
    sizes = node_sizes(N, L)
    off = [np.concatenate([[0], np.cumsum(s)]).astype(np.int64) for s in sizes]
    perm = np.arange(N, dtype=np.int64)
    split_dim = []
    for l in range(L):
        dims = np.empty(1 << l, dtype=np.int64)
        for i in range(1 << l):
            o, e = int(off[l][i]), int(off[l][i + 1])
            idx = perm[o:e].copy()
            pts = X[idx]
            spread = pts.max(axis=0) - pts.min(axis=0)
            c = int(np.argmax(spread))          # first maximum: lowest coordinate on ties
            dims[i] = c
            order = np.lexsort((idx, pts[:, c]))   # primary x_c, then original index
            k = (e - o) // 2
            perm[o:o + k] = np.sort(idx[order[:k]])
            perm[o + k:e] = np.sort(idx[order[k:]])
        split_dim.append(dims)
    iperm = np.empty(N, dtype=np.int64)
    iperm[perm] = np.arange(N, dtype=np.int64)
    return Tree(N=N, d=d, m=m, L=L, perm=perm, iperm=iperm, off=off, split_dim=split_dim)


def knn_bruteforce(X: np.ndarray, kappa: int, chunk: int = 512) -> np.ndarray:
    """kappa nearest neighbours of every point, self excluded, ascending (d^2, index).

    Returns int64 (N, min(kappa, N-1)) of original indices.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    k = min(kappa, N - 1)
    out = np.empty((N, k), dtype=np.int64)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        D = sqdist(X[s:e], X)
        D[np.arange(e - s), np.arange(s, e)] = np.inf
        # a stable sort of each row keeps equal distances in ascending index order
        order = np.argsort(D, axis=1, kind="stable")
        out[s:e] = order[:, :k]
    return out
