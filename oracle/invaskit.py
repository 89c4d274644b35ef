"""INV-ASKIT factorization and solve (Sec. II-C), written literally, plus metrics.

Part of the oracle (test infrastructure only).

``factorize`` follows Alg. "Factorize" as a post-order recursion:

* leaf alpha: LU with partial pivoting of lambda I + K_aa;
* internal alpha with children l, r: factorize both children; form
  K_{l r~}, K_{r l~} and the full P_{l~ l}, P_{r~ r} (eq. innerid);
  W_{l r~} = Solve(l, K_{l r~}), W_{r l~} = Solve(r, K_{r l~});
  LU of the reduced system Z = [[I, P_{r~ r} W_{r l~}], [P_{l~ l} W_{l r~}, I]]
  of eq. (blocksmw), rows and columns ordered [r~ part (s_r); l~ part (s_l)].

``solve`` follows Alg. "Solve": leaf LU solve; otherwise v = [Solve(l, u_l);
Solve(r, u_r)], y = Z^{-1} V v with V v = [P_{r~ r} v_r; P_{l~ l} v_l], and
w = v - W y, i.e. w_l = v_l - W_{l r~} y[:s_r], w_r = v_r - W_{r l~} y[s_r:]
(eq. smw: (I - W Z V) D^{-1}).  V is applied through the full P matrices.

``dense_solve`` assembles lambda I + K~ densely and solves it with numpy's dense
solver: the reference result the algorithm must reach up to rounding.

Metrics (eq. error, Sec. III, with S = 0): eps_I, the relative residual rho, and
eps_M estimated on sampled rows.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional, Tuple

import numpy as np

from .askit import Skeletons, dense_Ktilde, full_P, matvec, skeletonize
from .kernel import kernel_matrix
from .linalg import lu_factor, lu_solve
from .tree import Tree, build_tree, knn_bruteforce

Node = Tuple[int, int]


@dataclass
class Factorization:
    sk: Skeletons
    lam: float
    leaf_lu: Dict[Node, tuple] = field(default_factory=dict)
    W_l: Dict[Node, np.ndarray] = field(default_factory=dict)   # W_{l r~}, |l| x s_r
    W_r: Dict[Node, np.ndarray] = field(default_factory=dict)   # W_{r l~}, |r| x s_l
    Z_lu: Dict[Node, tuple] = field(default_factory=dict)
    Z: Dict[Node, np.ndarray] = field(default_factory=dict)
    Pfull: Dict[Node, np.ndarray] = field(default_factory=dict)

    @property
    def tree(self) -> Tree:
        return self.sk.tree


def _children(node: Node):
    l, i = node
    return (l + 1, 2 * i), (l + 1, 2 * i + 1)


def factorize(sk: Skeletons, lam: float) -> Factorization:
    """Alg. "Factorize" on the root (post-order recursion)."""
    F = Factorization(sk=sk, lam=lam)
    tree, Xp, h = sk.tree, sk.Xp, sk.h

    def fact(node: Node):
        l, i = node
        o, e = tree.node_range(l, i)
        if l == tree.L:
            A = lam * np.eye(e - o) + kernel_matrix(Xp[o:e], Xp[o:e], h)
            F.leaf_lu[node] = lu_factor(A)
            return
        left, right = _children(node)
        fact(left)
        fact(right)
        ol, el = tree.node_range(*left)
        orr, er = tree.node_range(*right)
        K_lr = kernel_matrix(Xp[ol:el], Xp[sk.skel[right]], h)      # K_{l r~}
        K_rl = kernel_matrix(Xp[orr:er], Xp[sk.skel[left]], h)      # K_{r l~}
        P_l = full_P(sk, left, F.Pfull)                               # P_{l~ l}
        P_r = full_P(sk, right, F.Pfull)                              # P_{r~ r}
        W_l = solve_node(F, left, K_lr)
        W_r = solve_node(F, right, K_rl)
        s_l, s_r = P_l.shape[0], P_r.shape[0]
        Z = np.eye(s_r + s_l)
        Z[:s_r, s_r:] = P_r @ W_r
        Z[s_r:, :s_r] = P_l @ W_l
        F.W_l[node], F.W_r[node] = W_l, W_r
        F.Z[node] = Z
        F.Z_lu[node] = lu_factor(Z)

    fact((0, 0))
    return F


def solve_node(F: Factorization, node: Node, U: np.ndarray) -> np.ndarray:
    """Alg. "Solve": (lambda I + K~_aa)^{-1} U for the node ``node`` (permuted rows)."""
    tree = F.tree
    l, i = node
    if l == tree.L:
        LU, ipiv = F.leaf_lu[node]
        return lu_solve(LU, ipiv, U)
    left, right = _children(node)
    ol, el = tree.node_range(*left)
    o, _ = tree.node_range(l, i)
    nl = el - ol
    vec = U.ndim == 1
    U2 = U[:, None] if vec else U
    v_l = solve_node(F, left, U2[:nl])
    v_r = solve_node(F, right, U2[nl:])
    P_l, P_r = F.Pfull[left], F.Pfull[right]
    s_r = P_r.shape[0]
    t = np.vstack([P_r @ v_r, P_l @ v_l])
    LU, ipiv = F.Z_lu[node]
    y = lu_solve(LU, ipiv, t)
    w = np.vstack([v_l - F.W_l[node] @ y[:s_r], v_r - F.W_r[node] @ y[s_r:]])
    return w[:, 0] if vec else w


def solve(F: Factorization, u: np.ndarray) -> np.ndarray:
    """w = (lambda I + K~)^{-1} u with u, w in ORIGINAL point order."""
    tree = F.tree
    u = np.asarray(u, dtype=np.float64)
    up = u[tree.perm]
    wp = solve_node(F, (0, 0), up)
    w = np.empty_like(wp)
    w[tree.perm] = wp
    return w


def dense_solve(sk: Skeletons, lam: float, u: np.ndarray) -> np.ndarray:
    """Reference result: (lambda I + K~)^{-1} u with K~ assembled densely (ORIGINAL order)."""
    tree = sk.tree
    A = lam * np.eye(tree.N) + dense_Ktilde(sk)
    wp = np.linalg.solve(A, np.asarray(u, dtype=np.float64)[tree.perm])
    w = np.empty_like(wp)
    w[tree.perm] = wp
    return w


def apply_operator(sk: Skeletons, lam: float, w: np.ndarray) -> np.ndarray:
    """(lambda I + K~) w by the hierarchical MatVec, ORIGINAL order in and out."""
    tree = sk.tree
    w = np.asarray(w, dtype=np.float64)
    up = matvec(sk, lam, w[tree.perm])
    u = np.empty_like(up)
    u[tree.perm] = up
    return u


def residual(sk: Skeletons, lam: float, w: np.ndarray, u: np.ndarray) -> float:
    """rho = ||u - (lambda I + K~) w|| / ||u|| (eq. error with S = 0)."""
    r = np.asarray(u) - apply_operator(sk, lam, w)
    return float(np.linalg.norm(r) / np.linalg.norm(u))


def eps_I(F: Factorization, w: np.ndarray) -> float:
    """eps_I = ||w - (lambda I + K~)^{-1} (lambda I + K~) w|| / ||w|| (eq. error)."""
    u = apply_operator(F.sk, F.lam, w)
    w2 = solve(F, u)
    return float(np.linalg.norm(np.asarray(w) - w2) / np.linalg.norm(w))


def eps_M_sampled(sk: Skeletons, X: np.ndarray, w: np.ndarray, rows: np.ndarray) -> float:
    """eps_M = ||K w - K~ w|| / ||K w|| restricted to the sampled rows (eq. error, S = 0)."""
    Kw_rows = kernel_matrix(np.asarray(X)[rows], X, sk.h) @ w
    Ktw = apply_operator(sk, 0.0, w)[rows]
    return float(np.linalg.norm(Kw_rows - Ktw) / np.linalg.norm(Kw_rows))


def build_all(X: np.ndarray, h: float, lam: float, m: int, s_max: int, tol: float,
              kappa: int = 16, samp_factor: int = 2, seed: int = 0,
              knn: Optional[np.ndarray] = None):
    """Tree, kNN, skeletons and factorization for one problem.  Returns (tree, knn, sk, F)."""
    tree = build_tree(X, m)
    if knn is None:
        knn = knn_bruteforce(X, kappa)
    sk = skeletonize(X, tree, knn, h, s_max, tol, samp_factor=samp_factor, seed=seed)
    F = factorize(sk, lam)
    return tree, knn, sk, F
