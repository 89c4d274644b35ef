"""Kernel regression for binary classification (Sec. III, "Kernel regression for
binary classification").

Part of the oracle (test infrastructure only).

Training: the regression weights w solve (lambda I + K~ + S) w = u for the training
labels u(i) in {-1, 1}; here by a dense solve of that matrix assembled from its
definition (``askit.dense_Ktilde``, plus ``nearfield.dense_Ktilde_knn`` when
neighbour lists are given; S = 0 without them).  Testing: a point x outside the
training set gets the label sign(K(x, X) w), K(x, X) the exact kernel row over all
training points; a score of exactly 0 is labelled +1 (the paper does not say).  The
accuracy is the fraction of test points whose computed label equals the given one.
Everything is FP64; w is returned in the training points' original order.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from .askit import Skeletons, dense_Ktilde
from .kernel import kernel_matrix
from .nearfield import dense_Ktilde_knn


def train_weights(sk: Skeletons, lam: float, labels: np.ndarray,
                  knn_pos: Optional[np.ndarray] = None) -> np.ndarray:
    """w with (lambda I + K~ [+ S]) w = labels (original order in and out)."""
    tree = sk.tree
    Kt = dense_Ktilde(sk) if knn_pos is None else dense_Ktilde_knn(sk, knn_pos)
    A = lam * np.eye(tree.N) + Kt
    wp = np.linalg.solve(A, np.asarray(labels, dtype=np.float64)[tree.perm])
    w = np.empty_like(wp)
    w[tree.perm] = wp
    return w


def scores(Xtrain: np.ndarray, h: float, w: np.ndarray, Xtest: np.ndarray) -> np.ndarray:
    """K(Xtest, Xtrain) w: one score per test point (per column of w)."""
    return kernel_matrix(np.asarray(Xtest, dtype=np.float64), np.asarray(Xtrain, dtype=np.float64), h) @ w


def classify(s: np.ndarray) -> np.ndarray:
    """sign of the scores, with +1 for a score of exactly 0."""
    return np.where(np.asarray(s) >= 0.0, 1.0, -1.0)


def accuracy(predicted: np.ndarray, truth: np.ndarray) -> float:
    return float(np.mean(np.asarray(predicted) == np.asarray(truth)))
