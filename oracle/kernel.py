"""Gaussian kernel of Sec. I, eq. (gaussian): K(x, y) = exp(-||x - y||^2 / (2 h^2)).

Part of the oracle (test infrastructure only).

The squared distance is the difference form summed over coordinates in index
order k = 0 .. d-1, each subtraction, product and addition rounded separately
(numpy applies the three ufuncs one after another, so nothing is fused).  The
kNN lists are defined on exactly this quantity.
"""
from __future__ import annotations

import numpy as np


def sqdist(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Pairwise squared distances |A| x |B|, difference form, coordinates summed in order."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros((A.shape[0], B.shape[0]), dtype=np.float64)
    for k in range(A.shape[1]):
        diff = A[:, k][:, None] - B[:, k][None, :]
        out = out + diff * diff
    return out


def gaussian_kernel(A: np.ndarray, B: np.ndarray, h: float) -> np.ndarray:
    """K(A, B)_{ij} = exp(-||a_i - b_j||^2 / (2 h^2)), eq. (gaussian)."""
    return np.exp(-sqdist(A, B) / (2.0 * h * h))
