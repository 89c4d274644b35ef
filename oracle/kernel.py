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


# ------------------------------------------------------------- the polynomial kernel
# Sec. IV (Tab. weak) reports tests with a polynomial kernel but gives neither its degree
# nor its constants; the one used here is K(x, y) = (x . y / h^2 + c)^p with an integer
# degree p >= 1 and c >= 0, h the factorization's length scale.


def dot_in_order(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Pairwise dot products |A| x |B|, coordinates summed in index order."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros((A.shape[0], B.shape[0]), dtype=np.float64)
    for k in range(A.shape[1]):
        out = out + A[:, k][:, None] * B[:, k][None, :]
    return out


def polynomial_kernel(A: np.ndarray, B: np.ndarray, h: float, p: int = 2, c: float = 1.0) -> np.ndarray:
    """K(A, B)_{ij} = (a_i . b_j / h^2 + c)^p, the power by repeated multiplication."""
    t = dot_in_order(A, B) / (h * h) + c
    v = t.copy()
    for _ in range(1, int(p)):
        v = v * t
    return v


class PolynomialKernel:
    """Selects the polynomial kernel (degree p, constant c) while active (a context)."""

    def __init__(self, p: int = 2, c: float = 1.0):
        self.p, self.c = int(p), float(c)

    def __enter__(self):
        global _CURRENT
        self._saved = _CURRENT
        _CURRENT = self
        return self

    def __exit__(self, *exc):
        global _CURRENT
        _CURRENT = self._saved
        return False


_CURRENT = None  # None: the Gaussian of eq. (gaussian)


def kernel_matrix(A: np.ndarray, B: np.ndarray, h: float) -> np.ndarray:
    """The kernel in use: the Gaussian, or the polynomial inside a PolynomialKernel block."""
    if _CURRENT is None:
        return gaussian_kernel(A, B, h)
    return polynomial_kernel(A, B, h, _CURRENT.p, _CURRENT.c)
