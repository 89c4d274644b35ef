"""Dense linear algebra named by the paper, written out (Sec. II-B, II-C).

Part of the oracle (test infrastructure only).

* ``lu_factor`` / ``lu_solve``: LU with partial pivoting, as the LAPACK routines
  GETRF / GETRS that Alg. "Factorize" and Alg. "Solve" call for the leaf blocks
  lambda I + K_aa and for the reduced systems of eq. (blocksmw).  The pivot of
  column k is the row of largest magnitude at or below k, ties to the lowest row.
  ``ipiv[k]`` is the row exchanged with row k at step k (LAPACK's convention).
* ``cpqr_id``: the interpolative decomposition that gives the skeletons, i.e. the
  pivot columns of a column-pivoted Householder QR of the sampled block (GEQP3),
  and P from the least-squares fit of the block on those columns (GELS), which for
  the same QR is [I, R11^{-1} R12] with the column permutation undone.
"""
from __future__ import annotations

import numpy as np


class SingularError(ArithmeticError):
    pass


def lu_factor(A: np.ndarray):
    """Right-looking LU with partial pivoting.  Returns (LU, ipiv)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    ipiv = np.empty(n, dtype=np.int64)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))   # first maximum: lowest row on ties
        ipiv[k] = p
        if p != k:
            A[[k, p], :] = A[[p, k], :]
        if A[k, k] == 0.0:
            raise SingularError(f"zero pivot at column {k}")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, ipiv


def lu_solve(LU: np.ndarray, ipiv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B from ``lu_factor`` output: row swaps, unit-lower, then upper solve."""
    X = np.array(B, dtype=np.float64, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = LU.shape[0]
    for k in range(n):
        p = int(ipiv[k])
        if p != k:
            X[[k, p], :] = X[[p, k], :]
    for k in range(n):                       # forward: L has a unit diagonal
        X[k + 1:, :] -= np.outer(LU[k + 1:, k], X[k, :])
    for k in range(n - 1, -1, -1):           # backward
        X[k, :] /= LU[k, k]
        X[:k, :] -= np.outer(LU[:k, k], X[k, :])
    return X[:, 0] if vec else X


def back_substitute(R: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = R^{-1} B for upper-triangular R; a zero diagonal entry gives a zero row of X."""
    s = R.shape[0]
    X = np.array(B, dtype=np.float64, copy=True)
    for k in range(s - 1, -1, -1):
        if R[k, k] == 0.0:
            X[k, :] = 0.0
        else:
            X[k, :] /= R[k, k]
        X[:k, :] -= np.outer(R[:k, k], X[k, :])
    return X


def cpqr_id(A: np.ndarray, s_max: int, tol: float):
    """Column-pivoted Householder QR of A and the interpolative decomposition.

    At step k every trailing column norm is recomputed from the updated trailing
    block (no downdating) and the column of largest norm is chosen, ties to the
    lowest column index.  The rank s:

    * tol <= 0: s = min(s_max, n_cols, n_rows);
    * tol > 0: the smallest k >= 1 with |R_kk| <= tol * |R_00| (the k-th pivot
      column's norm against the first), capped at min(s_max, n_cols, n_rows);
    * in both modes a pivot column of norm exactly 0 at k >= 1 ends the
      factorization with s = k.

    Returns (piv, s, P, rdiag, margin): ``piv[:s]`` are the skeleton columns in
    pivot order; P (s x n_cols) satisfies P[:, piv[:s]] = I and A ~= A[:, piv[:s]] P;
    rdiag holds |R_kk| for k < s; ``margin`` is the smallest relative gap seen
    between the two largest squared trailing norms over the pivot decisions taken,
    and between a pivot norm and the adaptive threshold (1.0 when there was no
    decision).  Two implementations whose roundings differ can only disagree on
    the skeletons when this margin is at rounding level.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    nr, nc = R.shape
    cap = min(s_max, nc, nr)
    piv = np.arange(nc)
    nu0 = 0.0
    rdiag = []
    margin = 1.0
    s = 0
    for k in range(cap):
        norms2 = np.sum(R[k:, k:] * R[k:, k:], axis=0)
        j = int(np.argmax(norms2))             # first maximum: lowest column on ties
        nu = float(np.sqrt(norms2[j]))
        if norms2.size > 1 and norms2[j] > 0.0:
            second = float(np.max(np.delete(norms2, j)))
            margin = min(margin, (norms2[j] - second) / norms2[j])
        if k == 0:
            nu0 = nu
        else:
            if tol > 0.0 and nu0 > 0.0:
                margin = min(margin, abs(nu - tol * nu0) / (tol * nu0))
            if nu == 0.0 or (tol > 0.0 and nu <= tol * nu0):
                break
        p = k + j
        if p != k:
            R[:, [k, p]] = R[:, [p, k]]
            piv[[k, p]] = piv[[p, k]]
        x = R[k:, k].copy()
        alpha = -nu if x[0] >= 0.0 else nu
        v = x
        v[0] -= alpha
        vv = float(v @ v)
        if vv > 0.0:
            beta = 2.0 / vv
            R[k:, k:] -= beta * np.outer(v, v @ R[k:, k:])
        R[k, k] = alpha
        R[k + 1:, k] = 0.0
        rdiag.append(abs(alpha))
        s = k + 1
    T = back_substitute(R[:s, :s], R[:s, s:])
    P = np.zeros((s, nc), dtype=np.float64)
    P[np.arange(s), piv[:s]] = 1.0
    P[:, piv[s:]] = T
    return piv, s, P, np.array(rdiag), margin
