"""Pins of the oracle's polynomial kernel (Sec. IV: "tests with a polynomial kernel";
the paper gives no degree or constants: K(x, y) = (x . y / h^2 + c)^p is chosen here).

* a closed form and a brute-force double loop;
* exact low rank: on d = 3 points the degree-2 kernel matrix has rank at most
  C(3 + 2, 2) = 10, so skeletons of 10 columns reproduce it: K~ = K to rounding and the
  sampled eps_M vanishes (the paper reports eps_M of order 1e-12 for its polynomial
  runs, Tab. weak), and the factorization's solve is the dense solve of lambda I + K;
* the selection is a context: the Gaussian holds again outside it.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.askit import dense_Ktilde
from oracle.kernel import PolynomialKernel, gaussian_kernel, kernel_matrix, polynomial_kernel


def test_closed_form_and_brute_force():
    K = polynomial_kernel(np.array([[1.0, 2.0]]), np.array([[3.0, -1.0]]), 2.0, p=3, c=1.0)
    assert K[0, 0] == (1.0 / 4.0 + 1.0) ** 3          # x.y = 1, h^2 = 4: exactly 1.953125
    rng = np.random.default_rng(71)
    A, B = rng.standard_normal((7, 5)), rng.standard_normal((4, 5))
    want = [[(sum(a * b for a, b in zip(x, y)) / 0.49 + 0.5) ** 4 for y in B] for x in A]
    np.testing.assert_allclose(polynomial_kernel(A, B, 0.7, p=4, c=0.5), want, rtol=1e-13)


def test_context_selects_the_kernel():
    X = np.random.default_rng(72).random((5, 3))
    with PolynomialKernel(p=2, c=1.0):
        np.testing.assert_array_equal(kernel_matrix(X, X, 0.9), polynomial_kernel(X, X, 0.9, 2, 1.0))
    np.testing.assert_array_equal(kernel_matrix(X, X, 0.9), gaussian_kernel(X, X, 0.9))


def test_exact_low_rank_is_reproduced():
    N, d = 600, 3
    X = np.random.default_rng(73).random((N, d))
    rank = math.comb(d + 2, 2)
    u = np.random.default_rng(74).standard_normal(N)
    with PolynomialKernel(p=2, c=1.0):
        tree, knn, sk, F = oracle.build_all(X, 1.0, 1.0, 40, 16, 1e-9)
        ranks = [sk.rank(n) for n in sk.skel]
        assert max(ranks) <= rank
        K = polynomial_kernel(X, X, 1.0, 2, 1.0)
        perm = tree.perm
        Kt = np.empty_like(K)
        Kt[np.ix_(perm, perm)] = dense_Ktilde(sk)
        assert np.linalg.norm(Kt - K) / np.linalg.norm(K) < 1e-9
        eps = oracle.eps_M_sampled(sk, X, u, np.arange(N))
        assert eps < 1e-9
        w = oracle.solve(F, u)
        w_dense = np.linalg.solve(np.eye(N) + K, u)
        assert np.linalg.norm(w - w_dense) / np.linalg.norm(w_dense) < 1e-8
