"""Pins of the oracle's kernel regression for binary classification (Sec. III).

* scores against a brute-force double loop of Gaussian kernel values;
* one training point: w = u / (lambda + 1) (K(x, x) = 1), so the score of x' is
  exp(-|x' - x|^2 / (2 h^2)) u / (lambda + 1), a closed form;
* a very large lambda: w = u / lambda + O(lambda^-2), so the labels are the signs of
  the Parzen sums K(x, X) u;
* with skeletons of full rank K~ = K and the weights are the dense solve with K;
* two well-separated clusters with opposite labels are classified without error, and
  the synthetic mixture task is learned far above chance.
"""
import math

import numpy as np

import oracle
from oracle.kernel import gaussian_kernel
from oracle.regression import accuracy, classify, scores, train_weights
from workloads import labeled_gaussian_mixture
from workloads.generators import _rng


def test_scores_brute_force():
    rng = np.random.default_rng(51)
    Xtr, Xte = rng.random((17, 3)), rng.random((5, 3))
    w = rng.standard_normal(17)
    h = 0.7
    want = [sum(math.exp(-sum((a - b) ** 2 for a, b in zip(x, y)) / (2 * h * h)) * wj
                for y, wj in zip(Xtr, w)) for x in Xte]
    np.testing.assert_allclose(scores(Xtr, h, w, Xte), want, rtol=1e-13)


def test_single_training_point_closed_form():
    # two training points so far apart that K between them is 0 in FP64: each weight
    # is its label / (lambda + 1), and a test point near the first scores
    # -exp(-|x' - x|^2 / (2 h^2)) / (lambda + 1)
    X = np.array([[0.2, 0.4], [100.0, 100.0]])
    y = np.array([-1.0, 1.0])
    lam, h = 0.3, 0.5
    _, _, sk, _ = oracle.build_all(X, h, lam, 4, 2, 0.0)
    w = train_weights(sk, lam, y)
    np.testing.assert_allclose(w, y / (lam + 1.0), rtol=1e-15)
    xt = np.array([[0.5, 0.1], [0.2, 0.4]])
    d2 = ((xt - X[0]) ** 2).sum(axis=1)
    np.testing.assert_allclose(scores(X, h, w, xt), -np.exp(-d2 / (2 * h * h)) / (lam + 1), rtol=1e-14)
    assert list(classify(scores(X, h, w, xt))) == [-1.0, -1.0]


def test_large_lambda_gives_parzen_signs():
    rng = np.random.default_rng(52)
    X = rng.random((300, 3))
    y = np.where(X[:, 0] + 0.3 * X[:, 1] > 0.6, 1.0, -1.0)
    h, lam = 0.3, 1e8
    _, _, sk, _ = oracle.build_all(X, h, lam, 40, 16, 0.0)
    w = train_weights(sk, lam, y)
    Xt = rng.random((200, 3))
    parzen = gaussian_kernel(Xt, X, h) @ y
    keep = np.abs(parzen) > 1e-3                       # away from exact ties
    assert np.array_equal(classify(scores(X, h, w, Xt))[keep], classify(parzen)[keep])


def test_full_rank_weights_are_the_dense_solve():
    rng = np.random.default_rng(53)
    X = rng.random((200, 2))
    y = np.where(rng.random(200) > 0.5, 1.0, -1.0)
    h, lam = 0.4, 0.1
    _, _, sk, _ = oracle.build_all(X, h, lam, 30, 10 ** 6, 0.0)
    w = train_weights(sk, lam, y)
    w_dense = np.linalg.solve(lam * np.eye(200) + gaussian_kernel(X, X, h), y)
    np.testing.assert_allclose(w, w_dense, rtol=1e-9, atol=1e-9 * np.abs(w_dense).max())


def test_separated_clusters_and_mixture_task():
    rng = np.random.default_rng(54)
    a = 0.05 * rng.standard_normal((120, 4))
    b = 5.0 + 0.05 * rng.standard_normal((120, 4))
    X = np.concatenate([a[:100], b[:100]])
    y = np.concatenate([np.ones(100), -np.ones(100)])
    Xt = np.concatenate([a[100:], b[100:]])
    yt = np.concatenate([np.ones(20), -np.ones(20)])
    _, _, sk, _ = oracle.build_all(X, 1.0, 1e-2, 25, 12, 1e-8)
    w = train_weights(sk, 1e-2, y)
    assert accuracy(classify(scores(X, 1.0, w, Xt)), yt) == 1.0
    # the synthetic mixture task (16 components in 8 dimensions, half of them +1)
    Xa, ya = labeled_gaussian_mixture(700, 8, 16, 0.03, 0.15, _rng(55))
    X, y, Xt, yt = Xa[:600], ya[:600], Xa[600:], ya[600:]
    _, knn, sk, _ = oracle.build_all(X, 0.3, 1e-2, 40, 24, 1e-6, kappa=8)
    knn_pos = sk.tree.iperm[knn[sk.tree.perm]]
    for kp in (None, knn_pos):
        w = train_weights(sk, 1e-2, y, kp)
        acc = accuracy(classify(scores(X, 0.3, w, Xt)), yt)
        assert acc > 0.8, acc
