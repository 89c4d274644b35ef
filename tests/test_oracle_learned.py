"""Pins of the learned-sampler oracle (oracle/learned.py) against independent facts."""
import math

import numpy as np
import pytest

from oracle import learned as L


def _small():
    p = L.mlp_init(seed=3, fin=L.NFEAT, width=16)
    X = np.random.default_rng(4).standard_normal((24, L.NFEAT))
    t = np.random.default_rng(5).standard_normal(24)
    return p, X, t


def test_mlp_gradients_match_central_differences():
    p, X, t = _small()
    y, cache = L.mlp_forward(p, X)
    g = L.mlp_backward(p, cache, y, t)
    eps = 1e-6
    rng = np.random.default_rng(6)
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = L.mse_loss(L.mlp_forward(p, X)[0], t)
            flat[idx] = old - eps
            lm = L.mse_loss(L.mlp_forward(p, X)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_mlp_forward_is_the_composition():
    p, X, _ = _small()
    y, _ = L.mlp_forward(p, X)
    x = X[3]
    h1 = np.maximum(p["W1"] @ x + p["b1"], 0)
    h2 = np.maximum(p["W2"] @ h1 + p["b2"], 0)
    assert y[3] == pytest.approx(float(p["w3"] @ h2 + p["b3"][0]), rel=1e-14)


def test_adam_first_step_closed_form():
    # with zero moments, one bias-corrected step moves every weight by -lr g / (|g| + eps)
    p, X, t = _small()
    p0 = {k: v.copy() for k, v in p.items()}
    y, cache = L.mlp_forward(p, X)
    g = L.mlp_backward(p, cache, y, t)
    L.adam_step(p, g, {}, lr=0.01)
    for k in p:
        np.testing.assert_allclose(p[k], p0[k] - 0.01 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=1e-15)


def test_ridge_leverage_matches_svd_and_trace():
    rng = np.random.default_rng(7)
    B = rng.standard_normal((200, 6)) @ rng.standard_normal((6, 30))   # rank 6
    G = B.T @ B
    mu = 1e-3
    lev = L.ridge_leverage(B, G, mu)
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    ref = (U ** 2 * (s ** 2 / (s ** 2 + mu))).sum(axis=1)
    np.testing.assert_allclose(lev, ref, rtol=1e-8, atol=1e-12)
    assert lev.sum() == pytest.approx(6.0, rel=1e-4)    # leverage sums to the rank
    assert np.all(lev <= 1.0 + 1e-12) and np.all(lev >= -1e-12)


def test_features_hand_computed():
    # points on a line; node columns 0 and 2, candidate 5
    Xp = np.array([[0.0], [1.0], [2.0], [3.0], [4.0], [6.0]])
    cols = np.array([0, 2])
    F = L.candidate_features(Xp, np.array([5]), np.array([3]), cols, h=2.0, level=2, L=4, n=8,
                             N=64, kappa=16)
    mu, r = 1.0, 1.0
    assert F[0, 0] == pytest.approx(math.log(4) / math.log(17))
    assert F[0, 1] == pytest.approx((6 - mu) / 2.0)
    k0, k2 = math.exp(-36 / 8), math.exp(-16 / 8)
    assert F[0, 2] == pytest.approx(k2)
    assert F[0, 3] == pytest.approx((k0 + k2) / 2)
    assert F[0, 4] == pytest.approx(0.5)
    assert F[0, 5] == pytest.approx(3 / 6)
    assert F[0, 6] == pytest.approx(5.0 / r)
    assert F[0, 7] == 0.0


def test_column_subset_is_evenly_spaced():
    cols = np.arange(100, 200)
    sub = L.column_subset(cols)
    assert sub.size == 32 and sub[0] == 100 and list(sub[:3]) == [100, 103, 106]
    assert list(L.column_subset(np.arange(5))) == [0, 1, 2, 3, 4]
