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


# ---------------------------------------------------------------- learned sampling
from oracle.sampling import sample_rows  # noqa: E402


def _knn_setup(N=120, kappa=6, seed=11):
    rng = np.random.default_rng(seed)
    return rng.integers(0, N, size=(16, kappa)), N


def test_knn_ranked_brute_force_and_plain_sampling_agree():
    knn_pos, N = _knn_setup()
    o, n = 40, 16
    vals, counts = L.knn_ranked(knn_pos, o, n)
    hits = {}
    for row in knn_pos:
        for c in row:
            if not (o <= c < o + n):
                hits[int(c)] = hits.get(int(c), 0) + 1
    ref = sorted(hits.items(), key=lambda kv: (-kv[1], kv[0]))
    assert [int(v) for v in vals] == [k for k, _ in ref]
    assert [int(c) for c in counts] == [v for _, v in ref]
    # the plain sample takes the same ranked list first
    ns = min(10, vals.size)
    assert set(sample_rows(knn_pos, o, n, N, ns, seed=3, uid=9)) == set(int(v) for v in vals[:ns])


def test_learned_candidates_structure():
    knn_pos, N = _knn_setup()
    o, n = 40, 16
    cand, hits = L.learned_candidates(knn_pos, o, n, N, n_samp=6, seed=5, uid=13)
    assert cand.size == 48 == np.unique(cand).size
    assert np.all((cand < o) | (cand >= o + n)) and np.all((cand >= 0) & (cand < N))
    vals, counts = L.knn_ranked(knn_pos, o, n)
    k = min(vals.size, 24)
    assert np.array_equal(cand[:k], vals[:k]) and np.array_equal(hits[:k], counts[:k])
    assert np.all(hits[k:] == 0)
    # a budget as large as the complement takes all of it
    cand, _ = L.learned_candidates(knn_pos, o, n, N, n_samp=50, seed=5, uid=13)
    assert sorted(cand.tolist()) == [p for p in range(N) if not (o <= p < o + n)]


def test_uniform_rows_cover_the_complement_evenly():
    o, n, N = 7, 5, 40
    rows = L.uniform_rows(o, n, N, 35000, seed=1, salt=L.HOLD_SALT, uid=6)
    assert np.all((rows < o) | (rows >= o + n))
    counts = np.bincount(rows, minlength=N)
    comp = [p for p in range(N) if not (o <= p < o + n)]
    assert np.all(counts[comp] > 0) and counts[o:o + n].sum() == 0
    chi2 = ((counts[comp] - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 80          # 34 degrees of freedom
    assert not np.array_equal(rows[:32], L.uniform_rows(o, n, N, 32, 1, L.GRAM_SALT, 6))


def test_select_top_brute_force():
    rng = np.random.default_rng(2)
    cand = rng.permutation(100)[:30]
    scores = rng.integers(0, 5, size=30).astype(float)        # many ties
    got = L.select_top(scores, cand, 12)
    ref = sorted(sorted(zip(-scores, cand))[:12], key=lambda t: t[1])
    assert got.tolist() == [int(c) for _, c in ref]


def test_heldout_error_exact_and_trivial_cases():
    rng = np.random.default_rng(3)
    Xp = rng.random((20, 3))
    Xp[5] = Xp[4]                                      # duplicate point: identical columns
    H, cols = np.arange(10, 20), np.array([4, 5, 6])
    w = rng.random(10) + 0.5
    assert L.heldout_error(Xp, H, w, cols, cols, np.eye(3), 0.7) == 0.0
    assert L.heldout_error(Xp, H, w, cols, cols, np.zeros((3, 3)), 0.7) == pytest.approx(1.0)
    P = np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    assert L.heldout_error(Xp, H, w, cols, np.array([4, 6]), P, 0.7) < 1e-30
    assert L.heldout_error(Xp, H, w, cols, np.array([4]), P[:1], 0.7) > 1e-3
    # weights act per row: a row of weight 2 counts as that row taken twice
    H2, w2 = np.concatenate([H, H[:1]]), np.concatenate([w, [w[0]]])
    w1 = w.copy()
    w1[0] *= 2
    Q = np.array([[0.9, 1.1, 0.2]])
    assert L.heldout_error(Xp, H2, w2, cols, np.array([4]), Q, 0.7) == pytest.approx(
        L.heldout_error(Xp, H, w1, cols, np.array([4]), Q, 0.7), rel=1e-12)


def test_stratified_rows_strata_and_weights():
    N, par_o, par_n = 100, 40, 20            # parent [40, 60): alpha [40, 50), sibling [50, 60)
    rows, w = L.stratified_rows(50, 10, par_o, par_n, N, 4000, seed=2, salt=L.HOLD_SALT, uid=9)
    assert np.all((rows[:2000] >= 50) & (rows[:2000] < 60))
    far = rows[2000:]
    assert np.all((far < 40) | (far >= 60))
    assert np.unique(far).size == 80 and np.unique(rows[:2000]).size == 10
    assert w.sum() == pytest.approx(10 + 80)  # each stratum's weights sum to its size
    # parent = the whole problem: all rows from the sibling
    rows, w = L.stratified_rows(0, 50, 0, 100, 100, 64, seed=2, salt=L.HOLD_SALT, uid=3)
    assert np.all(rows < 50) and w.sum() == pytest.approx(50)


def test_leverage_labels_sum_to_the_effective_rank():
    rng = np.random.default_rng(4)
    Xp = rng.random((80, 2))
    cols = np.arange(10)
    rest = np.arange(10, 80)
    lev, t = L.leverage_labels(Xp, rest, cols, rest, np.ones(rest.size), h=0.5, tol=1e-3)
    B = L.gaussian_kernel(Xp[rest], Xp[cols], 0.5)
    s = np.linalg.svd(B, compute_uv=False)
    mu = 1e-6 * float((s ** 2).sum())
    assert lev.sum() == pytest.approx(float((s ** 2 / (s ** 2 + mu)).sum()), rel=1e-6)
    assert t.mean() == pytest.approx(0.0, abs=1e-12) and t.std() == pytest.approx(1.0)


def test_gumbel_keys_sample_proportionally_to_exp_score():
    scores = np.log(np.array([1.0, 2.0, 3.0]))
    assert np.array_equal(L.gumbel_keys(scores, 1, 5, 0.0), scores.astype(np.float32))
    wins = np.zeros(3)
    for uid in range(6000):
        wins[int(np.argmax(L.gumbel_keys(scores, 1, uid, 1.0)))] += 1
    np.testing.assert_allclose(wins / 6000, [1 / 6, 2 / 6, 3 / 6], atol=0.025)
    # temperature 2 flattens to weights ~ sqrt(1), sqrt(2), sqrt(3)
    wins[:] = 0
    for uid in range(6000):
        wins[int(np.argmax(L.gumbel_keys(scores, 2, uid, 2.0)))] += 1
    p = np.sqrt([1.0, 2.0, 3.0])
    np.testing.assert_allclose(wins / 6000, p / p.sum(), atol=0.025)
