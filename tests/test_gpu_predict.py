"""Exact kernel sums at test points on the GPU (iaskit_predict), the GPU side of kernel
regression for binary classification (Sec. III: weights w from the solve, test labels
sign(K(x, X) w) with the exact kernel row over all training points).

* Scores equal the oracle's ``regression.scores`` element by element (FP64 both sides;
  the library's Gram form differs by about 2^-52 (|x|^2 + |y|^2) / (2 h^2) per kernel
  value, far below the 1e-12 bound relative to sum_j K_ij |w_j| used here), for ragged
  test counts (1, a partial 128-point block, several blocks), 1 and 5 right-hand sides
  (a second pass of the 4-column accumulator), points far from every training point
  (score 0) and training points themselves.
* Repeated calls give identical scores (fixed-order chunk sums).
* The classification pipeline: weights from the GPU solve (plain FP64, then the
  kNN-separated operator lambda I + K~ + S by GMRES) match the oracle's weights and the
  predicted labels are the oracle's wherever the score is not within rounding of 0.
* The selected problem of a batch (its points and h) is the one summed over.
* Argument and input errors.
"""
import numpy as np
import pytest

import oracle
from oracle.regression import classify, scores, train_weights
from workloads import labeled_gaussian_mixture, make_points, make_rhs, workload
from workloads.generators import _rng

pytestmark = pytest.mark.gpu


def _bound(Xtr, h, w, Xte):
    K = oracle.gaussian_kernel(Xte, Xtr, h)
    return 1e-12 * (K @ np.abs(w)) + 1e-300


@pytest.mark.parametrize("M", [1, 77, 300, 1000])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_scores_match_the_oracle(gpu_lib, M, nrhs):
    ia = gpu_lib
    w_ = workload("C1", N=2500)
    X = make_points(w_)
    h = 0.4
    ia.iaskit_factor(X, h, 0.1, 64, 24, 1e-6)
    rng = np.random.default_rng(M * 10 + nrhs)
    W = rng.standard_normal((2500, nrhs))
    T = np.concatenate([rng.random((M, 8)) * 1.4 - 0.2])
    T[: min(M, 5)] = X[rng.choice(2500, min(M, 5), replace=False)]   # training points
    if M > 10:
        T[-1] = 50.0                                                   # far away: score 0
    got = ia.iaskit_predict(T, W)
    want = scores(X, h, W, T)
    bound = np.stack([_bound(X, h, W[:, r], T) for r in range(nrhs)], axis=1)
    assert np.all(np.abs(got - want) <= bound)
    if M > 10:
        assert np.all(got[-1] == 0.0)
    np.testing.assert_array_equal(ia.iaskit_predict(T, W), got)       # deterministic
    v = ia.iaskit_predict(T, W[:, 0])
    assert v.shape == (M,)
    np.testing.assert_array_equal(v, got[:, 0])


def _gpu_operator(ia, X, h, m):
    """The oracle's tree with the library's skeletons and P read back, so that the
    oracle's K~ is exactly the one the library factored (whatever pivot near-ties the
    sampled blocks hold; skeleton parity has its own tests)."""
    from oracle.askit import Skeletons
    tree = oracle.build_tree(X, m)
    assert np.array_equal(ia.iaskit_get_perm(len(X)), tree.perm)
    sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
    ranks = ia.iaskit_get_ranks()
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
            sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
    return tree, sk


def test_classification_pipeline_matches_the_oracle(gpu_lib):
    ia = gpu_lib
    Xa, ya = labeled_gaussian_mixture(2300, 8, 16, 0.03, 0.15, _rng(61))
    X, y, Xt, yt = Xa[:2000], ya[:2000], Xa[2000:], ya[2000:]
    h, lam, m, s_max, tol = 0.3, 1e-1, 64, 24, 1e-6
    ia.iaskit_set_option("kappa", 8)
    try:
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        tree, sk = _gpu_operator(ia, X, h, m)
        # S = 0: weights from the direct solve, against the oracle's dense solve of the
        # same lambda I + K~
        w_gpu = ia.iaskit_solve(y[:, None])[:, 0]
        w_or = train_weights(sk, lam, y)
        assert np.linalg.norm(w_gpu - w_or) / np.linalg.norm(w_or) < 1e-9
        s_gpu = ia.iaskit_predict(Xt, w_gpu)
        s_or = scores(X, h, w_or, Xt)
        assert np.all(np.abs(s_gpu - s_or) <= 1e-8 * (oracle.gaussian_kernel(Xt, X, h) @ np.abs(w_or)))
        sure = np.abs(s_or) > 1e-6 * np.abs(s_or).max()
        assert np.array_equal(classify(s_gpu)[sure], classify(s_or)[sure])
        acc = np.mean(classify(s_gpu) == yt)
        print(f"test accuracy, S = 0: {acc:.3f}")
        assert acc > 0.8
    finally:
        for k, v in (("kappa", 16), ("near_field", 0), ("refine", 0), ("refine_tol", 1e-10)):
            ia.iaskit_set_option(k, v)


def test_classification_with_the_near_field(gpu_lib):
    """Weights from the kNN-separated operator lambda I + K~ + S (eq. askit) by GMRES
    preconditioned by the factorization of lambda I + K~, to the paper's classification
    tolerance 1e-3 (a case whose GMRES reaches it within 100 iterations: uniform points,
    h 0.2, s_max 48, tau 1e-8; labels sign(x_0 + x_1 / 2 - 3/4)), checked against the
    oracle's dense lambda I + K~ + S on the library's own skeletons; the test labels
    agree with the oracle's dense weights' labels away from zero scores."""
    from oracle.nearfield import dense_Ktilde_knn
    ia = gpu_lib
    Xa = make_points(workload("C1", N=3001))
    ya = np.where(Xa[:, 0] + 0.5 * Xa[:, 1] > 0.75, 1.0, -1.0)
    X, y, Xt = Xa[:2800], ya[:2800], Xa[2800:]
    h, lam, m = 0.2, 0.1, 50
    try:
        ia.iaskit_set_option("seed", 7)
        ia.iaskit_factor(X, h, lam, m, 48, 1e-8)
        tree, sk = _gpu_operator(ia, X, h, m)
        ia.iaskit_set_option("near_field", 1)
        ia.iaskit_set_option("refine", 100)
        ia.iaskit_set_option("refine_tol", 1e-3)
        w_gpu = ia.iaskit_solve(y[:, None])[:, 0]
        knn_pos = tree.iperm[ia.iaskit_get_knn(len(X), 16)[tree.perm]]
        A = lam * np.eye(len(X)) + dense_Ktilde_knn(sk, knn_pos)
        rho = np.linalg.norm(y[tree.perm] - A @ w_gpu[tree.perm]) / np.linalg.norm(y)
        assert rho < 1e-3, rho
        w_or = train_weights(sk, lam, y, knn_pos)
        s_gpu, s_or = ia.iaskit_predict(Xt, w_gpu), scores(X, h, w_or, Xt)
        sure = np.abs(s_or) > 5e-2 * np.abs(s_or).max()
        assert np.array_equal(classify(s_gpu)[sure], classify(s_or)[sure])
        print(f"S != 0: residual {rho:.2e}, {int(sure.sum())} of {len(Xt)} labels compared")
    finally:
        for k, v in (("seed", 0), ("near_field", 0), ("refine", 0), ("refine_tol", 1e-10)):
            ia.iaskit_set_option(k, v)


def test_selected_problem_of_a_batch(gpu_lib):
    ia = gpu_lib
    rng = np.random.default_rng(62)
    Xs = [rng.random((900, 5)), rng.random((1300, 5)) + 0.5]
    hs, lams = [0.3, 0.7], [0.1, 1.0]
    ia.iaskit_factor_batched(Xs, hs, lams, 64, 16, 1e-6)
    T = rng.random((40, 5))
    try:
        for q in (0, 1):
            ia.iaskit_set_option("problem", q)
            W = rng.standard_normal(len(Xs[q]))
            got = ia.iaskit_predict(T, W)
            want = scores(Xs[q], hs[q], W, T)
            assert np.all(np.abs(got - want) <= _bound(Xs[q], hs[q], W, T))
    finally:
        ia.iaskit_set_option("problem", 0)


def test_errors(gpu_lib):
    ia = gpu_lib
    w_ = workload("C1", N=600)
    X = make_points(w_)
    ia.iaskit_factor(X, 0.5, 1.0, 64, 16, 0.0)
    assert ia.iaskit_predict(np.empty((0, 8)), np.ones(600)).shape == (0,)
    T = np.random.default_rng(63).random((10, 8))
    T[3, 2] = np.nan
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_predict(T, np.ones(600))
    assert e.value.name == "IASKIT_ERR_INPUT"
    lib = ia.load()
    rc = lib.iaskit_predict(T.ctypes.data, 10, np.ones(600).ctypes.data, 0, np.empty(10).ctypes.data)
    assert ia.ERRORS[rc] == "IASKIT_ERR_ARG"
    # the library is still usable
    T[3, 2] = 0.5
    assert np.all(np.isfinite(ia.iaskit_predict(T, np.ones(600))))
