"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer and index work (tree permutation, kNN lists, samples, skeletons) must be
bit-exact.  Floating point (P, solutions, operator) must agree to 1e-10 relative,
the FP64 tolerance of the plain path: both sides compute the same quantities in
FP64, differing only in summation order and the exp implementation, so agreement
is limited by conditioning times ~1e-16, far inside 1e-10 for these cases.
Skeleton indices are compared where the oracle's pivot margin shows no near-tie.
"""
import numpy as np
import pytest

import oracle
from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu

RTOL = 1e-10
TIE_MARGIN = 1e-9


def _factor_both(ia, X, h, lam, m, s_max, tol, seed=0, kappa=16):
    ia.iaskit_set_option("seed", seed)
    ia.iaskit_set_option("kappa", kappa)
    ia.iaskit_factor(X, h, lam, m, s_max, tol)
    tree, knn, sk, F = oracle.build_all(X, h, lam, m, s_max, tol, kappa=kappa, seed=seed)
    return tree, knn, sk, F


CASES = {
    # name: (workload, N, h, lam, m, s_max, tol, nrhs)
    "c1_full": ("C1", 4096, 0.5, 1.0, 64, 32, 0.0, 1),
    "ragged_adaptive": ("C1", 3001, 0.4, 0.1, 50, 24, 1e-6, 3),
    "gmm54": ("C2", 2500, 1.0, 1e-2, 64, 24, 1e-5, 2),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, gpu_lib):
    ia = gpu_lib
    wname, N, h, lam, m, s_max, tol, nrhs = CASES[request.param]
    w = workload(wname, N=N)
    X = make_points(w)
    tree, knn, sk, F = _factor_both(ia, X, h, lam, m, s_max, tol, seed=7)
    u = make_rhs(w, N=N, nrhs=nrhs)
    return dict(ia=ia, X=X, tree=tree, knn=knn, sk=sk, F=F, u=u, N=N, lam=lam, s_max=s_max)


def test_tree_permutation_bitexact(case):
    ia = case["ia"]
    assert ia.iaskit_depth() == case["tree"].L
    assert np.array_equal(ia.iaskit_get_perm(case["N"]), case["tree"].perm)


def test_knn_bitexact(case):
    ia = case["ia"]
    assert np.array_equal(ia.iaskit_get_knn(case["N"], 16), case["knn"])


def test_samples_bitexact(case):
    ia, tree, sk = case["ia"], case["tree"], case["sk"]
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            assert np.array_equal(ia.iaskit_get_samples(l, i), sk.samp[(l, i)]), (l, i)


def test_skeletons_and_P(case):
    ia, tree, sk = case["ia"], case["tree"], case["sk"]
    assert min(sk.margin.values()) > TIE_MARGIN   # inputs chosen free of pivot near-ties
    ranks = ia.iaskit_get_ranks()
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            node = (l, i)
            s = sk.rank(node)
            assert ranks[(1 << l) + i] == s, node
            assert np.array_equal(ia.iaskit_get_skeleton(l, i), sk.skel[node]), node
            P = ia.iaskit_get_P(l, i, s)
            np.testing.assert_allclose(P, sk.P[node], rtol=RTOL, atol=RTOL * np.abs(sk.P[node]).max())


def test_solve_matches_oracle(case):
    ia, F, u = case["ia"], case["F"], case["u"]
    w_gpu = ia.iaskit_solve(u)
    w_ref = oracle.solve(F, u)
    err = np.linalg.norm(w_gpu - w_ref) / np.linalg.norm(w_ref)
    assert err < RTOL, err
    # the solve inverts the oracle's operator
    assert oracle.residual(case["sk"], case["lam"], w_gpu, u) < 1e-10


def test_apply_matches_oracle(case):
    ia, sk = case["ia"], case["sk"]
    w = make_rhs(workload("C1"), N=case["N"], nrhs=2) * 0.5
    u_gpu = ia.iaskit_apply(w)
    u_ref = oracle.invaskit.apply_operator(sk, case["lam"], w)
    err = np.linalg.norm(u_gpu - u_ref) / np.linalg.norm(u_ref)
    assert err < RTOL, err


def test_solve_then_apply_roundtrip(case):
    ia, u = case["ia"], case["u"]
    w = ia.iaskit_solve(u)
    r = u - ia.iaskit_apply(w)
    assert np.linalg.norm(r) / np.linalg.norm(u) < 1e-10


# ------------------------------------------------------------------ edge cases
def test_single_leaf_is_dense_solve(gpu_lib):
    ia = gpu_lib
    X = np.random.default_rng(1).random((40, 3))
    u = np.random.default_rng(2).standard_normal((40, 2))
    ia.iaskit_factor(X, 0.5, 0.1, 64, 8, 0.0)
    assert ia.iaskit_depth() == 0
    w = ia.iaskit_solve(u)
    A = 0.1 * np.eye(40) + oracle.gaussian_kernel(X, X, 0.5)
    np.testing.assert_allclose(w, np.linalg.solve(A, u), rtol=1e-10)


def test_two_points(gpu_lib):
    ia = gpu_lib
    X = np.array([[0.0, 0.0], [1.0, 0.0]])
    ia.iaskit_factor(X, 1.0, 0.5, 2, 1, 0.0)
    u = np.array([1.0, -2.0])
    w = ia.iaskit_solve(u)
    A = 0.5 * np.eye(2) + oracle.gaussian_kernel(X, X, 1.0)
    np.testing.assert_allclose(w, np.linalg.solve(A, u), rtol=1e-12)


def test_duplicate_points_use_exact_fallback(gpu_lib):
    # 200 copies of each of 10 points: every query has 199 exact ties at distance 0,
    # more than the prefilter keeps (4 lists of 32), so no cut can be certified and the
    # exact scan decides by index
    ia = gpu_lib
    rng = np.random.default_rng(4)
    X = np.repeat(rng.random((10, 3)), 200, axis=0)[rng.permutation(2000)]
    ia.iaskit_factor(X, 0.5, 1.0, 64, 16, 1e-8)
    assert np.array_equal(ia.iaskit_get_knn(len(X), 16), oracle.knn_bruteforce(X, 16))
    assert np.array_equal(ia.iaskit_get_perm(len(X)), oracle.build_tree(X, 64).perm)
    assert ia.iaskit_stats()["knn_fallback"] > 0


def test_duplicate_points_within_the_candidate_lists(gpu_lib):
    # 40 copies of each of 50 points: the 39 ties of a query fit in the candidate lists,
    # so the re-rank orders them by index without the exact scan
    ia = gpu_lib
    rng = np.random.default_rng(4)
    X = np.repeat(rng.random((50, 3)), 40, axis=0)[rng.permutation(2000)]
    ia.iaskit_factor(X, 0.5, 1.0, 64, 16, 1e-8)
    assert np.array_equal(ia.iaskit_get_knn(len(X), 16), oracle.knn_bruteforce(X, 16))


def test_error_codes(gpu_lib):
    ia = gpu_lib
    ia.iaskit_free()
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_solve(np.ones(10))
    assert e.value.name == "IASKIT_ERR_NOT_FACTORED"
    X = np.random.default_rng(3).random((100, 2))
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_factor(X, -1.0, 0.1, 16, 4, 0.0)
    assert e.value.name == "IASKIT_ERR_ARG"
    Xn = X.copy()
    Xn[5, 1] = np.nan
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_factor(Xn, 0.5, 0.1, 16, 4, 0.0)
    assert e.value.name == "IASKIT_ERR_INPUT"
    # identical points and lambda = 0: the leaf blocks are rank one
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_factor(np.zeros((100, 2)), 0.5, 0.0, 16, 4, 0.0)
    assert e.value.name == "IASKIT_ERR_SINGULAR"
    ia.iaskit_factor(X, 0.5, 0.1, 16, 4, 0.0)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_solve(np.full(100, np.inf))
    assert e.value.name == "IASKIT_ERR_INPUT"
