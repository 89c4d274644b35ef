"""Batched factorization of independent problems (grouped per-height launches).

Every problem of a batch must get exactly what it gets alone: the same tree, kNN
lists, samples, skeletons and P (bit-exact), and the same solution; and each must
match the oracle run on that problem by itself.
"""
import numpy as np
import pytest

import oracle
from workloads import batched_problems

pytestmark = pytest.mark.gpu


def _batch():
    probs = batched_problems(count=6, scale=1.0 / 16)       # N_i in [128, 4096]
    probs = [(X, h, lam) for X, h, lam in probs]
    probs.append((np.random.default_rng(9).random((50, 16)), 0.6, 0.1))   # one-leaf tree
    return probs


@pytest.fixture(scope="module")
def batched(gpu_lib):
    ia = gpu_lib
    probs = _batch()
    m, s_max, tol = 64, 24, 1e-6
    rng = np.random.default_rng(21)
    rhs = [rng.standard_normal((len(X), 2)) for X, _, _ in probs]
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             m, s_max, tol)
    assert ia.iaskit_num_problems() == len(probs)
    w = ia.iaskit_solve_batched(rhs)
    per = []
    for q in range(len(probs)):
        ia.iaskit_set_option("problem", q)
        L = ia.iaskit_depth()
        item = {"perm": ia.iaskit_get_perm(len(probs[q][0])), "L": L}
        if L > 0:
            item["knn"] = ia.iaskit_get_knn(len(probs[q][0]), 16)
            ranks = ia.iaskit_get_ranks()
            item["skel"] = {(l, i): ia.iaskit_get_skeleton(l, i)
                            for l in range(1, L + 1) for i in range(1 << l)}
            item["samp"] = {(l, i): ia.iaskit_get_samples(l, i)
                            for l in range(1, L + 1) for i in range(1 << l)}
            item["P"] = {(l, i): ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
                         for l in range(1, L + 1) for i in range(1 << l)}
        per.append(item)
    ia.iaskit_set_option("problem", 0)
    return dict(ia=ia, probs=probs, rhs=rhs, w=w, per=per, params=(m, s_max, tol))


def test_batched_matches_oracle_per_problem(batched):
    m, s_max, tol = batched["params"]
    for q, (X, h, lam) in enumerate(batched["probs"]):
        tree, knn, sk, F = oracle.build_all(X, h, lam, m, s_max, tol)
        got = batched["per"][q]
        assert got["L"] == tree.L
        assert np.array_equal(got["perm"], tree.perm), q
        if tree.L > 0:
            assert np.array_equal(got["knn"], knn), q
            for node, s in sk.samp.items():
                assert np.array_equal(got["samp"][node], s), (q, node)
            if min(sk.margin.values()) > 1e-9:
                for node in sk.skel:
                    assert np.array_equal(got["skel"][node], sk.skel[node]), (q, node)
                    np.testing.assert_allclose(got["P"][node], sk.P[node], rtol=1e-10,
                                               atol=1e-10 * np.abs(sk.P[node]).max())
        w_ref = oracle.solve(F, batched["rhs"][q])
        err = np.linalg.norm(batched["w"][q] - w_ref) / np.linalg.norm(w_ref)
        assert err < 1e-10, (q, err)


def test_batched_equals_single_problem_runs(batched):
    ia = batched["ia"]
    m, s_max, tol = batched["params"]
    for q, (X, h, lam) in enumerate(batched["probs"]):
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        w1 = ia.iaskit_solve(batched["rhs"][q])
        assert np.array_equal(ia.iaskit_get_perm(len(X)), batched["per"][q]["perm"])
        err = np.linalg.norm(w1 - batched["w"][q]) / np.linalg.norm(w1)
        assert err < 1e-13, (q, err)


def test_batched_mixed_refines_every_problem(gpu_lib):
    from oracle.askit import Skeletons
    ia = gpu_lib
    probs = _batch()
    rng = np.random.default_rng(22)
    rhs = [rng.standard_normal((len(X), 3)) for X, _, _ in probs]
    ia.iaskit_set_option("precision", 1)
    try:
        ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs],
                                 [p[2] for p in probs], 64, 24, 1e-6)
        w = ia.iaskit_solve_batched(rhs)
        assert ia.iaskit_stats()["refine_history"][-1] <= 1e-10
        for q, (X, h, lam) in enumerate(probs):
            # the oracle's MatVec of this problem's K~ (GPU skeletons and P) checks the residual
            ia.iaskit_set_option("problem", q)
            tree = oracle.build_tree(X, 64)
            sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
            if tree.L > 0:
                ranks = ia.iaskit_get_ranks()
                for l in range(1, tree.L + 1):
                    for i in range(1 << l):
                        sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
                        sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
            rho = oracle.residual(sk, lam, w[q], rhs[q])
            assert rho <= 1e-10, (q, rho)
    finally:
        ia.iaskit_set_option("problem", 0)
        ia.iaskit_set_option("precision", 0)
