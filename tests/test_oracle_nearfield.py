"""Pins of the oracle's kNN-separated operator lambda I + K~ + S (eq. askit, Sec. II-B).

* interaction_node against brute force over the tree's node ranges: the node holds q,
  not p, and its parent holds both; None exactly when p and q share a leaf.
* matvec_knn (the Evaluate recursion, target by target) against dense_Ktilde_knn (the
  matrix entry by entry): two independent restatements of the same definition.
* Special cases with closed forms: neighbour lists inside each point's own leaf give
  S = 0 (the i-not-in-alpha operator, askit.matvec); lists holding every other point
  make every node of every list exact, so K~ + S = K, the dense kernel matrix.
* S is zero outside the (target, node) pairs whose node holds a neighbour, and equals
  K_{i a} - K_{i a~} P_{a~ a} on them.
"""
import numpy as np
import pytest

import oracle
from oracle.askit import dense_Ktilde, matvec
from oracle.kernel import gaussian_kernel
from oracle.nearfield import S_block, dense_Ktilde_knn, interaction_node, matvec_knn, near_nodes


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(41)
    X = rng.random((160, 3))
    h, lam, m, s_max, tol = 0.35, 1e-2, 20, 12, 0.0
    tree, knn, sk, F = oracle.build_all(X, h, lam, m, s_max, tol, kappa=5, seed=3)
    knn_pos = tree.iperm[knn[tree.perm]]
    return dict(X=X, h=h, lam=lam, tree=tree, sk=sk, knn_pos=knn_pos)


def _leaf_of(tree, p):
    for i in range(1 << tree.L):
        o, e = tree.node_range(tree.L, i)
        if o <= p < e:
            return i


def test_interaction_node_brute_force(small):
    tree = small["tree"]
    assert tree.L == 3
    for p in range(0, tree.N, 7):
        for q in range(tree.N):
            a = interaction_node(tree, p, q)
            if _leaf_of(tree, p) == _leaf_of(tree, q):
                assert a is None
                continue
            l, i = a
            o, e = tree.node_range(l, i)
            po, pe = tree.node_range(l - 1, i // 2)
            assert o <= q < e and not (o <= p < e) and po <= p < pe and po <= q < pe


def test_matvec_matches_entrywise_definition(small):
    sk, lam, knn_pos = small["sk"], small["lam"], small["knn_pos"]
    w = np.random.default_rng(42).standard_normal((small["tree"].N, 2))
    A = lam * np.eye(small["tree"].N) + dense_Ktilde_knn(sk, knn_pos)
    np.testing.assert_allclose(matvec_knn(sk, lam, w, knn_pos), A @ w, rtol=1e-12, atol=1e-12)
    # some targets have neighbours outside their leaf, so S is not zero here
    assert sum(len(near_nodes(small["tree"], p, knn_pos)) for p in range(small["tree"].N)) > 0


def test_lists_inside_the_leaf_give_the_first_criterion(small):
    tree, sk, lam = small["tree"], small["sk"], small["lam"]
    own = np.zeros((tree.N, 2), dtype=np.int64)
    for i in range(1 << tree.L):
        o, e = tree.node_range(tree.L, i)
        own[o:e, 0] = o
        own[o:e, 1] = e - 1
    w = np.random.default_rng(43).standard_normal(tree.N)
    np.testing.assert_allclose(matvec_knn(sk, lam, w, own), matvec(sk, lam, w), rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(dense_Ktilde_knn(sk, own), dense_Ktilde(sk))


def test_full_lists_give_the_dense_kernel(small):
    tree, sk, lam = small["tree"], small["sk"], small["lam"]
    allq = np.tile(np.arange(tree.N), (tree.N, 1))
    K = gaussian_kernel(sk.Xp, sk.Xp, sk.h)
    np.testing.assert_array_equal(dense_Ktilde_knn(sk, allq), K)
    w = np.random.default_rng(44).standard_normal(tree.N)
    np.testing.assert_allclose(matvec_knn(sk, lam, w, allq), lam * w + K @ w, rtol=1e-12, atol=1e-12)


def test_S_blocks(small):
    tree, sk, knn_pos = small["tree"], small["sk"], small["knn_pos"]
    S = dense_Ktilde_knn(sk, knn_pos) - dense_Ktilde(sk)
    seen = 0
    for p in range(tree.N):
        near = near_nodes(tree, p, knn_pos)
        mask = np.zeros(tree.N, dtype=bool)
        for a in near:
            o, e = tree.node_range(*a)
            mask[o:e] = True
            np.testing.assert_allclose(S[p, o:e], S_block(sk, p, a), rtol=0, atol=1e-13)
            seen += 1
        assert np.all(S[p, ~mask] == 0.0)
    assert seen > 0
