"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test ties one oracle function to something other than itself: a closed
form, a library routine (LAPACK through scipy/numpy), an independent algorithm
(scipy's k-d tree), an invariant of the paper's construction, or brute force on
tiny inputs.
"""
import math
import os
from collections import Counter

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial import cKDTree

import oracle
from oracle.askit import dense_Ktilde, full_P, matvec
from oracle.invaskit import solve_node
from oracle.kernel import gaussian_kernel, sqdist
from oracle.linalg import SingularError, back_substitute, cpqr_id, lu_factor, lu_solve
from oracle.sampling import sample_rows, splitmix64
from oracle.tree import build_tree, knn_bruteforce, node_sizes, tree_depth
from workloads import make_points, make_rhs, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- kernel (eq. gaussian)
def test_kernel_closed_form():
    # ||(0,0) - (3,4)||^2 = 25, h = 5: exp(-25 / 50) = exp(-1/2)
    K = gaussian_kernel(np.array([[0.0, 0.0]]), np.array([[3.0, 4.0]]), 5.0)
    assert K[0, 0] == pytest.approx(math.exp(-0.5), rel=1e-15)
    X = np.random.default_rng(0).random((20, 5))
    K = gaussian_kernel(X, X, 0.7)
    assert np.all(np.diag(K) == 1.0)
    assert np.array_equal(K, K.T)


def test_sqdist_sums_coordinates_in_order():
    # squares 1, 1e-16, 1e-16: summed left to right in FP64 the small terms vanish
    x = np.array([[1.0, 1e-8, 1e-8]])
    assert sqdist(x, np.zeros((1, 3)))[0, 0] == 1.0
    assert (1.0 + (1e-16 + 1e-16)) != 1.0   # another order would differ


# --------------------------------------------------------------------- tree (Sec. II-A)
def _tree_reference(X, m):
    """Independent recursive restatement with Python tuple sorting."""
    N = X.shape[0]
    L = 0
    while math.ceil(N / 2 ** L) > m:
        L += 1

    def split(idx, level):
        if level == L:
            return [sorted(idx)]
        pts = X[idx]
        spread = [pts[:, k].max() - pts[:, k].min() for k in range(X.shape[1])]
        c = spread.index(max(spread))
        keyed = sorted(idx, key=lambda j: (X[j, c], j))
        k = len(idx) // 2
        return split(sorted(keyed[:k]), level + 1) + split(sorted(keyed[k:]), level + 1)

    leaves = split(list(range(N)), 0)
    return L, [j for leaf in leaves for j in leaf]


@pytest.mark.parametrize("N,m,d", [(37, 4, 3), (64, 8, 2), (100, 7, 5), (5, 2, 1)])
def test_tree_matches_bruteforce(N, m, d):
    X = np.random.default_rng(N).random((N, d))
    X[3 % N, 0] = X[1 % N, 0]          # a tie on coordinate values
    T = build_tree(X, m)
    L, perm = _tree_reference(X, m)
    assert T.L == L
    assert list(T.perm) == perm


def test_tree_invariants():
    w = workload("C1", N=3000)
    X = make_points(w)
    T = build_tree(X, 50)
    assert T.L == tree_depth(3000, 50) == 6
    assert np.array_equal(np.sort(T.perm), np.arange(3000))
    sizes = node_sizes(3000, T.L)
    assert sizes[-1].max() <= 50 and sizes[-1].min() >= 1
    for l in range(T.L):
        for i in range(1 << l):
            o, e = T.node_range(l, i)
            idx = T.perm[o:e]
            pts = X[idx]
            spread = pts.max(0) - pts.min(0)
            c = int(T.split_dim[l][i])
            assert spread[c] == spread.max() and np.all(spread[:c] < spread[c])
            ol, el = T.node_range(l + 1, 2 * i)
            assert el - ol == (e - o) // 2
            left, right = T.perm[ol:el], T.perm[el:e]
            kl = max((X[j, c], j) for j in left)
            kr = min((X[j, c], j) for j in right)
            assert kl < kr
    for i in range(1 << T.L):                  # inside a leaf: ascending original index
        o, e = T.node_range(T.L, i)
        assert np.all(np.diff(T.perm[o:e]) > 0)


# ----------------------------------------------------------------------- kNN (Sec. II-B)
def test_knn_lattice_ties_hand_derived():
    X = np.arange(10, dtype=np.float64)[:, None]
    knn = knn_bruteforce(X, 4)
    assert list(knn[5]) == [4, 6, 3, 7]        # distances 1, 1, 4, 4: ties by index
    assert list(knn[0]) == [1, 2, 3, 4]
    assert list(knn[9]) == [8, 7, 6, 5]


def test_knn_matches_kdtree():
    X = np.random.default_rng(3).random((1500, 6))
    knn = knn_bruteforce(X, 16)
    dist, idx = cKDTree(X).query(X, k=17)
    assert np.array_equal(idx[:, 0], np.arange(1500))
    assert np.array_equal(knn, idx[:, 1:])
    d2 = np.sum((X[:, None, :] - X[knn]) ** 2, axis=2)
    np.testing.assert_allclose(np.sqrt(d2), dist[:, 1:], rtol=1e-13)


def test_knn_small_N_caps_kappa():
    X = np.random.default_rng(4).random((5, 2))
    assert knn_bruteforce(X, 16).shape == (5, 4)


# ------------------------------------------------------------------ sampling (Sec. II-B)
def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for state, out in rows:
        assert splitmix64(int(state, 16)) == int(out, 16)


def test_sampling_rules():
    w = workload("C1", N=2000)
    X = make_points(w)
    T = build_tree(X, 64)
    knn = knn_bruteforce(X, 16)
    knn_pos = T.iperm[knn[T.perm]]
    for (l, i) in [(T.L, 0), (T.L, 5), (3, 2), (1, 1)]:
        o, e = T.node_range(l, i)
        n = e - o
        s = sample_rows(knn_pos[o:e], o, n, 2000, 64, 11, (1 << l) + i)
        assert s.size == min(64, 2000 - n)
        assert np.all(np.diff(s) > 0)
        assert not np.any((s >= o) & (s < e))
        # the nearest-neighbour part: an independent recount of the hits
        cnt = Counter(int(c) for c in knn_pos[o:e].ravel() if not (o <= c < e))
        ranked = sorted(cnt.items(), key=lambda kv: (-kv[1], kv[0]))
        top = {c for c, _ in ranked[:64]}
        assert top <= set(s.tolist())
        s2 = sample_rows(knn_pos[o:e], o, n, 2000, 64, 11, (1 << l) + i)
        assert np.array_equal(s, s2)


def test_sampling_uniform_fill_and_complement():
    # no neighbour outside the node: the whole sample comes from the fill
    knn_pos = np.tile(np.arange(10, 20), (10, 1))
    s = sample_rows(knn_pos, 10, 10, 100, 30, 5, 9)
    assert s.size == 30 and not np.any((s >= 10) & (s < 20))
    assert not np.array_equal(s, sample_rows(knn_pos, 10, 10, 100, 30, 6, 9))
    # n_samp >= N - n: the sample is the complement
    s = sample_rows(knn_pos, 10, 10, 25, 40, 5, 9)
    assert list(s) == list(range(10)) + list(range(20, 25))


# -------------------------------------------------------------- LU (GETRF / GETRS)
def test_lu_matches_lapack_getrf():
    A = np.random.default_rng(5).standard_normal((40, 40))
    LU, ipiv = lu_factor(A)
    LU2, piv2 = sla.lu_factor(A)
    assert np.array_equal(ipiv, piv2)
    np.testing.assert_allclose(LU, LU2, rtol=1e-12, atol=1e-12)
    b = np.random.default_rng(6).standard_normal((40, 3))
    np.testing.assert_allclose(lu_solve(LU, ipiv, b), np.linalg.solve(A, b), rtol=1e-10)


def test_lu_zero_pivot_raises():
    with pytest.raises(SingularError):
        lu_factor(np.ones((3, 3)))


def test_back_substitute():
    R = np.triu(np.random.default_rng(7).random((6, 6))) + np.eye(6)
    B = np.random.default_rng(8).random((6, 4))
    np.testing.assert_allclose(R @ back_substitute(R, B), B, atol=1e-13)


# --------------------------------------------------------- CPQR / ID (GEQP3 + GELS)
def test_cpqr_pivots_match_geqp3():
    A = np.random.default_rng(9).standard_normal((30, 20))
    piv, s, P, rdiag, margin = cpqr_id(A, 20, 0.0)
    Q, R, p2 = sla.qr(A, pivoting=True)
    assert margin > 1e-6
    assert list(piv) == list(p2)
    np.testing.assert_allclose(rdiag, np.abs(np.diag(R)), rtol=1e-12)


def test_id_invariants():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((40, 8)) @ rng.standard_normal((8, 25)) + 1e-3 * rng.standard_normal((40, 25))
    piv, s, P, rdiag, _ = cpqr_id(A, 12, 0.0)
    assert s == 12
    np.testing.assert_array_equal(P[:, piv[:s]], np.eye(s))
    # ||A - A(:, J) P||_F equals ||R22||_F of the same pivoted QR (GEQP3)
    Q, R, p2 = sla.qr(A, pivoting=True)
    assert list(p2[:s]) == list(piv[:s])
    err = np.linalg.norm(A - A[:, piv[:s]] @ P)
    assert err == pytest.approx(np.linalg.norm(R[s:, s:]), rel=1e-8)
    # P agrees with the least-squares fit of A on its skeleton columns (GELS)
    Xls = np.linalg.lstsq(A[:, piv[:s]], A, rcond=None)[0]
    np.testing.assert_allclose(P, Xls, atol=1e-8)


def test_id_full_rank_is_permutation():
    A = np.random.default_rng(11).standard_normal((20, 15))
    piv, s, P, _, _ = cpqr_id(A, 100, 0.0)
    assert s == 15
    E = np.zeros((15, 15))
    E[np.arange(15), piv] = 1.0
    np.testing.assert_array_equal(P, E)


def test_id_adaptive_rank_finds_exact_rank():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((50, 7)) @ rng.standard_normal((7, 30))
    _, s, _, _, _ = cpqr_id(A, 30, 1e-9)
    assert s == 7
    _, s, _, _, _ = cpqr_id(A, 5, 1e-9)
    assert s == 5


# ------------------------------------------------- factorization and solve (Sec. II-C)
@pytest.fixture(scope="module")
def small_problem():
    w = workload("C1", N=700)
    X = make_points(w)
    tree, knn, sk, F = oracle.build_all(X, 0.4, 0.5, 40, 12, 0.0, seed=3)
    u = make_rhs(w, N=700, nrhs=2)
    return X, tree, sk, F, u


def test_full_rank_reproduces_dense_lu_solve():
    # s equal to the full node size makes every P a permutation, so K~ = K
    w = workload("C1", N=600)
    X = make_points(w)
    u = make_rhs(w, N=600)[:, 0]
    _, _, sk, F = oracle.build_all(X, 0.5, 1.0, 40, 10 ** 6, 0.0, seed=1)
    K = gaussian_kernel(X, X, 0.5)
    w_dense = np.linalg.solve(np.eye(600) + K, u)
    w_alg = oracle.solve(F, u)
    assert np.linalg.norm(w_alg - w_dense) / np.linalg.norm(w_dense) < 1e-12


def test_algorithm_equals_dense_Ktilde(small_problem):
    X, tree, sk, F, u = small_problem
    w_alg = oracle.solve(F, u)
    w_den = oracle.dense_solve(sk, F.lam, u)
    assert np.linalg.norm(w_alg - w_den) / np.linalg.norm(w_den) < 1e-12
    assert oracle.residual(sk, F.lam, w_alg, u) < 1e-12
    assert oracle.eps_I(F, w_alg[:, 0]) < 1e-12


def test_smw_identity_per_node(small_problem):
    X, tree, sk, F, u = small_problem
    Kt = dense_Ktilde(sk)
    rng = np.random.default_rng(13)
    for l in range(tree.L + 1):
        for i in range(1 << l):
            o, e = tree.node_range(l, i)
            A = F.lam * np.eye(e - o) + Kt[o:e, o:e]
            x = rng.standard_normal(e - o)
            np.testing.assert_allclose(A @ solve_node(F, (l, i), x), x, atol=1e-11)


def test_matvec_equals_dense(small_problem):
    X, tree, sk, F, u = small_problem
    Kt = dense_Ktilde(sk)
    wp = np.random.default_rng(14).standard_normal((700, 3))
    np.testing.assert_allclose(matvec(sk, 0.5, wp), 0.5 * wp + Kt @ wp, rtol=1e-12, atol=1e-12)


def test_nested_P_is_identity_on_skeletons(small_problem):
    X, tree, sk, F, u = small_problem
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            o, e = tree.node_range(l, i)
            Pf = full_P(sk, (l, i))
            assert Pf.shape == (sk.rank((l, i)), e - o)
            np.testing.assert_allclose(Pf[:, sk.skel[(l, i)] - o], np.eye(sk.rank((l, i))), atol=1e-12)


def test_offdiagonal_blocks_follow_the_definition(small_problem):
    # K~ restricted to (l, r) is K_{l r~} P_{r~ r} (eq. offdiag-askit), never the exact K_{lr}
    X, tree, sk, F, u = small_problem
    Kt = dense_Ktilde(sk)
    ol, el = tree.node_range(1, 0)
    orr, er = tree.node_range(1, 1)
    Klr = gaussian_kernel(sk.Xp[ol:el], sk.Xp[sk.skel[(1, 1)]], sk.h) @ full_P(sk, (1, 1))
    np.testing.assert_allclose(Kt[ol:el, orr:er], Klr, rtol=1e-13, atol=1e-15)
    # the columns at the skeletons are exact kernel values
    sk_cols = sk.skel[(1, 1)]
    np.testing.assert_allclose(Kt[ol:el, sk_cols], gaussian_kernel(sk.Xp[ol:el], sk.Xp[sk_cols], sk.h),
                               rtol=1e-12, atol=1e-15)


def test_single_leaf_problem_is_dense_lu():
    X = np.random.default_rng(15).random((30, 3))
    u = np.random.default_rng(16).standard_normal(30)
    _, _, sk, F = oracle.build_all(X, 0.5, 0.1, 64, 8, 0.0)
    assert sk.tree.L == 0
    w = oracle.solve(F, u)
    A = 0.1 * np.eye(30) + gaussian_kernel(X, X, 0.5)
    assert np.linalg.norm(A @ w - u) / np.linalg.norm(u) < 1e-12


def test_new_lambda_reuses_skeletons(small_problem):
    # Sec. II-C: skeletons and P do not depend on lambda; a factorization for a new
    # lambda on the same skeletons inverts lambda' I + K~ (dense solve of that matrix)
    X, tree, sk, F, u = small_problem
    _, _, sk2, _ = oracle.build_all(X, 0.4, 3.0, 40, 12, 0.0, seed=3)
    for node in sk.skel:
        assert np.array_equal(sk.skel[node], sk2.skel[node])
        np.testing.assert_array_equal(sk.P[node], sk2.P[node])
    for lam2 in (1e-3, 2.0):
        F2 = oracle.factorize(sk, lam2)
        w = oracle.solve(F2, u)
        w_den = oracle.dense_solve(sk, lam2, u)
        assert np.linalg.norm(w - w_den) / np.linalg.norm(w_den) < 1e-10, lam2


# ------------------------------------------------- sampled eps_M (eq. error, Sec. III)
def _dense_K_original(X, h):
    """Exact kernel matrix in ORIGINAL order from scipy's distances (not the oracle's)."""
    from scipy.spatial.distance import cdist
    return np.exp(-cdist(X, X, "sqeuclidean") / (2.0 * h * h))


def _dense_Ktilde_original(sk):
    """The dense K~ of the oracle (permuted order) brought back to ORIGINAL order."""
    perm = sk.tree.perm
    Kt = dense_Ktilde(sk)
    out = np.empty_like(Kt)
    out[np.ix_(perm, perm)] = Kt
    return out


def test_eps_M_sampled_on_all_rows_is_the_dense_definition(small_problem):
    # eq. error with S = 0: eps_M = ||K w - K~ w|| / ||K w||, K~ without lambda, both
    # in original order.  Pinned against K from scipy's cdist and the dense K~.
    X, tree, sk, F, u = small_problem
    w = np.random.default_rng(21).standard_normal(X.shape[0])
    K = _dense_K_original(X, sk.h)
    Kt = _dense_Ktilde_original(sk)
    want = np.linalg.norm(K @ w - Kt @ w) / np.linalg.norm(K @ w)
    got = oracle.eps_M_sampled(sk, X, w, np.arange(X.shape[0]))
    assert want > 1e-8          # a low-rank K~ differs from K
    assert got == pytest.approx(want, rel=1e-9)
    # a subset of rows: the same quotient restricted to those rows
    rows = np.sort(np.random.default_rng(22).choice(X.shape[0], 100, replace=False))
    want_r = np.linalg.norm((K @ w - Kt @ w)[rows]) / np.linalg.norm((K @ w)[rows])
    assert oracle.eps_M_sampled(sk, X, w, rows) == pytest.approx(want_r, rel=1e-9)
    # a plausible slip would show: lambda inside K~, or rows read in permuted order
    slip_lam = np.linalg.norm((K @ w - (Kt @ w + F.lam * w))[rows]) / np.linalg.norm((K @ w)[rows])
    slip_perm = np.linalg.norm((K @ w)[rows] - (Kt @ w)[tree.perm[rows]]) / np.linalg.norm((K @ w)[rows])
    for slip in (slip_lam, slip_perm):
        assert abs(slip - want_r) > 1e-3 * want_r


def test_eps_M_is_zero_at_full_rank():
    # s = the full node size: every P is a permutation, K~ = K and eps_M vanishes
    w_ = workload("C1", N=500)
    X = make_points(w_)
    _, _, sk, _ = oracle.build_all(X, 0.5, 1.0, 40, 10 ** 6, 0.0, seed=2)
    w = np.random.default_rng(23).standard_normal(500)
    assert oracle.eps_M_sampled(sk, X, w, np.arange(500)) < 1e-13
