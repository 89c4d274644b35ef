"""The kNN lists of the pruned tree-order search (option "knn_prune" = 1, the default)
are bit for bit those of the brute-force search over every pair and of the oracle's
definition (Sec. II-B input: kappa nearest other points by (FP64 squared distance in
coordinate order, original index)).

Cases: low-dimensional clouds where most point tiles are skipped, clustered and
high-dimensional ones where few are (at these sizes), the three widths of the candidate
lists (kappa <= 16, <= 24, > 24), a problem of fewer than eight tiles (nothing to
prune), a batch of two problems, and ties at exactly equal distances (a lattice).  The oracle recomputes sampled rows one by one; the brute-force
GPU search (itself pinned to the oracle on every row at small sizes) checks all rows.
"""
import numpy as np
import pytest

from oracle.kernel import sqdist
from workloads import make_points, workload

pytestmark = pytest.mark.gpu


def _oracle_rows(X, rows, kappa):
    D = sqdist(X[rows], X)
    D[np.arange(len(rows)), rows] = np.inf
    return np.argsort(D, axis=1, kind="stable")[:, :kappa]


def _lists(ia, X, m, kappa, prune):
    ia.iaskit_set_option("knn_prune", prune)
    ia.iaskit_set_option("kappa", kappa)
    ia.iaskit_factor(X, 0.5, 1.0, m, 8, 0.0)
    st = ia.iaskit_stats()
    return ia.iaskit_get_knn(len(X), kappa), st


def _lattice(n_side, d):
    g = np.stack(np.meshgrid(*[np.arange(n_side, dtype=np.float64)] * d, indexing="ij"), -1).reshape(-1, d)
    return g[np.random.default_rng(3).permutation(len(g))] * 0.25


CASES = {
    # name: (points, leaf m, kappa, largest fraction of the pairs the search may scan)
    "gmm_d8_k16": (lambda: make_points(workload("C5", N=20000)), 1024, 16, 1.1),
    "gmm_d54_k16": (lambda: make_points(workload("C2", N=12000)), 512, 16, 1.1),
    "manifold_d64_k24": (lambda: make_points(workload("C4", N=9000)), 512, 24, 1.1),
    "uniform_d3_k40": (lambda: np.random.default_rng(5).random((9000, 3)), 64, 40, 0.5),
    "uniform_d2_k16": (lambda: np.random.default_rng(9).random((50000, 2)), 256, 16, 0.05),
    "small_k16": (lambda: np.random.default_rng(6).random((700, 5)), 64, 16, 1.1),
    "lattice_ties_k16": (lambda: _lattice(13, 3), 128, 16, 0.95),
}


@pytest.fixture()
def opts(gpu_lib):
    yield gpu_lib
    gpu_lib.iaskit_set_option("knn_prune", 1)
    gpu_lib.iaskit_set_option("kappa", 16)


@pytest.mark.parametrize("name", sorted(CASES))
def test_pruned_lists_are_exact(opts, name):
    ia = opts
    make, m, kappa, most = CASES[name]
    X = np.ascontiguousarray(make())
    pruned, st = _lists(ia, X, m, kappa, 1)
    brute, _ = _lists(ia, X, m, kappa, 0)
    assert np.array_equal(pruned, brute)
    rows = np.sort(np.random.default_rng(7).choice(len(X), min(300, len(X)), replace=False))
    assert np.array_equal(pruned[rows], _oracle_rows(X, rows, kappa))
    frac = st["knn_pairs_scanned"] / st["knn_pairs_all"]
    print(f"{name}: scanned {frac:.3f} of all pairs, exact fallback rows {st['knn_fallback']}")
    assert frac < most   # the seed tiles of small problems count whole 128-row tiles


def test_pruned_lists_of_a_batch(opts):
    ia = opts
    rng = np.random.default_rng(8)
    Xs = [make_points(workload("C5", N=6000)), rng.random((4100, 8)) * 3.0]
    for prune in (1, 0):
        ia.iaskit_set_option("knn_prune", prune)
        ia.iaskit_factor_batched(Xs, [0.3, 0.5], [1.0, 1.0], 256, 8, 0.0)
        got = []
        for q in (0, 1):
            ia.iaskit_set_option("problem", q)
            got.append(ia.iaskit_get_knn(len(Xs[q]), 16))
        ia.iaskit_set_option("problem", 0)
        if prune:
            first = got
    for q in (0, 1):
        assert np.array_equal(first[q], got[q])
        rows = np.arange(0, len(Xs[q]), 37)
        assert np.array_equal(first[q][rows], _oracle_rows(Xs[q], rows, 16))
