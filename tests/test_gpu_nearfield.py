"""The kNN-separated operator lambda I + K~ + S (eq. askit, Sec. II-B) on the GPU.

The oracle side runs on the library's own skeletons and P (read back through the ABI),
so each check covers the near-field part itself, whatever pivot near-ties the sampled
blocks hold (skeleton parity has its own tests).

* The operator apply with option "near_field" matches the oracle's matvec_knn (the
  Evaluate step with exact evaluation of the nodes holding a target's nearest
  neighbours) to 1e-10 relative (FP64 on both sides), for one problem and for a batch
  of two (per-problem offsets); S w is far above rounding on these inputs.
* GMRES on lambda I + K~ + S preconditioned by the factorization of lambda I + K~ (the
  paper's use of INV-ASKIT for K~ + S): to 1e-10 in the plain and mixed forms, and to
  the paper's rho < 1e-3 within 100 iterations on a case where S w is 20% of K~ w.
"""
import numpy as np
import pytest

import oracle
from oracle.nearfield import matvec_knn
from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu


def _oracle_apply(tree, sk, lam, knn, w):
    """matvec_knn in the original point order."""
    knn_pos = tree.iperm[knn[tree.perm]]
    up = matvec_knn(sk, lam, np.asarray(w)[tree.perm], knn_pos)
    u = np.empty_like(up)
    u[tree.perm] = up
    return u


def _gpu_skeletons(ia, X, h, m, q=0):
    """The oracle's tree with the library's skeletons and P of problem q (read back), so
    that the oracle's operator is the one the library built, whatever pivot near-ties
    the sampled blocks hold."""
    from oracle.askit import Skeletons
    ia.iaskit_set_option("problem", q)
    tree = oracle.build_tree(X, m)
    assert np.array_equal(ia.iaskit_get_perm(len(X)), tree.perm)
    sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
    ranks = ia.iaskit_get_ranks()
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
            sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
    ia.iaskit_set_option("problem", 0)
    return tree, sk


def _rho(u, Au):
    return (np.linalg.norm(u - Au, axis=0) / np.linalg.norm(u, axis=0)).max()


@pytest.fixture()
def opts(gpu_lib):
    yield gpu_lib
    for k, v in (("near_field", 0), ("refine", 0), ("refine_tol", 1e-10), ("precision", 0), ("seed", 0)):
        gpu_lib.iaskit_set_option(k, v)


def test_near_field_apply_matches_oracle(opts):
    """C1, 3001 points (d 8), h 0.4, lambda 0.1, m 50, s_max 24: S w is half of K~ w."""
    ia = opts
    w = workload("C1", N=3001)
    X = make_points(w)
    h, lam, m = 0.4, 0.1, 50
    ia.iaskit_set_option("seed", 7)
    ia.iaskit_factor(X, h, lam, m, 24, 1e-6)
    tree, sk = _gpu_skeletons(ia, X, h, m)
    knn = oracle.knn_bruteforce(X, 16)
    v = make_rhs(w, N=len(X), nrhs=3)
    u0 = ia.iaskit_apply(v)
    ia.iaskit_set_option("near_field", 1)
    assert ia.iaskit_get_option("near_field") == 1.0
    u = ia.iaskit_apply(v)
    ref = _oracle_apply(tree, sk, lam, knn, v)
    err = np.linalg.norm(u - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() < 1e-10, err
    diff = np.linalg.norm(u - u0, axis=0) / np.linalg.norm(u0, axis=0)
    print("relative size of S w:", diff)
    assert diff.min() > 1e-2


def test_near_field_gmres_plain(opts):
    """C2 generator, 3000 points (d 54), h 1.0, lambda 1e-2: |S w| / |K~ w| about 4%;
    preconditioned GMRES to 1e-10 (about 25 iterations)."""
    ia = opts
    w = workload("C2", N=3000)
    X = make_points(w)
    h, lam, m = 1.0, 1e-2, 128
    ia.iaskit_factor(X, h, lam, m, 48, 1e-5)
    tree, sk = _gpu_skeletons(ia, X, h, m)
    knn = oracle.knn_bruteforce(X, 16)
    u = make_rhs(w, N=len(X), nrhs=2)
    ia.iaskit_set_option("near_field", 1)
    ia.iaskit_set_option("refine", 100)
    ia.iaskit_set_option("refine_tol", 1e-10)
    sol = ia.iaskit_solve(u)
    st = ia.iaskit_stats()
    assert st["refine_iters"] >= 2
    assert _rho(u, ia.iaskit_apply(sol)) <= 1e-10
    rho = _rho(u, _oracle_apply(tree, sk, lam, knn, sol))
    assert rho < 1e-9, rho
    print("GMRES iterations with S:", st["refine_iters"])


def test_near_field_gmres_paper_tolerance(opts):
    """The paper's use: GMRES with INV-ASKIT as the preconditioner to rho < 1e-3 within
    100 iterations; C1, 3001 points, h 0.2, s_max 48, tau 1e-8 (|S w| / |K~ w| about 20%)."""
    ia = opts
    w = workload("C1", N=3001)
    X = make_points(w)
    h, lam, m = 0.2, 0.1, 50
    ia.iaskit_set_option("seed", 7)
    ia.iaskit_factor(X, h, lam, m, 48, 1e-8)
    tree, sk = _gpu_skeletons(ia, X, h, m)
    knn = oracle.knn_bruteforce(X, 16)
    u = make_rhs(w, N=len(X), nrhs=1)
    ia.iaskit_set_option("near_field", 1)
    ia.iaskit_set_option("refine", 100)
    ia.iaskit_set_option("refine_tol", 1e-3)
    sol = ia.iaskit_solve(u)
    st = ia.iaskit_stats()
    assert 1 <= st["refine_iters"] <= 100
    rho = _rho(u, _oracle_apply(tree, sk, lam, knn, sol))
    assert rho < 1e-3, rho
    print("GMRES iterations to 1e-3:", st["refine_iters"], "rho", rho)


def test_near_field_gmres_mixed(opts):
    ia = opts
    w = workload("C2", N=6000)
    X = make_points(w)
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("refine", 200)
    ia.iaskit_factor(X, 1.0, 1e-2, 128, 48, 1e-5)
    ia.iaskit_set_option("near_field", 1)
    u = make_rhs(w, N=len(X), nrhs=2)
    sol = ia.iaskit_solve(u)
    assert _rho(u, ia.iaskit_apply(sol)) <= 1e-10


def test_near_field_batched(opts):
    """Two problems in one batch (per-problem offsets of the near-field kernel)."""
    ia = opts
    import torch
    probs = []
    for N, seed in ((1500, 1), (2100, 2)):
        X = np.random.default_rng(seed).random((N, 3))
        probs.append((X, 0.3 if seed == 1 else 0.5, 0.1))
    m, s_max, tol = 40, 20, 1e-6
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             m, s_max, tol)
    sks = [_gpu_skeletons(ia, X, h, m, q) for q, (X, h, lam) in enumerate(probs)]
    ia.iaskit_set_option("near_field", 1)
    rng = np.random.default_rng(3)
    ws = [rng.standard_normal((len(p[0]), 2)) for p in probs]
    W = torch.from_numpy(np.concatenate([x.T.reshape(-1) for x in ws])).cuda()
    U = torch.empty_like(W)
    ia.iaskit_apply_device(W, U, 2)
    U = U.cpu().numpy()
    o = 0
    for (X, h, lam), w, (tree, sk) in zip(probs, ws, sks):
        n = len(X)
        got = U[o:o + 2 * n].reshape(2, n).T
        o += 2 * n
        ref = _oracle_apply(tree, sk, lam, oracle.knn_bruteforce(X, 16), w)
        err = (np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()
        assert err < 1e-10, err
