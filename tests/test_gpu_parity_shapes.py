"""Parity with the oracle at the tile shapes the benchmark runs (Alg. Factorize / Solve).

The small parity cases use leaves of at most 64 points and ranks of at most 32; these
cases reach the large-block paths: leaves of 512 and 1024 points, ranks 256 and 512,
sampled blocks of 512 x 512 and 1024 x 1024 (16- and 32-panel LUs, long substitution
chains, the 256 x 16 and tensor-core product tiles, and in the mixed form the
cluster-of-blocks ID of levels with at most 32 nodes).

* FP64 path, mixture in d = 54 (m 512, s_max 256, n_samp 512, tau 1e-5; N = 8192, L 4)
  and mixture in d = 8 (m 1024, s_max 512, n_samp 1024, tau 1e-7; N = 4096, L 2, the
  smallest N with two levels): kNN, samples and skeletons bit-exact (the inputs have no
  pivot near-tie), P, the solve and the operator within 1e-10 of the oracle.
* Mixed form at the d = 54 shape: its operator equals the oracle's MatVec on the
  library's own skeletons and P (1e-12), the refined solve meets 1e-10 against it, and
  every FP32 interpolative decomposition is within a factor 1.5 (plus FP32 rounding) of
  the oracle's FP64 CPQR at the same rank on the same sampled block.
"""
import numpy as np
import pytest

import oracle
from oracle.askit import Skeletons
from oracle.kernel import gaussian_kernel
from oracle.linalg import cpqr_id
from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu

RTOL = 1e-10
SHAPES = {
    # name: (generator, N, h, lambda, m, s_max, tol, nrhs)
    "d54_m512_s256": ("C2", 8192, 1.0, 1e-2, 512, 256, 1e-5, 2),
    "d8_m1024_s512": ("C5", 4096, 0.35, 1.0, 1024, 512, 1e-7, 2),
}


@pytest.fixture(scope="module", params=sorted(SHAPES))
def shape(request, gpu_lib):
    ia = gpu_lib
    gname, N, h, lam, m, s_max, tol, nrhs = SHAPES[request.param]
    X = make_points(workload(gname, N=N))
    u = make_rhs(workload(gname, N=N), N=N, nrhs=nrhs)
    ia.iaskit_set_option("seed", 7)
    ia.iaskit_set_option("precision", 0)
    ia.iaskit_factor(X, h, lam, m, s_max, tol)
    got = {"knn": ia.iaskit_get_knn(N, 16), "perm": ia.iaskit_get_perm(N), "ranks": ia.iaskit_get_ranks(),
           "w": ia.iaskit_solve(u), "Au": ia.iaskit_apply(u)}
    L = ia.iaskit_depth()
    got["skel"] = {(l, i): ia.iaskit_get_skeleton(l, i) for l in range(1, L + 1) for i in range(1 << l)}
    got["samp"] = {(l, i): ia.iaskit_get_samples(l, i) for l in range(1, L + 1) for i in range(1 << l)}
    got["P"] = {k: ia.iaskit_get_P(k[0], k[1], len(v)) for k, v in got["skel"].items()}
    tree, knn, sk, F = oracle.build_all(X, h, lam, m, s_max, tol, seed=7)
    ia.iaskit_set_option("seed", 0)
    return dict(name=request.param, X=X, u=u, got=got, tree=tree, knn=knn, sk=sk, F=F, lam=lam)


def test_indices_bitexact(shape):
    g, tree, sk = shape["got"], shape["tree"], shape["sk"]
    assert min(sk.margin.values()) > 1e-9
    assert np.array_equal(g["perm"], tree.perm)
    assert np.array_equal(g["knn"], shape["knn"])
    for node in sk.skel:
        assert np.array_equal(g["samp"][node], sk.samp[node]), node
        assert g["ranks"][(1 << node[0]) + node[1]] == sk.rank(node), node
        assert np.array_equal(g["skel"][node], sk.skel[node]), node


def test_P_solve_and_operator(shape):
    g, sk, F = shape["got"], shape["sk"], shape["F"]
    for node in sk.skel:
        np.testing.assert_allclose(g["P"][node], sk.P[node], rtol=RTOL, atol=RTOL * np.abs(sk.P[node]).max())
    w_ref = oracle.solve(F, shape["u"])
    assert np.linalg.norm(g["w"] - w_ref) / np.linalg.norm(w_ref) < RTOL
    Au_ref = oracle.invaskit.apply_operator(sk, shape["lam"], shape["u"])
    assert np.linalg.norm(g["Au"] - Au_ref) / np.linalg.norm(Au_ref) < RTOL


@pytest.fixture(scope="module")
def mixed_shape(gpu_lib):
    ia = gpu_lib
    gname, N, h, lam, m, s_max, tol, nrhs = SHAPES["d54_m512_s256"]
    X = make_points(workload(gname, N=N))
    u = make_rhs(workload(gname, N=N), N=N, nrhs=nrhs)
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("refine", 200)
    try:
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        w = ia.iaskit_solve(u)
        st = ia.iaskit_stats()
        probe = np.random.default_rng(9).standard_normal((N, 2))
        Au = ia.iaskit_apply(probe)
        tree = oracle.build_tree(X, m)
        sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
        ranks = ia.iaskit_get_ranks()
        samp = {}
        for l in range(1, tree.L + 1):
            for i in range(1 << l):
                sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
                sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
                samp[(l, i)] = ia.iaskit_get_samples(l, i).astype(np.int64)
    finally:
        ia.iaskit_set_option("precision", 0)
        ia.iaskit_set_option("refine", 0)
    return dict(X=X, u=u, w=w, st=st, probe=probe, Au=Au, sk=sk, samp=samp, tree=tree, lam=lam, h=h, s_max=s_max)


def test_mixed_operator_and_residual_at_shape(mixed_shape):
    c = mixed_shape
    ref = oracle.invaskit.apply_operator(c["sk"], c["lam"], c["probe"])
    assert np.linalg.norm(c["Au"] - ref) / np.linalg.norm(ref) < 1e-12
    assert oracle.residual(c["sk"], c["lam"], c["w"], c["u"]) <= 1e-10


def test_mixed_ids_against_fp64_cpqr_at_equal_rank(mixed_shape):
    c = mixed_shape
    sk, tree, Xp, h = c["sk"], c["tree"], c["sk"].Xp, c["h"]
    worst = 0.0
    for (l, i), skel in sk.skel.items():
        if l == tree.L:
            o, e = tree.node_range(l, i)
            cols = np.arange(o, e)
        else:
            cols = np.concatenate([sk.skel[(l + 1, 2 * i)], sk.skel[(l + 1, 2 * i + 1)]])
        A = gaussian_kernel(Xp[c["samp"][(l, i)]], Xp[cols], h)
        s = len(skel)
        J = np.searchsorted(cols, skel) if l == tree.L else np.array([list(cols).index(j) for j in skel])
        err_gpu = np.linalg.norm(A - A[:, J] @ sk.P[(l, i)])
        piv, s_or, P_or, _, _ = cpqr_id(A, s, 0.0)
        err_or = np.linalg.norm(A - A[:, piv[:s_or]] @ P_or)
        ratio = err_gpu / (1.5 * err_or + 1e-5 * np.linalg.norm(A))
        worst = max(worst, ratio)
        assert ratio <= 1.0, ((l, i), err_gpu, err_or)
    print(f"FP32 ID error / (1.5 x FP64 CPQR error + FP32 floor): largest {worst:.3f}")
