"""Refactoring for a new regularization lambda (Sec. II-C: skeletons and P do not depend
on lambda; only the leaf LUs, W and Z are recomputed).

* After iaskit_refactor(lambda') the skeletons and P are those of the first
  factorization, and the solve matches the oracle's Alg. "Factorize" / "Solve" run on
  those skeletons with lambda' (1e-10 relative, as the plain-path parity tests).
* The refactored solve equals the solve of a fresh factorization with lambda'.
* Mixed form, batched: the condition estimates scale as 1 + (c - 1) lambda / lambda',
  the precision choice follows them, and refinement meets the target.
* Argument errors leave the factorization usable.
"""
import numpy as np
import pytest

import oracle
from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu


@pytest.fixture()
def plain(gpu_lib):
    ia = gpu_lib
    w = workload("C1", N=3001)
    X = make_points(w)
    h, lam, m, s_max, tol = 0.4, 0.1, 50, 24, 1e-6
    ia.iaskit_set_option("seed", 7)
    ia.iaskit_set_option("kappa", 16)
    ia.iaskit_factor(X, h, lam, m, s_max, tol)
    tree, knn, sk, F = oracle.build_all(X, h, lam, m, s_max, tol, kappa=16, seed=7)
    yield dict(ia=ia, X=X, w=w, tree=tree, sk=sk, params=(h, lam, m, s_max, tol))
    ia.iaskit_set_option("seed", 0)


def _skeletons(ia, L):
    return {(l, i): ia.iaskit_get_skeleton(l, i) for l in range(1, L + 1) for i in range(1 << l)}


@pytest.mark.parametrize("lam2", [1.0, 1e-2])
def test_refactor_matches_oracle(plain, lam2):
    ia, tree, sk = plain["ia"], plain["tree"], plain["sk"]
    before = _skeletons(ia, tree.L)
    P_before = ia.iaskit_get_P(2, 1, sk.rank((2, 1)))
    ia.iaskit_refactor(lam2)
    after = _skeletons(ia, tree.L)
    assert all(np.array_equal(before[k], after[k]) for k in before)
    assert np.array_equal(ia.iaskit_get_P(2, 1, sk.rank((2, 1))), P_before)
    u = make_rhs(plain["w"], N=len(plain["X"]), nrhs=2)
    w_gpu = ia.iaskit_solve(u)
    w_ref = oracle.solve(oracle.factorize(sk, lam2), u)
    err = np.linalg.norm(w_gpu - w_ref) / np.linalg.norm(w_ref)
    assert err < 1e-10, err
    assert oracle.residual(sk, lam2, w_gpu, u) < 1e-10
    # the operator applies the new lambda
    r = u - ia.iaskit_apply(w_gpu)
    assert (np.linalg.norm(r, axis=0) / np.linalg.norm(u, axis=0)).max() < 1e-10


def test_refactor_equals_fresh_factorization(plain):
    ia, X = plain["ia"], plain["X"]
    h, lam, m, s_max, tol = plain["params"]
    u = make_rhs(plain["w"], N=len(X), nrhs=3)
    ia.iaskit_refactor(0.5)
    w1 = ia.iaskit_solve(u)
    ia.iaskit_factor(X, h, 0.5, m, s_max, tol)
    w2 = ia.iaskit_solve(u)
    assert np.linalg.norm(w1 - w2) / np.linalg.norm(w2) < 1e-13
    # and back to the first lambda
    ia.iaskit_refactor(lam)
    w3 = ia.iaskit_solve(u)
    w_ref = oracle.solve(oracle.factorize(plain["sk"], lam), u)
    assert np.linalg.norm(w3 - w_ref) / np.linalg.norm(w_ref) < 1e-10


def test_refactor_argument_errors_keep_the_factorization(plain):
    ia = plain["ia"]
    u = make_rhs(plain["w"], N=len(plain["X"]), nrhs=1)
    w0 = ia.iaskit_solve(u)
    for bad in ([0.1, 0.2], [-1.0], [np.nan], [np.inf]):
        with pytest.raises(ia.IaskitError) as e:
            ia.iaskit_refactor(bad)
        assert e.value.name == "IASKIT_ERR_ARG"
    np.testing.assert_array_equal(ia.iaskit_solve(u), w0)
    ia.iaskit_free()
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_refactor(0.1)
    assert e.value.name == "IASKIT_ERR_NOT_FACTORED"


def _uniform(n, seed):
    return np.ascontiguousarray(np.random.default_rng(seed).random((n, 16)))


def test_mixed_batched_refactor_rechooses_precisions(gpu_lib):
    ia = gpu_lib
    Xs = [_uniform(6000, 31), _uniform(3000, 32)]
    hs = [1.2, 0.6]
    ia.iaskit_set_option("precision", 1)
    try:
        ia.iaskit_factor_batched(Xs, hs, [1e-1, 1e-1], 128, 64, 1e-6)
        st0 = ia.iaskit_stats()
        assert st0["fp64_problems"] == 0
        lam2 = [1e-3, 1e-1]
        ia.iaskit_refactor(lam2)
        st = ia.iaskit_stats()
        for q in range(2):
            want = 1.0 + (st0["cond_est"][q] - 1.0) * 1e-1 / lam2[q]
            assert st["cond_est"][q] == pytest.approx(want, rel=1e-9), q
        assert st["cond_est"][0] > 1e6 > st["cond_est"][1]
        assert st["fp64_problems"] == 1
        rng = np.random.default_rng(35)
        rhs = [rng.standard_normal((len(x), 2)) for x in Xs]
        w = ia.iaskit_solve_batched(rhs)
        st = ia.iaskit_stats()
        # residuals against the batched FP64 operator with the new lambdas
        import torch
        W = torch.from_numpy(np.concatenate([x.T.reshape(-1) for x in w])).cuda()
        AW = torch.empty_like(W)
        ia.iaskit_apply_device(W, AW, 2)
        AW = AW.cpu().numpy()
        o = 0
        for q, x in enumerate(Xs):
            n = len(x)
            Au = AW[o:o + 2 * n].reshape(2, n).T
            o += 2 * n
            res = (np.linalg.norm(rhs[q] - Au, axis=0) / np.linalg.norm(rhs[q], axis=0)).max()
            if q == 1:
                assert res <= 1e-10, res
            else:   # the ill-conditioned problem meets the target unless its floor is above it
                assert res <= 1e-10 or (st["refine_stagnated"] >= 1 and res <= 1e-9), res
    finally:
        ia.iaskit_set_option("precision", 0)
