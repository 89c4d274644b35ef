"""The polynomial kernel (option "kernel" = 1: K(x, y) = (x . y / h^2 + poly_c)^poly_p;
Sec. IV reports tests with a polynomial kernel without its degree or constants) on the
GPU, against the oracle's polynomial kernel.

* Kernel blocks in FP64, on FP32 pairs and in FP32 against the closed form.
* The FP64 path: tree, kNN lists, samples and skeletons bit-exact, P, the solve, the
  operator and the exact kernel sums at test points within 1e-10 of the oracle; the
  degree-2 kernel on d = 3 points has rank at most 10, so the skeletons reproduce K.
* The mixed form refines to 1e-10 against its own operator (checked by the oracle).
* Learned sampling, built for the Gaussian, refuses the polynomial kernel.
"""
import numpy as np
import pytest

import oracle
from oracle.askit import Skeletons
from oracle.kernel import PolynomialKernel, polynomial_kernel
from oracle.regression import scores

pytestmark = pytest.mark.gpu

P_DEG, P_C, H = 2, 1.0, 1.0


@pytest.fixture()
def poly(gpu_lib):
    ia = gpu_lib
    ia.iaskit_set_option("kernel", 1)
    ia.iaskit_set_option("poly_p", P_DEG)
    ia.iaskit_set_option("poly_c", P_C)
    yield ia
    for k, v in (("kernel", 0), ("poly_p", 2), ("poly_c", 1.0), ("precision", 0), ("refine", 0), ("sampling", 0)):
        ia.iaskit_set_option(k, v)


def test_kernel_blocks(poly):
    ia = poly
    X = np.random.default_rng(81).random((300, 5)) * 2 - 0.5
    rows, cols = np.arange(0, 300, 3), np.arange(1, 300, 2)
    want = polynomial_kernel(X[rows], X[cols], 0.8, P_DEG, P_C)
    for form, tol in (("fp64", 1e-13), ("pair", 1e-12), ("fp32", 2e-6)):
        got = ia.iaskit_kernel_block(X, 0.8, rows, cols, form=form)
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), form


def test_fp64_path_matches_the_oracle(poly):
    ia = poly
    N = 3000
    X = np.random.default_rng(82).random((N, 3))
    u = np.random.default_rng(83).standard_normal((N, 2))
    m, s_max, tol, lam = 64, 16, 1e-9, 1.0
    ia.iaskit_factor(X, H, lam, m, s_max, tol)
    with PolynomialKernel(P_DEG, P_C):
        tree, knn, sk, F = oracle.build_all(X, H, lam, m, s_max, tol)
        assert np.array_equal(ia.iaskit_get_perm(N), tree.perm)
        assert np.array_equal(ia.iaskit_get_knn(N, 16), knn)
        ranks = ia.iaskit_get_ranks()
        for (l, i), skel in sk.skel.items():
            assert ranks[(1 << l) + i] == len(skel) <= 10
            if sk.margin[(l, i)] > 1e-9:
                assert np.array_equal(ia.iaskit_get_skeleton(l, i), skel), (l, i)
        w = ia.iaskit_solve(u)
        ref = oracle.solve(F, u)
        assert np.linalg.norm(w - ref) / np.linalg.norm(ref) < 1e-10
        Au = ia.iaskit_apply(u)
        Au_ref = oracle.invaskit.apply_operator(sk, lam, u)
        assert np.linalg.norm(Au - Au_ref) / np.linalg.norm(Au_ref) < 1e-10
        T = np.random.default_rng(84).random((50, 3))
        s_gpu = ia.iaskit_predict(T, w)
        s_ref = scores(X, H, w, T)
        # FP64 sums of N signed terms: |error| <= gamma_N sum_j |K(t, x_j) w_j| (Higham's
        # summation bound, gamma_N ~ N 2^-53 = 3.3e-13 here), not relative to the
        # cancelled sum itself
        absum = np.abs(polynomial_kernel(T, X, H, P_DEG, P_C)) @ np.abs(w)
        assert np.all(np.abs(s_gpu - s_ref) <= 1e-12 * absum)


def test_mixed_form_refines(poly):
    ia = poly
    N = 3000
    X = np.random.default_rng(85).random((N, 3))
    u = np.random.default_rng(86).standard_normal((N, 2))
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("refine", 200)
    ia.iaskit_factor(X, H, 1e-2, 64, 16, 1e-9)
    w = ia.iaskit_solve(u)
    with PolynomialKernel(P_DEG, P_C):
        tree = oracle.build_tree(X, 64)
        sk = Skeletons(tree=tree, Xp=X[tree.perm], h=H)
        ranks = ia.iaskit_get_ranks()
        for l in range(1, tree.L + 1):
            for i in range(1 << l):
                sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
                sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
        assert oracle.residual(sk, 1e-2, w, u) <= 1e-10


def test_learned_sampling_refuses_the_polynomial_kernel(poly):
    ia = poly
    X = np.random.default_rng(87).random((2000, 3))
    ia.iaskit_set_option("sampling", 1)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_factor(X, H, 1.0, 64, 16, 1e-9)
    assert e.value.name in ("IASKIT_ERR_UNSUPPORTED", "IASKIT_ERR_ARG")
