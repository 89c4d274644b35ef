"""FP64 operator products on the BF16 tensor cores by exact slicing (option "op_slices").

The mixed form keeps FP64 operator blocks for problems whose condition estimate exceeds
"pair_cond_max" (set to 1 here, so every problem does); with "op_slices" = 1 (default)
its Skeletonize (P) and Evaluate (K blocks) steps (Sec. II-B) multiply them as 8 signed
8-bit digits per value on the tensor cores.  Checks, on the library's own skeletons and P read back into the oracle:

* the operator equals the oracle's MatVec and the FP64-pipe products ("op_slices" = 0)
  within FP64-level error, column by column relative to || |K~| |w| || (the splitting's
  error is at most a few 2^-64 of a row's largest entry times a column's largest value per
  term), on ragged tiles (leaves of ~94 points, ranks <= 40, N not a multiple of 128) and
  on several exact 128-column segments (leaves of 512, ranks 256);
* exact invariants of the splitting: a zero column gives exactly zero, scaling a column
  by 2^300 or 2^-300 scales the result exactly (no partial result leaves FP64's normal
  range), negation is exact, and a column's result
  does not depend on the other columns (1, 8, 16, 17 and 33 right-hand sides: the
  16-column passes and a ragged last pass);
* columns whose values span 200 decades, or with one nonzero;
* the refined solve reaches 1e-10 against the oracle's operator with the sliced products.
"""
import numpy as np
import pytest

import oracle
from oracle.askit import Skeletons, dense_Ktilde
from workloads import make_points, workload

pytestmark = pytest.mark.gpu

CASES = {
    # name: (generator, N, h, lambda, m, s_max, tol)
    "ragged": ("C1", 3000, 0.5, 1e-2, 100, 40, 1e-9),
    "segments": ("C2", 8192, 1.0, 1e-2, 512, 256, 1e-7),
}


def _gpu_skeletons(ia, X, tree, h):
    sk = Skeletons(tree=tree, Xp=np.asarray(X)[tree.perm], h=h)
    ranks = ia.iaskit_get_ranks()
    for l in range(1, tree.L + 1):
        for i in range(1 << l):
            sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
            sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
    return sk


def _probe(N, seed):
    """Columns: normal, zero, one nonzero, values over 200 decades with random signs, normal."""
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((N, 5))
    W[:, 1] = 0.0
    W[:, 2] = 0.0
    W[N // 3, 2] = 1.7
    W[:, 3] = rng.choice([-1.0, 1.0], N) * 10.0 ** (-200.0 * rng.random(N))
    return W


@pytest.fixture(scope="module", params=sorted(CASES))
def sliced(request, gpu_lib):
    ia = gpu_lib
    gname, N, h, lam, m, s_max, tol = CASES[request.param]
    X = make_points(workload(gname, N=N))
    W = _probe(N, 11)
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("pair_cond_max", 1.0)
    try:
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        st = ia.iaskit_stats()
        ia.iaskit_set_option("op_slices", 1)
        got = ia.iaskit_apply(W)
        scaled = [ia.iaskit_apply(np.ldexp(W[:, :1], e)) for e in (300, -300)]
        neg = ia.iaskit_apply(-W)
        ia.iaskit_set_option("op_slices", 0)
        fp64 = ia.iaskit_apply(W)
        ia.iaskit_set_option("op_slices", 1)
        tree = oracle.build_tree(X, m)
        sk = _gpu_skeletons(ia, X, tree, h)
    finally:
        ia.iaskit_set_option("op_slices", 1)
        ia.iaskit_set_option("pair_cond_max", 1e5)
        ia.iaskit_set_option("precision", 0)
    return dict(ia=ia, name=request.param, X=X, W=W, got=got, scaled=scaled, neg=neg, fp64=fp64, sk=sk,
                lam=lam, st=st, params=(h, lam, m, s_max, tol))


def _absop(c, W):
    """|lambda I + K~| |W| columns (dense K~ of the library's skeletons, original order)."""
    sk, tree = c["sk"], c["sk"].tree
    A = np.abs(dense_Ktilde(sk)) + c["lam"] * np.eye(tree.N)
    out = np.empty_like(W)
    out[tree.perm] = A @ np.abs(W)[tree.perm]
    return out


def test_every_problem_keeps_fp64_blocks(sliced):
    assert sliced["st"]["fp64_operator_problems"] == 1
    assert sliced["st"]["bytes"]["operator_slices"] == 0  # built at the first apply


def test_operator_matches_oracle_and_fp64_products(sliced):
    c = sliced
    W, got = c["W"], c["got"]
    ref = oracle.invaskit.apply_operator(c["sk"], c["lam"], W)
    bound = np.linalg.norm(_absop(c, W), axis=0)
    for col in range(W.shape[1]):
        err = np.linalg.norm(got[:, col] - ref[:, col])
        err64 = np.linalg.norm(got[:, col] - c["fp64"][:, col])
        assert err <= 2e-14 * bound[col], (c["name"], col, err / max(bound[col], 1e-300))
        assert err64 <= 2e-14 * bound[col], (c["name"], col, err64 / max(bound[col], 1e-300))
    assert np.all(got[:, 1] == 0.0)
    # the normal column: relative error of the order of FP64's
    assert np.linalg.norm(got[:, 0] - ref[:, 0]) / np.linalg.norm(ref[:, 0]) < 1e-13


def test_exact_invariants(sliced):
    c = sliced
    assert np.array_equal(c["scaled"][0][:, 0], np.ldexp(c["got"][:, 0], 300))
    assert np.array_equal(c["scaled"][1][:, 0], np.ldexp(c["got"][:, 0], -300))
    assert np.array_equal(c["neg"], -c["got"])


@pytest.mark.parametrize("nrhs", [1, 8, 16, 17, 33])
def test_columns_are_independent(sliced, nrhs):
    c = sliced
    ia = c["ia"]
    h, lam, m, s_max, tol = c["params"]
    N = c["X"].shape[0]
    rng = np.random.default_rng(100 + nrhs)
    W = rng.standard_normal((N, nrhs)) * np.ldexp(1.0, rng.integers(-30, 30, nrhs))
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("pair_cond_max", 1.0)
    try:
        ia.iaskit_factor(c["X"], h, lam, m, s_max, tol)
        U = ia.iaskit_apply(W)
        last = ia.iaskit_apply(W[:, -1])
        first = ia.iaskit_apply(W[:, 0])
    finally:
        ia.iaskit_set_option("pair_cond_max", 1e5)
        ia.iaskit_set_option("precision", 0)
    assert np.array_equal(U[:, -1], last)
    assert np.array_equal(U[:, 0], first)


def test_refined_solve_with_sliced_operator(sliced):
    c = sliced
    ia = c["ia"]
    h, lam, m, s_max, tol = c["params"]
    N = c["X"].shape[0]
    u = np.random.default_rng(21).standard_normal((N, 3))
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("pair_cond_max", 1.0)
    ia.iaskit_set_option("refine", 200)
    try:
        ia.iaskit_factor(c["X"], h, lam, m, s_max, tol)
        w = ia.iaskit_solve(u)
        st = ia.iaskit_stats()
        sk = _gpu_skeletons(ia, c["X"], oracle.build_tree(c["X"], m), h)
    finally:
        ia.iaskit_set_option("refine", 0)
        ia.iaskit_set_option("pair_cond_max", 1e5)
        ia.iaskit_set_option("precision", 0)
    assert st["bytes"]["operator_slices"] > 0
    assert st["kernels"]["operator_slices"]["calls"] > 0
    assert oracle.residual(sk, lam, w, u) <= 1e-10
