"""Refinement and the per-problem precision of the mixed form.

* The condition estimate each problem gets is 1 + max_i sum_j K(x_i, x_j) / lambda over
  64 rows i spread evenly over the tree order; recomputed here with numpy from the
  returned permutation.
* The mixed form factors a problem in FP64 when that estimate exceeds
  "mixed_cond_max", and every column of a batch mixing both precisions is refined.
* A target below the FP64 rounding floor of the residual ends with the columns marked
  "stagnated" instead of spending the whole iteration budget.
* A refinement that stops at the FP32-pair operator's floor upgrades that problem's
  operator blocks to FP64; a later refactor for a new lambda still solves to the
  target against the operator at that lambda.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _uniform(n, seed):
    return np.ascontiguousarray(np.random.default_rng(seed).random((n, 16)))


ILL = (_uniform(6000, 31), 1.2, 1e-3)     # ||K|| ~ 0.4 N, cond ~ 2e6
WELL = (_uniform(3000, 32), 0.6, 1e-1)    # cond ~ 1e3


def _cond_est(X, perm, h, lam):
    N = len(X)
    Xp = X[perm]
    rows = Xp[(np.arange(64) * N) // 64]
    d2 = ((rows[:, None, :] - Xp[None, :, :]) ** 2).sum(axis=2)
    return 1.0 + np.exp(-d2 / (2 * h * h)).sum(axis=1).max() / lam


@pytest.fixture()
def mixed_opts(gpu_lib):
    ia = gpu_lib
    ia.iaskit_set_option("precision", 1)
    yield ia
    ia.iaskit_set_option("precision", 0)
    ia.iaskit_set_option("mixed_cond_max", 1e6)
    ia.iaskit_set_option("refine", 0)
    ia.iaskit_set_option("refine_tol", 1e-10)


def test_condition_estimate_and_precision_choice(mixed_opts):
    ia = mixed_opts
    probs = [ILL, WELL]
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             128, 64, 1e-6)
    st = ia.iaskit_stats()
    for q, (X, h, lam) in enumerate(probs):
        ia.iaskit_set_option("problem", q)
        ref = _cond_est(X, ia.iaskit_get_perm(len(X)), h, lam)
        assert st["cond_est"][q] == pytest.approx(ref, rel=1e-3), q
    ia.iaskit_set_option("problem", 0)
    assert st["cond_est"][0] > 1e6 > st["cond_est"][1]
    assert st["fp64_problems"] == 1
    ia.iaskit_set_option("mixed_cond_max", 1e300)
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             128, 64, 1e-6)
    assert ia.iaskit_stats()["fp64_problems"] == 0
    ia.iaskit_set_option("mixed_cond_max", 1.0)
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             128, 64, 1e-6)
    assert ia.iaskit_stats()["fp64_problems"] == 2
    with pytest.raises(ia.IaskitError):
        ia.iaskit_set_option("mixed_cond_max", 0.5)


def _batch_residuals(ia, probs, rhs, w):
    """Per problem, the worst relative residual of its columns against the FP64 operator
    (the batched operator applied to all solutions at once)."""
    import torch
    Ns = [len(p[0]) for p in probs]
    nrhs = rhs[0].shape[1]
    W = torch.from_numpy(np.concatenate([np.asarray(x).T.reshape(-1) for x in w])).cuda()
    AW = torch.empty_like(W)
    ia.iaskit_apply_device(W, AW, nrhs)
    AW = AW.cpu().numpy()
    out, o = [], 0
    for q, n in enumerate(Ns):
        Au = AW[o:o + n * nrhs].reshape(nrhs, n).T
        o += n * nrhs
        out.append((np.linalg.norm(rhs[q] - Au, axis=0) / np.linalg.norm(rhs[q], axis=0)).max())
    return out


def test_mixed_batch_with_an_ill_conditioned_problem_is_refined(mixed_opts):
    ia = mixed_opts
    probs = [ILL, WELL]
    rng = np.random.default_rng(33)
    rhs = [rng.standard_normal((len(p[0]), 3)) for p in probs]
    ia.iaskit_factor_batched([p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                             128, 64, 1e-6)
    w = ia.iaskit_solve_batched(rhs)
    st = ia.iaskit_stats()
    assert st["fp64_problems"] == 1
    res = _batch_residuals(ia, probs, rhs, w)
    print("residuals", res, "history", st["refine_history"], "stagnated", st["refine_stagnated"])
    assert res[1] <= 1e-10
    # the FP64-factored problem meets the target unless its rounding floor is above it
    assert res[0] <= 1e-10 or (st["refine_stagnated"] >= 1 and res[0] <= 1e-9)
    assert st["refine_iters"] <= 40


def test_target_below_the_rounding_floor_stagnates(gpu_lib):
    ia = gpu_lib
    X, h, lam = ILL
    u = np.random.default_rng(34).standard_normal((len(X), 2))
    ia.iaskit_set_option("refine", 60)
    ia.iaskit_set_option("refine_tol", 1e-17)
    try:
        ia.iaskit_factor(X, h, lam, 128, 64, 1e-6)
        w = ia.iaskit_solve(u)
        st = ia.iaskit_stats()
    finally:
        ia.iaskit_set_option("refine", 0)
        ia.iaskit_set_option("refine_tol", 1e-10)
    assert st["refine_stagnated"] == 2
    assert st["refine_sweeps"] <= 6
    assert 1e-17 < st["refine_history"][-1] <= 1e-9
    Au = ia.iaskit_apply(w)
    rho = (np.linalg.norm(u - Au, axis=0) / np.linalg.norm(u, axis=0)).max()
    assert rho <= 1e-9


def test_pair_operator_floor_upgrades_to_fp64(mixed_opts):
    """A smooth, ill-conditioned problem (h = 1.2, lambda = 1e-3 on [0,1]^16) whose
    refinement stops at the FP32-pair operator's rounding floor above the target gets
    its operator blocks in FP64 and is refined again: the operator then agrees with
    the FP64 oracle's blocks to FP64 rounding, and the residual reaches the target or
    the FP64 floor."""
    ia = mixed_opts
    X = _uniform(2400, 35)
    u = np.random.default_rng(36).standard_normal((len(X), 2))
    ia.iaskit_set_option("refine", 400)
    ia.iaskit_set_option("pair_cond_max", 1e300)   # start from the pair operator
    try:
        ia.iaskit_factor(X, 1.2, 1e-3, 128, 64, 1e-6)
        w = ia.iaskit_solve(u)
        st = ia.iaskit_stats()
    finally:
        ia.iaskit_set_option("pair_cond_max", 1e5)
    print("upgrades", st["operator_upgrades"], "history", st["refine_history"])
    assert st["operator_upgrades"] == 1 and st["fp64_operator_problems"] == 1
    Au = ia.iaskit_apply(w)
    rho = (np.linalg.norm(u - Au, axis=0) / np.linalg.norm(u, axis=0)).max()
    assert rho <= 1e-10 or (st["refine_stagnated"] >= 1 and rho <= 1e-9), rho


def test_refactor_after_an_operator_upgrade(mixed_opts):
    """After a solve whose refinement upgraded the operator blocks to FP64, a refactor
    for a new lambda re-chooses every problem's precisions from 1 + r / lambda' and forms
    the leaf blocks, U, W and Z again: the next solve meets the target against the
    operator at the new lambda, checked by the oracle on the library's own skeletons."""
    from oracle.askit import Skeletons
    ia = mixed_opts
    X = _uniform(2400, 35)
    u = np.random.default_rng(37).standard_normal((len(X), 2))
    h, m = 1.2, 128
    ia.iaskit_set_option("refine", 400)
    ia.iaskit_set_option("pair_cond_max", 1e300)
    try:
        ia.iaskit_factor(X, h, 1e-3, m, 64, 1e-6)
        ia.iaskit_solve(u)
        assert ia.iaskit_stats()["operator_upgrades"] == 1
        for lam2 in (1e-1, 1e-3):
            ia.iaskit_refactor(lam2)
            w = ia.iaskit_solve(u)
            st = ia.iaskit_stats()
            tree = oracle.build_tree(X, m)
            sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
            ranks = ia.iaskit_get_ranks()
            for l in range(1, tree.L + 1):
                for i in range(1 << l):
                    sk.skel[(l, i)] = ia.iaskit_get_skeleton(l, i).astype(np.int64)
                    sk.P[(l, i)] = ia.iaskit_get_P(l, i, int(ranks[(1 << l) + i]))
            rho = oracle.residual(sk, lam2, w, u)
            print(f"lambda' {lam2}: residual {rho:.3e}, upgrades {st['operator_upgrades']}, "
                  f"history {st['refine_history']}")
            assert rho <= 1e-10 or (st["refine_stagnated"] >= 1 and rho <= 1e-9), (lam2, rho)
    finally:
        ia.iaskit_set_option("pair_cond_max", 1e5)
