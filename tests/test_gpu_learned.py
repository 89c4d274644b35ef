"""Learned row proposal: BF16 MLP kernels, candidates, features, selection, judge, labels.

The GPU's BF16 MLP is compared with the FP64 oracle MLP on the same (BF16-rounded)
inputs: scores and gradients within a few BF16 roundings, in norm (relative 2e-2 and
5e-2) and element by element (4 2^-8 of the absolute-value network's output or
gradient), Adam's update exactly as the oracle's Adam applied to the GPU's gradient.
Integer parts (candidates, selection, held-out rows) are bit-exact; features within
BF16 rounding; the held-out errors and the kept IDs match the oracle in FP64.
"""
import numpy as np
import pytest

import oracle
from oracle import learned as OL
from oracle.linalg import cpqr_id
from oracle.kernel import gaussian_kernel
from workloads import make_points, workload

pytestmark = pytest.mark.gpu


def bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _features(n, seed):
    rng = np.random.default_rng(seed)
    F = np.column_stack([rng.random(n) * 1.5, rng.random(n) * 3, rng.random(n), rng.random(n) * 0.5,
                         rng.random(n), rng.random(n), rng.random(n) * 2, np.zeros(n)])
    return F.astype(np.float32)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-30)


@pytest.fixture()
def mlp(gpu_lib):
    ia = gpu_lib
    p = OL.mlp_init(seed=7)
    p["b1"] = np.random.default_rng(8).uniform(-0.1, 0.1, 128)
    p["b2"] = np.random.default_rng(9).uniform(-0.1, 0.1, 128)
    p["b3"] = np.array([0.05])
    ia.iaskit_sampler_set_weights(ia.mlp_pack(p))
    return ia, ia.mlp_unpack(ia.iaskit_sampler_get_weights())


# Element-by-element bounds: the GPU rounds the weights and the inputs of every layer
# to BF16 (8 significant bits, relative error 2^-9 each) and accumulates in FP32, so
# every output differs from the FP64 oracle's by at most a few 2^-8 of the same
# network evaluated on absolute values with every unit active (an upper bound of the
# sum of the absolute terms).  BF16_C = 4 covers the roundings of one layer's inputs,
# weights and outputs plus the occasional unit whose pre-activation lies within
# rounding of 0 and switches on one side only.
BF16_C = 4 * 2.0 ** -8


def _abs_net(p, X):
    A1 = np.abs(X) @ np.abs(p["W1"]).T + np.abs(p["b1"])
    A2 = A1 @ np.abs(p["W2"]).T + np.abs(p["b2"])
    return A2 @ np.abs(p["w3"]) + abs(p["b3"][0]), A1, A2


def _abs_grad(p, X, dy_abs):
    y, A1, A2 = _abs_net(p, X)
    dA2 = np.outer(dy_abs, np.abs(p["w3"]))
    dA1 = dA2 @ np.abs(p["W2"])
    return {"w3": A2.T @ dy_abs, "b3": np.array([dy_abs.sum()]), "W2": dA2.T @ A1, "b2": dA2.sum(axis=0),
            "W1": dA1.T @ np.abs(X), "b1": dA1.sum(axis=0)}


def test_mlp_forward_matches_oracle(mlp):
    ia, p = mlp
    F = _features(3000, 1)
    y = ia.iaskit_mlp_forward(F)
    ref, _ = OL.mlp_forward(p, bf16(F))
    assert _rel(y, ref) < 2e-2, _rel(y, ref)
    bound = BF16_C * _abs_net(p, bf16(F))[0]
    worst = np.max(np.abs(y - ref) / bound)
    print(f"forward: largest error / element bound = {worst:.3f}")
    assert worst <= 1.0


def test_mlp_gradient_matches_oracle(mlp):
    ia, p = mlp
    F = _features(4096, 2)
    y, cache = OL.mlp_forward(p, bf16(F))
    # residuals of one sign, so that no gradient entry is a cancelling sum
    t = y - 1.0 + 0.1 * np.random.default_rng(3).standard_normal(4096)
    g, loss = ia.iaskit_mlp_train_step(F, t, lr=0.0)
    gref = OL.mlp_backward(p, cache, y, t)
    assert loss == pytest.approx(OL.mse_loss(y, t), rel=2e-2)
    gg = ia.mlp_unpack(g)
    for k in gref:
        assert _rel(gg[k], gref[k]) < 5e-2, (k, _rel(gg[k], gref[k]))
    # element by element: dy = 2 (y - t) / B is of one sign and size ~1 / B here
    gabs = _abs_grad(p, bf16(F), np.abs(2.0 * (y - t) / t.size))
    for k in gref:
        worst = np.max(np.abs(np.asarray(gg[k]) - gref[k]) / (BF16_C * gabs[k] + 1e-30))
        print(f"gradient {k}: largest error / element bound = {worst:.3f}")
        assert worst <= 1.0, k


def test_adam_steps_match_oracle(mlp):
    ia, p = mlp
    F = _features(1024, 4)
    t = np.random.default_rng(5).standard_normal(1024)
    state = {}
    pw = {k: v.copy() for k, v in p.items()}
    for step in range(2):
        g, _ = ia.iaskit_mlp_train_step(F, t, lr=1e-3)
        OL.adam_step(pw, ia.mlp_unpack(g), state, lr=1e-3)
        got = ia.mlp_unpack(ia.iaskit_sampler_get_weights())
        for k in pw:
            np.testing.assert_allclose(got[k], pw[k], rtol=1e-5, atol=1e-6, err_msg=f"{k} step {step}")


# ------------------------------------------------------------- pipeline checks
def _cols(ia, Xp_n, tree, l, i):
    """ID columns of node (l, i): its points (leaf) or its children's kept skeletons."""
    if l == tree.L:
        o, e = _range(tree, l, i)
        return np.arange(o, e)
    return np.concatenate([ia.iaskit_get_skeleton(l + 1, 2 * i), ia.iaskit_get_skeleton(l + 1, 2 * i + 1)])


def _range(tree, l, i):
    sizes = [tree.N]
    offs = [0]
    for _ in range(l):
        ns, no = [], []
        for o, n in zip(offs, sizes):
            no += [o, o + n // 2]
            ns += [n // 2, n - n // 2]
        sizes, offs = ns, no
    return offs[i], offs[i] + sizes[i]


def _strat(tree, l, i, N, count, salt):
    so, se = _range(tree, l, i ^ 1)
    po, pe = _range(tree, l - 1, i >> 1)
    return OL.stratified_rows(so, se - so, po, pe - po, N, count, 0, salt, (1 << l) + i)


@pytest.fixture(scope="module")
def learned_run(gpu_lib):
    ia = gpu_lib
    w = workload("C4", N=3000)
    X = make_points(w)
    h, lam, m, s_max, tol = 0.8, 1e-3, 128, 32, 1e-6
    p = OL.mlp_init(seed=11)
    ia.iaskit_sampler_set_weights(ia.mlp_pack(p))
    ia.iaskit_set_option("sampling", 1)
    ia.iaskit_set_option("keep_candidates", 1)
    ia.iaskit_set_option("learned_temp", 1.0)     # exercise the Gumbel selection
    try:
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        st = ia.iaskit_stats()
        tree = oracle.build_tree(X, m)
        L = tree.L
        nodes = {}
        for l in range(1, L + 1):
            for i in range(1 << l):
                cand, feat, score, info = ia.iaskit_get_learned(l, i)
                nodes[(l, i)] = dict(cand=cand, feat=feat, score=score, info=info,
                                     samp=ia.iaskit_get_samples(l, i),
                                     skel=ia.iaskit_get_skeleton(l, i),
                                     cols=_cols(ia, None, tree, l, i))
                s = len(nodes[(l, i)]["skel"])
                nodes[(l, i)]["P"] = ia.iaskit_get_P(l, i, s)
        u = np.random.default_rng(12).standard_normal((len(X), 2))
        wsol = ia.iaskit_solve(u)
    finally:
        ia.iaskit_set_option("sampling", 0)
        ia.iaskit_set_option("keep_candidates", 0)
        ia.iaskit_set_option("learned_temp", 0.0)
    return dict(X=X, tree=tree, nodes=nodes, st=st, p=ia.mlp_unpack(ia.mlp_pack(p)), u=u, w=wsol,
                params=(h, lam, m, s_max, tol), ia=ia)


def test_learned_candidates_and_features_match_oracle(learned_run):
    r = learned_run
    tree, X = r["tree"], r["X"]
    h, lam, m, s_max, tol = r["params"]
    knn = oracle.knn_bruteforce(X, 16)
    knn_pos = tree.iperm[knn[tree.perm]]
    Xp = X[tree.perm]
    N = len(X)
    checked = 0
    for (l, i), nd in r["nodes"].items():
        o, e = _range(tree, l, i)
        n = e - o
        ns = min(2 * s_max, N - n)
        uid = (1 << l) + i
        if ns >= N - n:
            assert nd["cand"].size == 0
            continue
        cand, hits = OL.learned_candidates(knn_pos[o:e], o, n, N, ns, seed=0, uid=uid)
        assert np.array_equal(nd["cand"], cand), (l, i)
        F = OL.candidate_features(Xp, cand, hits, nd["cols"], h, l, tree.L, n, N, 16)
        err = np.abs(nd["feat"] - F) / np.maximum(1.0, np.abs(F))
        assert err.max() < 1.5e-2, ((l, i), err.max(axis=0))
        checked += 1
    assert checked > 0


def test_learned_scores_selection_and_judge(learned_run):
    r = learned_run
    tree, X = r["tree"], r["X"]
    h, lam, m, s_max, tol = r["params"]
    Xp = X[tree.perm]
    N = len(X)
    knn = oracle.knn_bruteforce(X, 16)
    knn_pos = tree.iperm[knn[tree.perm]]
    kept = judged = 0
    for (l, i), nd in r["nodes"].items():
        if nd["cand"].size == 0:
            continue
        o, e = _range(tree, l, i)
        n, uid, ns = e - o, (1 << l) + i, int(nd["info"][3])
        ref, _ = OL.mlp_forward(r["p"], nd["feat"].astype(np.float64))
        keys = OL.gumbel_keys(ref, 0, uid, 1.0)       # the kept scores carry the perturbation
        assert _rel(nd["score"], keys) < 2e-2
        err_p, err_l, chosen = nd["info"][:3]
        assert chosen == (1.0 if err_l <= err_p else 0.0)
        if chosen == 1.0:
            assert np.array_equal(nd["samp"], OL.select_top(nd["score"], nd["cand"], ns)), (l, i)
            kept += 1
        else:
            from oracle.sampling import sample_rows
            assert np.array_equal(nd["samp"], sample_rows(knn_pos[o:e], o, n, N, ns, seed=0, uid=uid))
        H, wts = _strat(tree, l, i, N, OL.NHOLD, OL.HOLD_SALT)
        e_ref = OL.heldout_error(Xp, H, wts, nd["cols"], nd["skel"], nd["P"], h)
        e_gpu = err_l if chosen == 1.0 else err_p
        assert e_gpu == pytest.approx(e_ref, rel=1e-6, abs=1e-24), (l, i)
        # the kept ID is the ID of the kept sample
        A = gaussian_kernel(Xp[nd["samp"]], Xp[nd["cols"]], h)
        piv, s, P, _, margin = cpqr_id(A, s_max, tol)
        if margin > 1e-9:
            assert np.array_equal(nd["cols"][piv[:s]], nd["skel"]), (l, i)
            np.testing.assert_allclose(nd["P"], P, rtol=1e-10, atol=1e-10 * np.abs(P).max())
        judged += 1
    assert judged > 0
    st = r["st"]
    assert st["learned_nodes"] + st["fallback_nodes"] == judged
    print(f"learned kept at {kept} of {judged} judged nodes")


def test_learned_factorization_solves_its_operator(learned_run):
    from oracle.askit import Skeletons
    r = learned_run
    tree, X = r["tree"], r["X"]
    h, lam = r["params"][:2]
    sk = Skeletons(tree=tree, Xp=X[tree.perm], h=h)
    for (l, i), nd in r["nodes"].items():
        sk.skel[(l, i)] = nd["skel"].astype(np.int64)
        sk.P[(l, i)] = nd["P"]
    rho = oracle.residual(sk, lam, r["w"], r["u"])
    assert rho < 1e-10, rho


def test_training_labels_match_oracle_and_loss_falls(gpu_lib):
    ia = gpu_lib
    w = workload("C4", N=2048)
    X = make_points(w)
    h, m, s_max, tol = 0.8, 128, 24, 1e-6
    ia.iaskit_sampler_set_weights(ia.mlp_pack(OL.mlp_init(seed=3)))
    ia.iaskit_set_option("keep_candidates", 1)
    try:
        ia.iaskit_sampler_train(X, h, m, s_max, tol, epochs=12, lr=2e-3)
        st = ia.iaskit_stats()
        tree = oracle.build_tree(X, m)
        Xp = X[tree.perm]
        N = len(X)
        checked = 0
        for l in range(1, tree.L + 1):
            for i in (0, (1 << l) - 1):
                cand, feat, target, info = ia.iaskit_get_learned(l, i)
                if cand.size == 0:
                    continue
                o, e = _range(tree, l, i)
                cols = _cols(ia, None, tree, l, i)
                gram, wts = _strat(tree, l, i, N, OL.NGRAM, OL.GRAM_SALT)
                _, t_ref = OL.leverage_labels(Xp, cand, cols, gram, wts, h, tol)
                assert np.abs(target - t_ref).max() < 2e-3, (l, i, np.abs(target - t_ref).max())
                checked += 1
        assert checked > 0
    finally:
        ia.iaskit_set_option("keep_candidates", 0)
    loss = st["train_loss"]
    assert len(loss) == 12 and st["train_rows"] > 0
    assert loss[-1] < loss[0], loss
