"""What the trained row proposal gains (the learned part of the skeletonization: an MLP
scores candidate rows in place of the neighbour + uniform rule of Sec. II-B).

The sampler is trained on the GPU (labels from full-row IDs, BF16 forward/backward
and Adam kernels) on one draw of a generator, then a factorization of another draw
of the same generator is made with the plain rule and with the trained proposal (the
held-out judge keeping the better ID per node).  The quantity compared is the sampled
error eps_M = ||K w - K~ w|| / ||K w|| of eq. (error) (S = 0) on 1000 seeded rows,
K w from the oracle's exact kernel rows, K~ w from the library's operator minus
lambda w; the mean rank is printed beside it (both saturate at s_max here, so the
comparison is at equal rank).

* Anisotropic Gaussian mixture in 54 dimensions (the generator of the precision
  workload, N = 32768, m 256, s_max 64, tau 1e-5): the proposal lowers eps_M by more
  than 5% (measured: 0.2316 plain, 0.2121 learned, 8.4% lower).
* Tanh manifold in 64 dimensions (the learned-sampling workload's generator, N =
  16384, m 256, s_max 128, tau 1e-6): no gain; the judge keeps eps_M within 5% of the
  plain rule's.  The proposal is therefore not part of the benchmark's chosen form.
"""
import numpy as np
import pytest

from oracle.kernel import gaussian_kernel
from workloads import make_points, workload

pytestmark = pytest.mark.gpu


def _eps_M(ia, X, h, lam, rows, w):
    Kw = np.zeros(len(rows))
    for a in range(0, len(X), 8192):
        Kw += gaussian_kernel(X[rows], X[a:a + 8192], h) @ w[a:a + 8192]
    Ktw = ia.iaskit_apply(w[:, None])[:, 0] - lam * w
    return float(np.linalg.norm(Kw - Ktw[rows]) / np.linalg.norm(Kw))


def _gain(ia, name, N, h, lam, m, s_max, tol):
    wl = workload(name, N=N)
    train = make_points(wl.scaled(N, seed=wl.seed + 77))
    X = make_points(wl)
    rng = np.random.default_rng(17)
    rows = np.sort(rng.choice(N, 1000, replace=False))
    w = rng.standard_normal(N)
    ia.iaskit_sampler_train(train, h, m, s_max, tol, epochs=20, lr=2e-3)
    out = {}
    for sampling in (0, 1):
        ia.iaskit_set_option("sampling", sampling)
        ia.iaskit_factor(X, h, lam, m, s_max, tol)
        st = ia.iaskit_stats()
        ranks = st["mean_rank_per_height"]
        out[sampling] = (_eps_M(ia, X, h, lam, rows, w), float(np.mean(ranks)), st["learned_nodes"],
                         st["fallback_nodes"])
    ia.iaskit_set_option("sampling", 0)
    print(f"{name}: plain eps_M {out[0][0]:.4f} (mean rank {out[0][1]:.1f}); learned eps_M "
          f"{out[1][0]:.4f} (mean rank {out[1][1]:.1f}; learned ID kept at {out[1][2]} of "
          f"{out[1][2] + out[1][3]} judged nodes)")
    return out


@pytest.fixture()
def opts(gpu_lib):
    yield gpu_lib
    gpu_lib.iaskit_set_option("sampling", 0)
    gpu_lib.iaskit_set_option("precision", 0)


def test_learned_proposal_gains_on_the_mixture(opts):
    out = _gain(opts, "C2", 32768, 1.0, 1e-2, 256, 64, 1e-5)
    assert out[1][1] == pytest.approx(out[0][1], rel=0.02)     # equal rank
    assert out[1][0] < 0.95 * out[0][0]


def test_learned_proposal_on_the_manifold(opts):
    out = _gain(opts, "C4", 16384, 0.8, 1e-3, 256, 128, 1e-6)
    assert out[1][1] == pytest.approx(out[0][1], rel=0.02)
    assert out[1][0] < 1.05 * out[0][0]
