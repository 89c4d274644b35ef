"""Seeded generators for the synthetic point clouds and right-hand sides.

The paper measures on COVTYPE, SUSY, MNIST and a synthetic NORMAL cloud (Sec. III,
Tab. "datasets"); none of those files are used here.  Synthetic clouds with the
shapes of those workloads stand in for them:

* ``C1`` uniform points in [0,1]^8 (the small plain FP64 case);
* ``C2`` a 16-component anisotropic Gaussian mixture in 54 dimensions (the
  COVTYPE shape: N of a few hundred thousand, d = 54);
* ``C3`` 64 independent uniform problems in [0,1]^16 of log-uniform size;
* ``C4`` a 6-dimensional nonlinear manifold embedded in 64 dimensions plus
  isotropic noise (the NORMAL shape: high ambient, low intrinsic dimension);
* ``C5`` a 32-component Gaussian mixture in 8 dimensions with N = 4M (the SUSY
  shape).

Every draw uses numpy's PCG64 with seed ``1602013760 + k`` for workload ``Ck``.
Nothing here evaluates a kernel, a tree or a factorization.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Callable, Optional

import numpy as np

SEED_BASE = 1602013760


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(N: int, d: int, rng: np.random.Generator) -> np.ndarray:
    """N points uniform on [0,1]^d, float64, row-major (N, d)."""
    return rng.random((N, d))


def gaussian_mixture(N: int, d: int, ncomp: int, std_lo: float, std_hi: float,
                     rng: np.random.Generator) -> np.ndarray:
    """Equal-weight mixture of axis-aligned Gaussians.

    Component counts are multinomial with equal weights; means are uniform on
    [0,1]^d; each component and axis draws its standard deviation log-uniformly in
    [std_lo, std_hi].  Rows are shuffled so the original index carries no
    component structure.
    """
    counts = rng.multinomial(N, np.full(ncomp, 1.0 / ncomp))
    means = rng.random((ncomp, d))
    stds = np.exp(rng.uniform(np.log(std_lo), np.log(std_hi), size=(ncomp, d)))
    parts = []
    for c in range(ncomp):
        parts.append(means[c] + stds[c] * rng.standard_normal((counts[c], d)))
    X = np.concatenate(parts, axis=0)
    return X[rng.permutation(N)]


def labeled_gaussian_mixture(N: int, d: int, ncomp: int, std_lo: float, std_hi: float,
                             rng: np.random.Generator):
    """Points of an equal-weight axis-aligned Gaussian mixture (drawn as in
    ``gaussian_mixture``) with binary labels: +1 for the first ncomp // 2 components,
    -1 for the others (a one-versus-rest task of the shape of the paper's
    classification sets).  Returns (X (N, d), labels (N,) in {-1, +1})."""
    counts = rng.multinomial(N, np.full(ncomp, 1.0 / ncomp))
    means = rng.random((ncomp, d))
    stds = np.exp(rng.uniform(np.log(std_lo), np.log(std_hi), size=(ncomp, d)))
    parts, labels = [], []
    for c in range(ncomp):
        parts.append(means[c] + stds[c] * rng.standard_normal((counts[c], d)))
        labels.append(np.full(counts[c], 1.0 if c < ncomp // 2 else -1.0))
    X, y = np.concatenate(parts, axis=0), np.concatenate(labels)
    order = rng.permutation(N)
    return np.ascontiguousarray(X[order]), y[order]


def tanh_manifold(N: int, rng: np.random.Generator, d: int = 64, intrinsic: int = 6,
                  noise: float = 0.01) -> np.ndarray:
    """Points on a random two-layer tanh image of N(0, I_6) in R^64 plus noise.

    x = W2 tanh(W1 z + b1) + 0.01 eps with z ~ N(0, I_6), W1 (64 x 6) ~ N(0, 1/6),
    b1 ~ N(0, 0.1^2), W2 (64 x 64) ~ N(0, 1/64) and eps ~ N(0, I_64).  The map is
    drawn first, then the points, from the same generator.
    """
    W1 = rng.standard_normal((d, intrinsic)) / np.sqrt(intrinsic)
    b1 = 0.1 * rng.standard_normal(d)
    W2 = rng.standard_normal((d, d)) / np.sqrt(d)
    z = rng.standard_normal((N, intrinsic))
    H = np.tanh(z @ W1.T + b1)
    return H @ W2.T + noise * rng.standard_normal((N, d))


@dataclass(frozen=True)
class Workload:
    """Problem statement of one synthetic workload (kernel, solver and RHS sizes)."""

    name: str
    N: int
    d: int
    h: float
    lam: float
    m: int
    s_max: int
    tol: float
    nrhs: int
    kappa: int = 16
    samp_factor: int = 2
    seed: int = SEED_BASE
    kind: str = "uniform"
    ncomp: int = 0
    std_lo: float = 0.0
    std_hi: float = 0.0

    def scaled(self, N: int, **kw) -> "Workload":
        """Same generator and parameters at another N (other fields may be overridden)."""
        return replace(self, N=N, **kw)


WORKLOADS = {
    "C1": Workload("C1", N=4096, d=8, h=0.5, lam=1.0, m=64, s_max=32, tol=0.0,
                   nrhs=1, seed=SEED_BASE + 1, kind="uniform"),
    "C2": Workload("C2", N=262144, d=54, h=1.0, lam=1e-2, m=512, s_max=256, tol=1e-5,
                   nrhs=16, seed=SEED_BASE + 2, kind="gmm", ncomp=16, std_lo=0.05,
                   std_hi=1.0),
    "C3": Workload("C3", N=0, d=16, h=0.0, lam=0.0, m=128, s_max=128, tol=1e-6,
                   nrhs=4, seed=SEED_BASE + 3, kind="batched"),
    "C4": Workload("C4", N=1048576, d=64, h=0.8, lam=1e-3, m=512, s_max=256, tol=1e-6,
                   nrhs=8, seed=SEED_BASE + 4, kind="manifold"),
    "C5": Workload("C5", N=4194304, d=8, h=0.35, lam=1e-4, m=1024, s_max=512, tol=1e-7,
                   nrhs=64, seed=SEED_BASE + 5, kind="gmm", ncomp=32, std_lo=0.02,
                   std_hi=0.5),
}


def workload(name: str, N: Optional[int] = None, **kw) -> Workload:
    w = WORKLOADS[name]
    if N is not None or kw:
        w = w.scaled(N if N is not None else w.N, **kw)
    return w


def make_points(w: Workload) -> np.ndarray:
    """The seeded point cloud of workload ``w`` as a C-contiguous (N, d) float64 array."""
    rng = _rng(w.seed)
    if w.kind == "uniform":
        X = uniform_cube(w.N, w.d, rng)
    elif w.kind == "gmm":
        X = gaussian_mixture(w.N, w.d, w.ncomp, w.std_lo, w.std_hi, rng)
    elif w.kind == "manifold":
        X = tanh_manifold(w.N, rng, d=w.d)
    else:
        raise ValueError(f"workload {w.name} has no single point cloud (kind={w.kind})")
    return np.ascontiguousarray(X, dtype=np.float64)


def make_rhs(w: Workload, nrhs: Optional[int] = None, N: Optional[int] = None) -> np.ndarray:
    """RHS ~ N(0,1), shape (N, nrhs), column-major (Fortran order) float64."""
    n = w.N if N is None else N
    k = w.nrhs if nrhs is None else nrhs
    rng = _rng(w.seed + 1000003)
    return np.asfortranarray(rng.standard_normal((n, k)))


def batched_problems(count: int = 64, scale: float = 1.0, seed: int = SEED_BASE + 3):
    """Independent uniform problems of log-uniform size in [2048, 65536].

    Problem i has N_i = round(2048 * 32^u_i) (times ``scale``), d = 16 points uniform
    on [0,1]^16, h = (0.3, 0.6, 1.2)[i mod 3] and lambda = (1e-1, 1e-3)[(i div 3) mod 2].
    Returns a list of (X_i, h_i, lambda_i).
    """
    rng = _rng(seed)
    u = rng.random(count)
    out = []
    for i in range(count):
        n = max(2, int(round(2048 * 32.0 ** u[i] * scale)))
        X = np.ascontiguousarray(uniform_cube(n, 16, rng))
        out.append((X, (0.3, 0.6, 1.2)[i % 3], (1e-1, 1e-3)[(i // 3) % 2]))
    return out


GeneratorFn = Callable[[Workload], np.ndarray]
