"""Kernel blocks (Sec. I, eq. gaussian) from the library's three evaluators.

* "pair" (FP32 pairs: the mixed form's operator blocks) against exact values: the
  squared distance of the FP64 coordinates as a rational number and its exp in
  40-digit decimal arithmetic, on sampled entries.  The bound: a coordinate x held as
  hi + lo is off by at most 2^-48 |x|, and the difference t_k = x_k - y_k formed from
  the pairs by at most 2^-47 (|x_k| + |y_k|), so the squared distance is off by
  2^-46 rho |t|^2 with rho = sum_k |t_k| (|x_k| + |y_k|) / |t|^2, plus the rounding of
  the low part of the running sum, (d + 2) 2^-48 |t|^2; an error of the argument
  a = |t|^2 / (2 h^2) moves exp(-a) by a times its relative error, and the pair exp
  and products add a few 2^-48.  Tolerance 2^-45 + a (2^-46 rho + (d + 2) 2^-48)
  relative, plus 1e-44 absolute: below 2^-102 the low part of a pair is an FP32
  subnormal (spacing 1.4e-45).
* all three forms against the FP64 oracle on whole blocks with several 64 x 64 tiles
  and a ragged edge; the tolerance adds the oracle's own rounding (d 2^-53 of the
  squared distance) and, for FP64, the Gram form's cancellation bound.
* values under the FP32 normal range come back as 0 from the pair form.
* "sliced" (FP64 Gram form with the dot products on the tensor cores from 8-digit slices
  of the coordinates: the mixed form's FP64 operator blocks) against the oracle with the
  FP64 form's bound (the slices' dot-product error, about 2^-60 d max|x| max|y|, lies far
  below the Gram form's cancellation), within 2 ulp of the FP64 form on points with small
  integer coordinates (every dot product exact in both; the two forms differ only in their
  exp: the sliced form's table-driven exp is within about 1 ulp), on ragged 128-row and
  32-column tiles and for d = 3, 8, 54 and 64 (the four operand widths); refused for the
  polynomial kernel and for d > 64.
"""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle.kernel import gaussian_kernel, sqdist
from workloads import make_points, workload

pytestmark = pytest.mark.gpu


def _oracle(X, rows, cols, h, diag):
    K = gaussian_kernel(X[rows], X[cols], h)
    K[np.asarray(rows)[:, None] == np.asarray(cols)[None, :]] += diag
    return K


def _pair_rel_tol(X, rows, cols, h):
    """2^-45 + a (2^-46 rho + (d + 2) 2^-48) per entry (module docstring)."""
    A, B = X[rows], X[cols]
    num = np.zeros((len(rows), len(cols)))
    for k in range(X.shape[1]):
        t = A[:, k][:, None] - B[:, k][None, :]
        num += np.abs(t) * (np.abs(A[:, k])[:, None] + np.abs(B[:, k])[None, :])
    d2 = sqdist(A, B)
    a = d2 / (2 * h * h)
    a_rho = np.where(d2 > 0, num / (2 * h * h), 0.0)     # a rho = sum |t_k| (|x_k| + |y_k|) / (2 h^2)
    return 2.0 ** -45 + 2.0 ** -46 * a_rho + (X.shape[1] + 2) * 2.0 ** -48 * a


def _exact(x, y, h, same, diag):
    getcontext().prec = 40
    d2 = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, y))
    arg = d2 / (2 * Fraction(float(h)) ** 2)
    v = (-(Decimal(arg.numerator) / Decimal(arg.denominator))).exp()
    return float(v + (Decimal(float(diag)) if same else 0)), float(arg)


@pytest.fixture(scope="module")
def gmm():
    X = make_points(workload("C2", N=700))
    rng = np.random.default_rng(3)
    rows = rng.choice(len(X), 150, replace=False)
    cols = np.concatenate([rows[:40], rng.choice(len(X), 90, replace=False)])   # shared points: diagonal
    return X, rows, cols


def test_pair_blocks_match_exact_values(gpu_lib, gmm):
    ia = gpu_lib
    X, rows, cols = gmm
    h, diag = 1.0, 1e-2
    K = ia.iaskit_kernel_block(X, h, rows, cols, diag, form="pair")
    tol = _pair_rel_tol(X, rows, cols, h)
    rng = np.random.default_rng(4)
    picks = [(i, i) for i in range(0, 40, 7)] + [tuple(p) for p in rng.integers(0, [150, 130], size=(120, 2))]
    worst = 0.0
    for i, j in picks:
        v, a = _exact(X[rows[i]], X[cols[j]], h, rows[i] == cols[j], diag)
        worst = max(worst, abs(K[i, j] - v) / (tol[i, j] * abs(v) + 1e-44))
    print(f"pair form: worst error {worst:.3f} of the bound")
    assert worst <= 1.0


@pytest.mark.parametrize("form", ["fp64", "pair", "fp32", "sliced"])
def test_forms_match_oracle_blocks(gpu_lib, gmm, form):
    ia = gpu_lib
    X, rows, cols = gmm
    d = X.shape[1]
    for h, diag in ((1.0, 1e-2), (4.0, 0.0)):
        K = ia.iaskit_kernel_block(X, h, rows, cols, diag, form=form)
        ref = _oracle(X, rows, cols, h, diag)
        a = sqdist(X[rows], X[cols]) / (2 * h * h)
        base = np.exp(-a)
        oracle_err = d * 2.0 ** -53 * a * base
        if form in ("fp64", "sliced"):
            nrm = (X ** 2).sum(axis=1)
            tol = 8 * 2.0 ** -53 * (nrm[rows][:, None] + nrm[cols][None, :]) / (2 * h * h) * base + 4 * 2.0 ** -53 * np.abs(ref)
        elif form == "pair":
            tol = _pair_rel_tol(X, rows, cols, h) * base + 4 * 2.0 ** -53 * np.abs(ref) + 1e-44
        else:
            tol = 2.0 ** -21 * (1 + d * a) * base + 2.0 ** -22 * np.abs(ref)
        err = np.abs(K - ref)
        assert np.all(err <= tol + oracle_err), (form, h, (err / (tol + oracle_err)).max())


def test_ragged_and_degenerate_blocks(gpu_lib):
    ia = gpu_lib
    X = np.random.default_rng(5).random((300, 3))
    # one entry, a single row, a column of identical points
    for rows, cols in (([7], [7]), ([3], list(range(130))), (list(range(200)), [11, 11, 11])):
        for form in ("fp64", "pair", "fp32", "sliced"):
            K = ia.iaskit_kernel_block(X, 0.3, rows, cols, 0.5, form=form)
            ref = _oracle(X, np.array(rows), np.array(cols), 0.3, 0.5)
            assert K.shape == ref.shape
            # arguments up to 3 / (2 0.3^2) = 16.7
            if form == "pair":
                tol = _pair_rel_tol(X, np.array(rows), np.array(cols), 0.3) + 4 * 2.0 ** -53
                assert np.all(np.abs(K - ref) <= tol * np.abs(ref) + 1e-44)
            else:
                np.testing.assert_allclose(K, ref, rtol=2e-5 if form == "fp32" else 1e-13, atol=0)
    # a narrow bandwidth: arguments up to ~1e3; the pair form gives 0 for arguments
    # above 87 (values under 1.7e-38, below the FP32 normal range)
    K = ia.iaskit_kernel_block(X, 0.02, list(range(100)), list(range(100, 250)), 0.0, form="pair")
    ref = _oracle(X, np.arange(100), np.arange(100, 250), 0.02, 0.0)
    a = sqdist(X[:100], X[100:250]) / (2 * 0.02 ** 2)
    small, big = a > 87.5, a < 85.0
    assert small.any() and big.any() and np.all(K[small] == 0.0)
    tol = _pair_rel_tol(X, np.arange(100), np.arange(100, 250), 0.02) + 3 * 2.0 ** -53 * a
    assert np.all(np.abs(K[big] - ref[big]) <= tol[big] * ref[big] + 1e-44)


@pytest.mark.parametrize("d", [3, 8, 54, 64])
def test_sliced_matches_fp64_on_integer_points(gpu_lib, d):
    ia = gpu_lib
    rng = np.random.default_rng(40 + d)
    X = rng.integers(-100, 101, size=(400, d)).astype(np.float64)
    rows = np.arange(13, 400, 2)                          # 194 rows: two 128-row tiles
    cols = np.concatenate([rows[:20], rng.choice(400, 77, replace=False)])
    h = 3.0 * np.sqrt(d)
    a = ia.iaskit_kernel_block(X, h, rows, cols, 0.25, form="sliced")
    b = ia.iaskit_kernel_block(X, h, rows, cols, 0.25, form="fp64")
    assert np.all(np.abs(a - b) <= 2 * np.spacing(np.abs(b)))
    ref = _oracle(X, rows, cols, h, 0.25)
    arg = sqdist(X[rows], X[cols]) / (2 * h * h)          # exact squared distances, rounded argument
    assert np.all(np.abs(a - ref) <= 4 * 2.0 ** -52 * (1 + arg) * np.abs(ref) + 1e-300)


@pytest.mark.parametrize("h", [0.05, 0.2])
def test_sliced_over_the_exp_range(gpu_lib, h):
    # arguments |x - y|^2 / (2 h^2) up to 600 (h = 0.05) on points of [0, 1]^3: the
    # table-driven exp over its whole reduction range, against the oracle with the FP64
    # form's bound; values far under FP64's range are 0 on both sides
    ia = gpu_lib
    X = np.random.default_rng(47).random((400, 3))
    rows, cols = np.arange(0, 400, 2), np.arange(1, 400, 3)
    K = ia.iaskit_kernel_block(X, h, rows, cols, 0.0, form="sliced")
    ref = _oracle(X, rows, cols, h, 0.0)
    a = sqdist(X[rows], X[cols]) / (2 * h * h)
    base = np.exp(-a)
    nrm = (X ** 2).sum(axis=1)
    tol = (8 * 2.0 ** -53 * (nrm[rows][:, None] + nrm[cols][None, :]) / (2 * h * h) * base
           + 4 * 2.0 ** -53 * np.abs(ref) + 3 * 2.0 ** -53 * a * base + 1e-300)
    assert h > 0.1 or a.max() > 100
    assert np.all(np.abs(K - ref) <= tol), (np.abs(K - ref) / tol).max()


def test_sliced_refuses_outside_its_range(gpu_lib):
    ia = gpu_lib
    X = np.random.default_rng(7).random((50, 65))
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_kernel_block(X, 1.0, [0, 1], [2, 3], 0.0, form="sliced")
    assert e.value.name == "IASKIT_ERR_UNSUPPORTED"
    ia.iaskit_set_option("kernel", 1)
    try:
        with pytest.raises(ia.IaskitError) as e:
            ia.iaskit_kernel_block(X[:, :8], 1.0, [0, 1], [2, 3], 0.0, form="sliced")
        assert e.value.name == "IASKIT_ERR_UNSUPPORTED"
    finally:
        ia.iaskit_set_option("kernel", 0)


def test_invalid_arguments(gpu_lib):
    ia = gpu_lib
    X = np.random.default_rng(6).random((50, 2))
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_kernel_block(X, 1.0, [0, 50], [1], 0.0)
    assert e.value.name == "IASKIT_ERR_ARG"
    with pytest.raises(ia.IaskitError):
        ia.iaskit_kernel_block(X, -1.0, [0], [1], 0.0)
    Y = X.copy()
    Y[3, 1] = np.nan
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_kernel_block(Y, 1.0, [0], [1], 0.0)
    assert e.value.name == "IASKIT_ERR_INPUT"
