"""The grouped GEMM's autotuned tile shapes change the speed, never a result.

Every CUDA-core tile shape sums each output over k in the same order, so a
factorization and solve with every bucket of the tile table forced to one shape are
bit for bit those with the default rule, in the plain FP64 form and in the mixed form
with its FP32 products on the CUDA cores.  The tuning call times each shape.
"""
import numpy as np
import pytest

from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu

SHAPES = ["64x64", "256x16", "128x32", "512x8"]


def _clear(ia):
    for fp64 in (0, 1):
        for nb in range(6):
            for mb in range(5):
                ia.iaskit_gemm_tile(fp64, nb, mb, None)


def _force(ia, shape):
    for fp64 in (0, 1):
        if fp64 and shape == "512x8":
            continue
        for nb in range(6):
            for mb in range(5):
                ia.iaskit_gemm_tile(fp64, nb, mb, shape)


def _run(ia, X, u, precision):
    ia.iaskit_set_option("precision", precision)
    ia.iaskit_set_option("gemm_tc", 0)
    ia.iaskit_set_option("refine", 200 if precision else 0)
    ia.iaskit_factor(X, 1.0, 1e-2, 256, 96, 1e-5)
    w = ia.iaskit_solve(u)
    return w, ia.iaskit_apply(w)


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_shapes_give_identical_results(gpu_lib, precision):
    ia = gpu_lib
    X = make_points(workload("C2", N=6000))
    u = make_rhs(workload("C2"), N=6000, nrhs=20)   # 20 columns: more than one 16-column tile
    try:
        _clear(ia)
        w0, a0 = _run(ia, X, u, precision)
        for shape in SHAPES:
            _force(ia, shape)
            w, a = _run(ia, X, u, precision)
            assert np.array_equal(w, w0), shape
            assert np.array_equal(a, a0), shape
    finally:
        for k, v in (("precision", 0), ("gemm_tc", 1), ("refine", 0)):
            ia.iaskit_set_option(k, v)
        _clear(ia)
        ia.load_tile_table()


def test_tuning_call(gpu_lib):
    ia = gpu_lib
    for shape in SHAPES:
        assert ia.iaskit_tune_gemm(False, 256, 32, 256, 64, shape, reps=2) > 0.0
    assert ia.iaskit_tune_gemm(True, 256, 8, 256, 64, "256x16", reps=2) > 0.0
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_tune_gemm(True, 256, 8, 256, 64, "512x8", reps=2)   # FP32 only
    assert e.value.name == "IASKIT_ERR_ARG"
