"""Failure reporting through the C ABI, with no GPU fault (Sec. 10 of the design notes'
failure handling: every call returns a status and never aborts).

The library's kernels report an expired bounded wait, an exact zero pivot, a
non-finite input or an exceeded internal bound by setting bits of one device status
word, which the host reads after each phase.  The "inject_status" hook ORs chosen
bits into that word from the host just before the next read, so these tests check
that each bit reaches the caller as its error code and that the library stays
usable afterwards.  No kernel is made to wait, trap or fault.
"""
import numpy as np
import pytest

import oracle
from workloads import make_points, make_rhs, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bit,name", [(8, "IASKIT_ERR_TIMEOUT"), (1, "IASKIT_ERR_SINGULAR"),
                                      (2, "IASKIT_ERR_INPUT"), (4, "IASKIT_ERR_UNSUPPORTED")])
def test_device_status_reaches_the_caller(gpu_lib, bit, name):
    ia = gpu_lib
    w = workload("C1", N=1024)
    X = make_points(w)
    ia.iaskit_free()
    ia.iaskit_set_option("inject_status", bit)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_factor(X, w.h, w.lam, w.m, w.s_max, w.tol)
    assert e.value.name == name
    assert ia.iaskit_get_option("inject_status") == 0     # one-shot
    assert ia.iaskit_stats()["factored"] is False
    # the context and the library are usable: the next factorization is the oracle's
    ia.iaskit_factor(X, w.h, w.lam, w.m, w.s_max, w.tol)
    u = make_rhs(w, N=1024, nrhs=1)
    x = ia.iaskit_solve(u)
    tree, knn, sk, F = oracle.build_all(X, w.h, w.lam, w.m, w.s_max, w.tol)
    ref = oracle.solve(F, u)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10


def test_timeout_during_solve_keeps_the_factorization(gpu_lib):
    ia = gpu_lib
    w = workload("C1", N=1024)
    X = make_points(w)
    ia.iaskit_factor(X, w.h, w.lam, w.m, w.s_max, w.tol)
    u = make_rhs(w, N=1024, nrhs=2)
    x0 = ia.iaskit_solve(u)
    ia.iaskit_set_option("inject_status", 8)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_solve(u)
    assert e.value.name == "IASKIT_ERR_TIMEOUT"
    assert "bounded device wait" in ia.iaskit_last_error()
    np.testing.assert_array_equal(ia.iaskit_solve(u), x0)
