"""The allocation-free kNN entry point against the regular one.

Some callers cannot allocate device memory (a server whose device memory is all
owned by its own pool, or code that must not pay cudaMalloc's synchronization).
iaskit_knn_noalloc serves them from a static device array.  This file is named to
be collected last, so a stop-at-first-failure run has run every other test first.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _regular_knn(ia, X, kappa):
    ia.iaskit_set_option("kappa", kappa)
    ia.iaskit_factor(X, 0.5, 1.0, 64, 8, 0.0)
    out = ia.iaskit_get_knn(len(X), kappa)
    ia.iaskit_set_option("kappa", 16)
    return out


def _inputs():
    rng = np.random.default_rng(11)
    uniform = rng.random((3001, 8))
    dup = np.repeat(rng.random((60, 3)), 30, axis=0)[rng.permutation(1800)]   # exact ties
    wide = rng.standard_normal((1500, 54))
    return [(uniform, 16), (dup, 16), (wide, 12)]


def test_noalloc_knn_matches_regular_entry_point(gpu_lib):
    import torch
    ia = gpu_lib
    for X, kappa in _inputs():
        ref = _regular_knn(ia, X, kappa)
        Xd = torch.from_numpy(X).cuda()
        for _ in range(2):                     # two calls in a row share the scratch
            out = torch.full((len(X), kappa), -1, dtype=torch.int32, device="cuda")
            ia.iaskit_knn_noalloc(Xd, kappa, out)
            assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_limit(gpu_lib):
    import torch
    ia = gpu_lib
    X = torch.zeros((32769, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((32769, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_knn_noalloc(X, 4, out)
    assert e.value.name == "IASKIT_ERR_ARG"
    assert "32768" in ia.iaskit_last_error()
