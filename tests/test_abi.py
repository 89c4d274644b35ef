"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here (no GPU needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1602_01376_gb300 import build
    return build.build()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "iaskit.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(iaskit_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("iaskit_factor", "iaskit_solve", "iaskit_factor_device",
                     "iaskit_solve_device", "iaskit_apply", "iaskit_last_error", "iaskit_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    import paper_1602_01376_gb300 as ia
    assert sorted(ia.EXPORTS) == declared_symbols()
    for n in declared_symbols():
        assert callable(getattr(ia, n))


def test_error_paths_without_device_work(lib_path):
    import paper_1602_01376_gb300 as ia
    ia.load(lib_path)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_set_option("no_such_option", 1.0)
    assert e.value.name == "IASKIT_ERR_ARG"
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_set_option("kappa", 0)
    assert e.value.name == "IASKIT_ERR_ARG"
    ia.iaskit_set_option("seed", 5)
    assert ia.iaskit_get_option("seed") == 5.0
    ia.iaskit_set_option("seed", 0)
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_depth()
    assert e.value.name == "IASKIT_ERR_NOT_FACTORED"
    # refactoring needs a factorization; option checks need no device
    with pytest.raises(ia.IaskitError) as e:
        ia.iaskit_refactor(0.1)
    assert e.value.name == "IASKIT_ERR_NOT_FACTORED"
    for bad in (2, -1):
        with pytest.raises(ia.IaskitError) as e:
            ia.iaskit_set_option("near_field", bad)
        assert e.value.name == "IASKIT_ERR_ARG"
    ia.iaskit_set_option("near_field", 1)
    assert ia.iaskit_get_option("near_field") == 1.0
    ia.iaskit_set_option("near_field", 0)


def test_kernels_are_compiled_for_sm103a_only():
    from paper_1602_01376_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_committed_tile_table_is_well_formed():
    # the autotuner's committed cache: valid buckets and CUDA-core shapes
    import json
    import paper_1602_01376_gb300 as ia
    if not os.path.exists(ia.TILE_TABLE):
        pytest.skip("no committed tile table")
    with open(ia.TILE_TABLE) as f:
        table = json.load(f)
    assert table["entries"]
    for e in table["entries"]:
        assert e["fp64"] in (0, 1)
        assert 0 <= e["n_bucket"] < 6 and 0 <= e["m_bucket"] < 5
        assert e["shape"] in ia.GEMM_SHAPES
        assert not (e["fp64"] and e["shape"] == "512x8")
        assert e["shape"] == min(e["ms"], key=e["ms"].get)
