"""The C ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes

import pytest

from paper_1810_00900_gb300 import _lib, build


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = _lib.header_functions()
    for required in ("gbs_ctx_create", "gbs_ctx_destroy", "gbs_build_state", "gbs_state_from_V",
                     "gbs_torontonian", "gbs_sigma_inv_block", "gbs_subset_sum", "gbs_state_free"):
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _lib.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_loads_and_status_strings(libpath):
    L = _lib.load()
    assert L.gbs_status_string(0) == b"ok"
    assert L.gbs_status_string(3) == b"matrix not positive definite"


def test_no_gpu_context_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(_lib.GbsError):
        _lib.Context(0)
