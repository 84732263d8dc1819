"""The C ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes

import numpy as np

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


def test_seed_drawn_click_positions_follow_the_published_generator(libpath):
    # gbs_draw_click_positions runs on the host: it must give the positions the seeded input
    # generator's definition gives (SplitMix64 stream "clicks", partial Fisher-Yates, sorted)
    import gbs_inputs as gi
    import paper_1810_00900_gb300 as gbs
    for M, n, seed, count in ((800, 20, 2, 5), (7, 3, 5, 4), (60, 8, 2, 1), (12, 12, 9, 2)):
        got = gbs.draw_click_positions(M, n, seed, count)
        want = np.array([gi.random_modes(M, n, seed, stream="clicks", start=i * n) for i in range(count)])
        assert np.array_equal(got, want), (M, n, seed)
    # the benchmark's forced trajectories are exactly these draws
    _, clicks = gi.chain_sampling_workload(800, 20, 4, seed=2)
    assert np.array_equal(gbs.draw_click_positions(800, 20, 2, 4), np.array(clicks))
