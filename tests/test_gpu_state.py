"""GPU state construction and Sigma^-1 click blocks vs the oracle (FP64 data path)."""
import math

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import real_basis_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("M,eta", [(1, 1.0), (8, 1.0), (37, 0.6), (200, 0.25)])
def test_covariance_matches_oracle(ctx, M, eta):
    U = gi.haar_unitary(M, 7)
    r = gi.uniform_range(7, "squeezing", M, 0.3, 1.0)
    st, V = gbs.build_state(ctx, U, r, eta, want_V=True)
    Vo = oracle.covariance(U, r, eta)
    assert np.abs(V - Vo).max() <= 1e-13 * max(1.0, np.abs(Vo).max()) * M ** 0.5
    ld = oracle.logdet_sigma(oracle.sigma(Vo))
    assert abs(st.logdet_sigma - ld) <= 1e-12 * max(1.0, abs(ld))
    st.free()


@pytest.mark.parametrize("basis", ["complex", "real"])
def test_closed_form_click_block(ctx, basis):
    M = 120
    U = gi.haar_unitary(M, 3)
    r = gi.uniform_range(3, "squeezing", M, 0.4, 1.0)
    st = gbs.build_state(ctx, U, r, 0.8)
    Sig = oracle.sigma(oracle.covariance(U, r, 0.8))
    for N in (1, 5, 24):
        modes = gi.random_modes(M, N, 11)
        H = gbs.sigma_inv_block(ctx, st, modes, basis)
        Ho = oracle.sigma_inv_block(Sig, modes)
        if basis == "real":
            Ho = real_basis_block(Ho)
        assert np.abs(H - Ho).max() <= 1e-12


@pytest.mark.parametrize("basis", ["complex", "real"])
def test_state_from_V(ctx, basis):
    M = 24
    U = gi.haar_unitary(M, 4)
    r = gi.uniform_range(4, "squeezing", M, 0.3, 0.9)
    V = oracle.covariance(U, r, 0.9)
    st = gbs.state_from_V(ctx, V)
    Sig = oracle.sigma(V)
    assert abs(st.logdet_sigma - oracle.logdet_sigma(Sig)) <= 1e-11
    modes = [0, 3, 7, 19, 23]
    H = gbs.sigma_inv_block(ctx, st, modes, basis)
    Ho = oracle.sigma_inv_block(Sig, modes)
    if basis == "real":
        Ho = real_basis_block(Ho)
    assert np.abs(H - Ho).max() <= 1e-11


def test_bad_inputs_rejected(ctx):
    U = gi.haar_unitary(4, 1)
    with pytest.raises(gbs.GbsError) as e:
        gbs.build_state(ctx, U, np.full(4, 0.5), 1.5)
    assert e.value.status == 1
    with pytest.raises(gbs.GbsError) as e:
        gbs.state_from_V(ctx, -np.eye(8, dtype=complex))
    assert e.value.status == 3
    st = gbs.build_state(ctx, U, np.full(4, 0.5), 1.0)
    for modes in ([0, 0], [4], [-1]):
        with pytest.raises(gbs.GbsError):
            gbs.torontonian(ctx, st, modes)
