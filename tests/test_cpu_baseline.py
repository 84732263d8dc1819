"""The bench's same-precision CPU baseline (cpu_baseline/, a plain FP64 decision tree with OpenMP)
against the oracle, within the FP64 error model of the subset sums (8 n u sum|terms|), on one
thread and on several, and with different prefix splits (the split only shares out the work)."""
import numpy as np
import pytest

import cpu_baseline
import gbs_inputs as gi
import oracle
from helpers import real_basis_block


def block(N, seed=1, M=120, r=0.7, eta=0.8):
    st = gi.uniform_squeezed_state(M, r, seed=seed, eta=eta)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    return real_basis_block(oracle.sigma_inv_block(Sig, gi.random_modes(M, N, seed=seed)))


@pytest.mark.parametrize("N", [1, 2, 5, 9])
def test_matches_oracle(N):
    G = block(N)
    ref, ref_abs = oracle.torontonian(G.astype(np.complex128), "bruteforce")
    for threads, split in ((1, 0), (0, 3), (2, N)):
        tor, asum, _ = cpu_baseline.torontonian_fp64(G, threads, split)
        assert abs(tor - float(ref.to_fraction())) <= 8 * N * 2.0 ** -53 * ref_abs
        assert abs(asum - ref_abs) <= 1e-12 * ref_abs


def test_independent_modes_closed_form():
    # identity interferometer: Tor = prod_j (sqrt(det Sigma_j) - 1), exact up to FP64 rounding
    r = np.array([0.3, 0.9, 0.5, 1.2, 0.7])
    st = gi.identity_state(r, 0.7)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    G = real_basis_block(oracle.sigma_inv_block(Sig, range(5)))
    tor, _, _ = cpu_baseline.torontonian_fp64(G, 1, 2)
    want = oracle.identity_torontonian(r, 0.7, range(5))
    assert abs(tor - want) <= 1e-12 * abs(want)


def test_not_positive_definite_is_reported():
    G = block(4)
    G[2, 2] = -G[2, 2]
    with pytest.raises(np.linalg.LinAlgError):
        cpu_baseline.torontonian_fp64(G, 1, 0)
