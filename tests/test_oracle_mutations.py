"""The pins catch plausible mistakes: each test plants one mistake in the oracle (on the
CPU, by replacing one of its functions for the duration of the test) and checks that at
least one of the pins -- closed forms, invariants, the paper's mixture algorithm -- no
longer holds, while all of them hold for the unmodified oracle."""

import numpy as np
import pytest

import gbs_inputs as gi
from oracle import gbs_oracle as go


def pins():
    """Small versions of the pins of test_oracle_pins.py, evaluated through the module's
    own namespace (so that a replaced function is the one used).  True = pin holds."""
    out = {}
    # closed form: one lossy squeezed mode
    r, eta = 0.9, 0.6
    st = gi.identity_state([r], eta)
    try:
        p, _, _ = go.click_probability(st.U, st.r, st.eta, [0])
        out["single_mode"] = abs(p - go.single_mode_click_probability(r, eta)) < 1e-12
    except Exception:
        out["single_mode"] = False
    # closed form: independent modes, Tor = prod (sqrt(d_j) - 1)
    rr = np.array([0.4, 0.9, 1.3, 0.7])
    st = gi.identity_state(rr, 0.7)
    try:
        Sig = go.sigma(go.covariance(st.U, st.r, 0.7))
        tor, _ = go.torontonian(go.sigma_inv_block(Sig, [0, 2, 3]), "bruteforce")
        want = go.identity_torontonian(rr, 0.7, [0, 2, 3])
        out["identity_product"] = abs(float(tor) - want) < 1e-12 * abs(want)
    except Exception:
        out["identity_product"] = False
    # invariant: vacuum has Tor = 0
    try:
        Sig = go.sigma(go.covariance(gi.haar_unitary(4, 3), np.zeros(4), 1.0))
        tor, _ = go.torontonian(go.sigma_inv_block(Sig, [0, 1, 3]), "bruteforce")
        out["vacuum"] = abs(float(tor)) < 1e-14
    except Exception:
        out["vacuum"] = False
    # invariant: the 2^M pattern probabilities are a distribution
    U = gi.haar_unitary(5, 8)
    r5 = gi.uniform_range(8, "squeezing", 5, 0.3, 0.9)
    try:
        ps = go.all_pattern_probabilities(U, r5, 0.8, "bruteforce")
        out["sum_to_one"] = bool(ps.min() > 0) and abs(ps.sum() - 1.0) < 1e-12
    except Exception:
        out["sum_to_one"] = False
    # the paper's mixture algorithm (Eqs. 3-7) on the real covariance gives the same numbers
    try:
        V = go.covariance(U, r5, 0.8)
        Vr = go.to_real_basis(V)
        agree = True
        for clicks in ([1], [0, 3], [1, 2, 4]):
            p, _, _ = go.click_probability(U, r5, 0.8, clicks)
            agree &= abs(go.mixture_pattern_probability(Vr, clicks) - p) < 1e-11
        out["mixture"] = bool(agree)
    except Exception:
        out["mixture"] = False
    # brute force: pure-state click probability = truncated photon-number sum (hafnians of
    # U tanh R U^T, built without the covariance)
    try:
        U3 = gi.haar_unitary(3, 41)
        r3 = np.array([0.35, 0.25, 0.3])
        ok = True
        for clicks in ([0], [0, 2], [0, 1, 2]):
            p, _, _ = go.click_probability(U3, r3, 1.0, clicks)
            part, total = go.pnr_click_probability(U3, r3, clicks, n_max=10)
            ok &= part <= p + 1e-15 and p - part <= (1.0 - total) + 1e-14
        out["photon_number_sum"] = bool(ok)
    except Exception:
        out["photon_number_sum"] = False
    return out


def test_unmodified_oracle_passes_every_pin():
    assert all(pins().values()), pins()


def _transposed_covariance(U, r, eta=1.0):
    r = np.asarray(r, dtype=np.float64)
    S = go.symplectic(np.asarray(U, dtype=np.complex128), r)
    V = 0.5 * (S @ S.T)  # planted: transpose instead of conjugate transpose
    V = 0.5 * (V + V.conj().T)
    M = r.shape[0]
    return eta * V + (1.0 - eta) * 0.5 * np.eye(2 * M)


def _covariance_without_loss_term(U, r, eta=1.0):
    r = np.asarray(r, dtype=np.float64)
    S = go.symplectic(np.asarray(U, dtype=np.complex128), r)
    V = 0.5 * (S @ S.conj().T)
    return eta * V  # planted: the (1 - eta) I/2 vacuum admixture is dropped


def _sigma_with_unit_shift(V):
    return V + np.eye(V.shape[0])  # planted: V + I instead of V + I/2


def _torontonian_wrong_sign(H, method="auto", nthreads=None):
    n = H.shape[0] // 2
    return go.subset_sum(H, range(n), (), "incl", method, nthreads)  # planted: (-1)^|Z| for (-1)^(N-|Z|)


def _mode_rows_shifted(modes, M):
    modes = np.asarray(modes, dtype=np.int64)
    out = np.empty(2 * modes.size, dtype=np.int64)
    out[0::2] = modes
    out[1::2] = (modes + M + 1) % (2 * M)  # planted: off-by-one on the creation-operator row
    return out


def _symplectic_swapped_blocks(U, r):
    ch, sh = np.cosh(r), np.sinh(r)
    top = np.hstack([U * ch[None, :], U.conj() * sh[None, :]])  # planted: U* where U belongs
    bot = np.hstack([U * sh[None, :], U.conj() * ch[None, :]])
    return np.vstack([top, bot])


def _logdet_full(Sig):
    sign, ld = np.linalg.slogdet(Sig)
    return 2.0 * float(ld)  # planted: p = Tor / det Sigma instead of Tor / sqrt(det Sigma)


MUTATIONS = {
    "transposed_covariance": ("covariance", _transposed_covariance),
    "dropped_loss_term": ("covariance", _covariance_without_loss_term),
    "sigma_shift": ("sigma", _sigma_with_unit_shift),
    "torontonian_sign": ("torontonian", _torontonian_wrong_sign),
    "mode_row_index": ("mode_rows", _mode_rows_shifted),
    "symplectic_blocks": ("symplectic", _symplectic_swapped_blocks),
    "determinant_power": ("logdet_sigma", _logdet_full),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_breaks_a_pin(monkeypatch, name):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(go, attr, fn)
    held = pins()
    broken = [k for k, ok in held.items() if not ok]
    assert broken, "no pin caught the planted mistake %s: %s" % (name, held)
