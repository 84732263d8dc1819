"""Pins of the oracle's probabilities against closed forms, invariants, the paper's
own mixture algorithm, photon-number brute force and the paper's printed numbers."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gbs_inputs as gi
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return abs(a - b) / abs(b)


# ---------------------------------------------------------- closed forms --

@pytest.mark.parametrize("eta", [1.0, 0.6, 0.25])
def test_single_mode_click_probability(eta):
    for r in (0.1, 0.5, 0.9, 1.7):
        st = gi.identity_state([r], eta)
        p, tor, _ = oracle.click_probability(st.U, st.r, st.eta, [0])
        assert rel(p, oracle.single_mode_click_probability(r, eta)) < 1e-13
        if eta == 1.0:
            assert rel(p, 1.0 - 1.0 / math.cosh(r)) < 1e-13


@pytest.mark.parametrize("method", ["bruteforce", "tree"])
def test_identity_interferometer_product_formula(method):
    rng = np.random.default_rng(11)
    r = rng.uniform(0.2, 1.5, size=12)
    for eta in (1.0, 0.5):
        st = gi.identity_state(r, eta)
        Sig = oracle.sigma(oracle.covariance(st.U, st.r, eta))
        for N in (1, 3, 7, 10):
            modes = sorted(rng.choice(12, size=N, replace=False).tolist())
            H = oracle.sigma_inv_block(Sig, modes)
            tor, _ = oracle.torontonian(H, method)
            assert rel(float(tor), oracle.identity_torontonian(r, eta, modes)) < 1e-12


def test_identity_interferometer_n20_tree():
    r = np.linspace(1.6, 2.2, 20)
    st = gi.identity_state(r, 1.0)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, 1.0))
    H = oracle.sigma_inv_block(Sig, range(20))
    tor, asum = oracle.torontonian(H, "tree")
    assert rel(float(tor), oracle.identity_torontonian(r, 1.0, range(20))) < 1e-12


# ------------------------------------------------------------ invariants --

def test_vacuum_torontonian():
    st = gi.identity_state(np.zeros(6))
    Sig = oracle.sigma(oracle.covariance(gi.haar_unitary(6, 4), st.r, 1.0))
    for N in range(1, 6):
        H = oracle.sigma_inv_block(Sig, range(N))
        tor, _ = oracle.torontonian(H)
        assert abs(float(tor)) < 1e-14
    tor0, _ = oracle.torontonian(np.zeros((0, 0), dtype=complex))
    assert float(tor0) == 1.0


def test_all_patterns_sum_to_one_small_workload():
    st, pats = gi.small_all_patterns_workload()
    ps = oracle.all_pattern_probabilities(st.U, st.r, st.eta)
    assert ps.min() > 0
    assert abs(ps.sum() - 1.0) < 1e-13


def test_all_patterns_sum_to_one_lossy():
    U = gi.haar_unitary(6, 9)
    r = gi.uniform_range(9, "squeezing", 6, 0.3, 1.0)
    ps = oracle.all_pattern_probabilities(U, r, 0.4)
    assert abs(ps.sum() - 1.0) < 1e-13


def test_sigma_form_equals_inverse_form():
    U = gi.haar_unitary(6, 21)
    r = gi.uniform_range(21, "squeezing", 6, 0.3, 1.0)
    V = oracle.covariance(U, r, 0.7)
    for modes in ([0], [1, 4], [0, 2, 3, 5], list(range(6))):
        p_inv, _, _ = oracle.click_probability(U, r, 0.7, modes)
        p_sig = oracle.click_probability_sigma_form(V, modes)
        assert rel(p_sig, p_inv) < 1e-11


def test_marginal_consistency():
    # p over modes T with clicks S = p over T+k with clicks S+k  +  p over T+k with clicks S.
    U = gi.haar_unitary(7, 5)
    r = np.full(7, 0.7)
    Sig = oracle.sigma(oracle.covariance(U, r, 0.8))

    def p_marg(T, S):
        # reduced state of the modes T, kept in block order (a_T, a_T^+)
        ix = np.concatenate([np.array(T), np.array(T) + 7])
        SigT = Sig[np.ix_(ix, ix)]
        loc = [T.index(j) for j in S]
        H = oracle.sigma_inv_block(SigT, loc)
        tor, _ = oracle.torontonian(H)
        return float(tor) * math.exp(-0.5 * oracle.logdet_sigma(SigT))

    T = [0, 2, 3, 6]
    S = [2, 6]
    k = 4
    lhs = p_marg(T, S)
    rhs = p_marg(sorted(T + [k]), S + [k]) + p_marg(sorted(T + [k]), S)
    assert rel(lhs, rhs) < 1e-12


def test_permutation_and_phase_invariance():
    U = gi.haar_unitary(8, 13)
    r = np.full(8, 0.6)
    modes = [1, 3, 4, 6, 7]
    p, _, _ = oracle.click_probability(U, r, 1.0, modes)
    perm = np.random.default_rng(2).permutation(8)
    Up = U[perm, :]  # relabel output ports
    inv = np.argsort(perm)
    modes_p = sorted(int(inv[j]) for j in modes)
    pp, _, _ = oracle.click_probability(Up, r, 1.0, modes_p)
    assert rel(pp, p) < 1e-12
    ph = np.exp(1j * np.random.default_rng(3).uniform(0, 2 * np.pi, 8))
    pq, _, _ = oracle.click_probability(ph[:, None] * U, r, 1.0, modes)
    assert rel(pq, p) < 1e-12


def test_real_basis_determinants_and_eq5():
    U = gi.haar_unitary(5, 17)
    r = np.array([0.3, 0.8, 0.5, 1.1, 0.2])
    V = oracle.covariance(U, r, 0.9)
    Vr = oracle.to_real_basis(V)
    assert np.allclose(oracle.from_real_basis(Vr), V, atol=1e-13)
    Sig = oracle.sigma(V)
    for modes in ([0], [2, 4], [0, 1, 3]):
        # paper's Eq. (5): q = 2^k / sqrt(det(V_B + 1)) for k modes (2 per mode), hbar = 2
        ixr = np.array([[2 * j, 2 * j + 1] for j in modes]).ravel()
        q_paper = 2.0 ** len(modes) / math.sqrt(np.linalg.det(Vr[np.ix_(ixr, ixr)] + np.eye(2 * len(modes))))
        assert rel(q_paper, oracle.vacuum_probability(Sig, modes)) < 1e-12


# ------------------------------------------- the paper's mixture algorithm --

def test_paper_mixture_algorithm_matches_torontonian():
    U = gi.haar_unitary(5, 31)
    r = gi.uniform_range(31, "squeezing", 5, 0.3, 1.0)
    eta = 0.8
    V = oracle.covariance(U, r, eta)
    Vr = oracle.to_real_basis(V)
    ps = oracle.all_pattern_probabilities(U, r, eta)
    for m in range(32):
        clicks = [j for j in range(5) if (m >> j) & 1]
        pm = oracle.mixture_pattern_probability(Vr, clicks)
        assert abs(pm - ps[m]) < 1e-12 * max(1.0, 1 / ps[m]) * ps[m] + 1e-15


# ------------------------------------------- photon-number brute force --

def test_pnr_hafnian_sum_matches_click_probability():
    U = gi.haar_unitary(3, 41)
    r = np.array([0.35, 0.25, 0.3])
    for clicks in ([0], [0, 2], [0, 1, 2]):
        p, _, _ = oracle.click_probability(U, r, 1.0, clicks)
        part, total = oracle.pnr_click_probability(U, r, clicks, n_max=12)
        tail = 1.0 - total
        assert 0 <= tail < 1e-5
        assert part <= p + 1e-15
        assert p - part <= tail + 1e-14


def test_hafnian_known_values():
    A = np.ones((4, 4))
    assert oracle.hafnian(A) == 3.0
    B = np.arange(16, dtype=float).reshape(4, 4)
    B = B + B.T
    # haf = b01 b23 + b02 b13 + b03 b12
    assert oracle.hafnian(B) == B[0, 1] * B[2, 3] + B[0, 2] * B[1, 3] + B[0, 3] * B[1, 2]


# ---------------------------------------------- O2 against O1 (the definition) --

@pytest.mark.parametrize("N", [1, 2, 5, 9, 12, 14, pytest.param(16, marks=pytest.mark.slow)])
def test_tree_equals_bruteforce(N):
    # O2 (the decision tree) against O1 (every subset by its own LU) up to 16 modes:
    # every GPU comparison beyond 14 modes uses O2.
    st = gi.uniform_squeezed_state(200, 0.8, seed=1)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    modes = gi.random_modes(200, 24, seed=1)[:N]
    H = oracle.sigma_inv_block(Sig, modes)
    a, asum_a = oracle.torontonian(H, "bruteforce")
    b, asum_b = oracle.torontonian(H, "tree")
    d = abs(a.to_fraction() - b.to_fraction())
    assert d <= abs(b.to_fraction()) * Fraction(1, 10 ** 40)
    assert rel(asum_a, asum_b) < 1e-14


def test_tree_fixed_modes_equal_bruteforce():
    U = gi.haar_unitary(9, 8)
    r = np.full(9, 0.7)
    Sig = oracle.sigma(oracle.covariance(U, r, 0.9))
    G = Sig[np.ix_(oracle.mode_rows(range(9), 9), oracle.mode_rows(range(9), 9))]
    F, X = [0, 2, 5, 7], [3, 8]
    for sign in ("tor", "incl"):
        a, _ = oracle.subset_sum(G, F, X, sign, "bruteforce")
        b, _ = oracle.subset_sum(G, F, X, sign, "tree")
        assert abs(a.to_fraction() - b.to_fraction()) <= abs(b.to_fraction()) * Fraction(1, 10 ** 40)


# ---------------------------------------------------------- sampler --

def test_splitmix_known_answer():
    # SplitMix64 seeded with 1234567: the published first outputs.
    assert [int(x) for x in gi.u64_block(1234567, 0, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]
    assert oracle.splitmix_uniform(1234567, 0, 0) == (6457827717110365317 >> 11) * 2.0 ** -53


def test_chain_probabilities_multiply_to_pattern_probability():
    U = gi.haar_unitary(6, 51)
    r = np.full(6, 0.8)
    Sig = oracle.sigma(oracle.covariance(U, r, 0.7))
    ps = oracle.all_pattern_probabilities(U, r, 0.7)
    for m in (0b000000, 0b101001, 0b111111, 0b010110):
        clicks = [j for j in range(6) if (m >> j) & 1]
        res = oracle.sample_chain(Sig, 0, forced_clicks=clicks)
        prob = 1.0
        for step, k in enumerate(range(5, -1, -1)):
            p0 = res["p0"][step]
            prob *= (1 - p0) if k in clicks else p0
        assert rel(prob, ps[m]) < 1e-11


def test_free_sampling_frequencies():
    # The chain with the seeded coin reproduces the pattern distribution.
    U = gi.haar_unitary(4, 61)
    r = np.full(4, 0.9)
    Sig = oracle.sigma(oracle.covariance(U, r, 1.0))
    ps = oracle.all_pattern_probabilities(U, r, 1.0)
    n = 600
    counts = np.zeros(16)
    for s in range(n):
        pat = oracle.sample_chain(Sig, 99, sample=s)["pattern"]
        counts[int(sum(int(b) << j for j, b in enumerate(pat)))] += 1
    # chi-square-like bound: every bin within 5 sigma of its expectation
    exp = ps * n
    assert np.all(np.abs(counts - exp) <= 5 * np.sqrt(exp * (1 - ps)) + 1)


# ------------------------------------------------------ the paper's Table I --

def test_memory_model_reproduces_table_1():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_memory.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                ell, m, gb = line.split()
                rows.append((int(ell), int(m), float(gb)))
    assert len(rows) == 4
    for ell, m, gb in rows:
        val = oracle.memory_gb(ell, m, k=m, eta=2.0)
        digits = len(str(gb).split(".")[1]) if "." in str(gb) and gb < 1000 else 0
        assert abs(val - gb) <= 0.5 * 10.0 ** -digits + 1e-12 * gb, (ell, m, val, gb)
