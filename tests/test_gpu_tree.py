"""GPU subset-determinant enumeration vs the oracle, on identical input matrices.

Tolerances follow the error model of the per-term arithmetic: each of the 2^n
terms carries a relative error of at most about 4 n u (n rank-2 Schur steps and
one inverse square root), so |Tor_gpu - Tor_exact| <= 8 n u sum|terms| with
u = 2^-53 (FP64), 2^-102 (double-double), 2^-152 (triple-double); the
fixed-point type's errors are absolute (2^-160 per operation), covered by
u = 2^-140 for the matrices here (entries O(1), abs sum >= 1); the wide type
(2^-192) is limited by the three-double tree output, u = 2^-158.
"""
from fractions import Fraction

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import frac3, oracle_tor, real_basis_block

pytestmark = pytest.mark.gpu

U_OF = {"fp64": 2.0 ** -53, "dd": 2.0 ** -102, "td": 2.0 ** -152, "fp32": 2.0 ** -24, "fxn": 2.0 ** -108,
        "fx": 2.0 ** -140, "fxw": 2.0 ** -158}


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def haar_H(N, seed=1, M=200, r=0.8, eta=1.0):
    st = gi.uniform_squeezed_state(M, r, seed=seed, eta=eta)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    modes = gi.random_modes(M, N, seed=seed)
    return oracle.sigma_inv_block(Sig, modes)


def check(ctx, H, prec, basis):
    n = H.shape[0] // 2
    G = real_basis_block(H) if basis == "real" else H
    ref, ref_abs = oracle_tor(G)
    inc, exc, tor, a = gbs.subset_sum(ctx, G, basis, prec)
    err = abs(frac3(tor) - ref.to_fraction())
    bound = 8 * n * U_OF[prec] * ref_abs
    assert float(err) <= bound, (prec, basis, n, float(err), bound)
    assert abs(a - ref_abs) <= 1e-12 * ref_abs
    # tor = inc + exc
    assert abs(frac3(inc) + frac3(exc) - frac3(tor)) <= Fraction(ref_abs) * Fraction(2) ** -150
    return float(err), float(ref.to_fraction())


@pytest.mark.parametrize("basis", ["real", "complex"])
@pytest.mark.parametrize("prec", ["fp64", "dd", "td"])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 11])
def test_parity_small(ctx, prec, basis, N):
    check(ctx, haar_H(N), prec, basis)


@pytest.mark.parametrize("basis", ["real", "complex"])
@pytest.mark.parametrize("prec", ["fp64", "dd", "td"])
def test_parity_n14_lossy(ctx, prec, basis):
    check(ctx, haar_H(14, seed=5, M=100, r=0.6, eta=0.5), prec, basis)


@pytest.mark.parametrize("prec", ["dd", "td"])
def test_parity_n16_relative(ctx, prec):
    G = real_basis_block(haar_H(16))
    ref, ref_abs = oracle_tor(G)  # the same FP64 matrix on both sides
    _, _, tor, _ = gbs.subset_sum(ctx, G, "real", prec)
    rel = abs(float((frac3(tor) - ref.to_fraction()) / ref.to_fraction()))
    # kappa ~ 3e18 here: double-double still has ~1e-13 margin, triple-double far more
    assert rel < (1e-9 if prec == "dd" else 1e-20), rel


def test_identity_interferometer_closed_form(ctx):
    r = np.linspace(0.3, 1.4, 12)
    st = gi.identity_state(r, 0.7)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, 0.7))
    H = oracle.sigma_inv_block(Sig, range(12))
    want = oracle.identity_torontonian(r, 0.7, range(12))
    for basis in ("real", "complex"):
        G = real_basis_block(H) if basis == "real" else H
        _, _, tor, _ = gbs.subset_sum(ctx, G, basis, "dd")
        assert abs(tor[0] + tor[1] - want) <= 1e-13 * abs(want)


def test_vacuum_gives_zero(ctx):
    H = np.eye(12, dtype=np.complex128)
    for prec in ("fp64", "dd", "td"):
        _, _, tor, a = gbs.subset_sum(ctx, H, "complex", prec)
        assert tor[0] == 0.0 and a == 2.0 ** 6


def test_fp32_diagnostic_runs(ctx):
    H = haar_H(6)
    ref, ref_abs = oracle_tor(H)
    _, _, tor, _ = gbs.subset_sum(ctx, real_basis_block(H), "real", "fp32")
    assert abs(tor[0] + tor[1] - float(ref.to_fraction())) <= 8 * 6 * 2.0 ** -24 * ref_abs


def test_not_positive_definite_is_reported(ctx):
    H = np.eye(6, dtype=np.complex128)
    H[4, 4] = -1.0
    with pytest.raises(gbs.GbsError) as e:
        gbs.subset_sum(ctx, H, "complex", "fp64")
    assert e.value.status == 3
    # the context stays usable
    _, _, tor, _ = gbs.subset_sum(ctx, np.eye(6, dtype=np.complex128), "complex", "fp64")
    assert tor[0] == 0.0


@pytest.mark.parametrize("prec", ["fxn", "fx", "fxw"])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 11, 13])
def test_parity_fixed_point(ctx, prec, N):
    check(ctx, haar_H(N), prec, "real")


@pytest.mark.parametrize("prec", ["fxn", "fx", "fxw"])
def test_parity_fixed_point_n14_lossy_and_n16_relative(ctx, prec):
    check(ctx, haar_H(14, seed=5, M=100, r=0.6, eta=0.5), prec, "real")
    G = real_basis_block(haar_H(16))
    ref, _ = oracle_tor(G)
    _, _, tor, _ = gbs.subset_sum(ctx, G, "real", prec)
    rel = abs(float((frac3(tor) - ref.to_fraction()) / ref.to_fraction()))
    # kappa ~ 3e18: 128 fraction bits leave ~1e-13, 160 and 192 far below 1e-20
    assert rel < (1e-11 if prec == "fxn" else 1e-20), rel


@pytest.mark.parametrize("prec", ["fxn", "fx", "fxw"])
def test_fixed_point_exact_cases(ctx, prec):
    # vacuum: every term is 1, the alternating sum is exactly zero
    _, _, tor, a = gbs.subset_sum(ctx, np.eye(16), "real", prec)
    assert list(tor) == [0.0, 0.0, 0.0] and a == 2.0 ** 8
    # independent modes: Tor = prod (det(G_j)^(-1/2) - 1), here with det G_j = 1/4
    G = np.kron(np.eye(6), np.diag([0.5, 0.5]))
    _, _, tor, _ = gbs.subset_sum(ctx, G, "real", prec)
    assert frac3(tor) == Fraction(1)


def test_fixed_point_refusals(ctx):
    H = haar_H(5)
    with pytest.raises(gbs.GbsError) as e:  # complex basis
        gbs.subset_sum(ctx, H, "complex", "fx")
    assert e.value.status == 4
    G = np.eye(10)
    G[3, 3] = 1e-4  # eigenvalue below the fixed-point range: refused on the host
    with pytest.raises(gbs.GbsError) as e:
        gbs.subset_sum(ctx, G, "real", "fx")
    assert e.value.status == 4
    G = np.eye(10)
    G[8, 8] = G[9, 9] = 100.0  # eigenvalue above the fixed-point range: refused on the host
    with pytest.raises(gbs.GbsError) as e:
        gbs.subset_sum(ctx, G, "real", "fx")
    assert e.value.status == 4
    G = np.eye(10)
    G[8, 8] = G[9, 9] = 64.0  # admitted, but its pivot determinant 4096 = 2^12: reported by the device
    with pytest.raises(gbs.GbsError) as e:
        gbs.subset_sum(ctx, G, "real", "fx")
    assert e.value.status == 4
    with pytest.raises(gbs.GbsError) as e:  # the narrow width: same range, same refusals
        gbs.subset_sum(ctx, G, "real", "fxn")
    assert e.value.status == 4
    with pytest.raises(gbs.GbsError) as e:
        gbs.subset_sum(ctx, H, "complex", "fxn")
    assert e.value.status == 4
    # the context stays usable
    _, _, tor, _ = gbs.subset_sum(ctx, np.eye(10), "real", "fx")
    assert tor[0] == 0.0
