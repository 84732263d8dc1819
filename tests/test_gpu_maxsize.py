"""Maximum sizes: the largest click patterns the API takes, checked against the closed form
that holds at any size.  With an identity interferometer the modes are independent and
Tor(O_S) = prod_{j in S} (sqrt(det Sigma_j) - 1), det Sigma_j = 1 + eta (2 - eta) sinh^2 r_j
(the paper's Eq. 5 for one mode); the GPU still runs every level of the full tree."""
import math

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def closed_form(r, eta, modes):
    tor = oracle.identity_torontonian(r, eta, modes)
    kappa = 1.0
    for j in modes:
        sd = math.sqrt(1.0 + eta * (2.0 - eta) * math.sinh(r[j]) ** 2)
        kappa *= (sd + 1.0) / (sd - 1.0)
    return tor, kappa


def test_n32_fp64_all_levels(ctx):
    # the API maximum, N = 32 (2^32 terms), in FP64; kappa ~ 3e7 keeps FP64 meaningful
    r = np.concatenate([np.linspace(1.9, 2.1, 32), np.full(4, 0.5)])
    st_p = gi.identity_state(r, 1.0)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    modes = np.arange(32)
    want, kappa = closed_form(r, 1.0, modes)
    pr = gbs.torontonian(ctx, st, modes, "fp64", "real")
    assert abs(pr.tor_value - want) <= 4 * 32 * 2.0 ** -53 * kappa * abs(want)
    assert abs(pr.kappa / kappa - 1.0) < 1e-6
    st.free()


def test_n30_fixed_point_certified(ctx):
    # N = 30 in fixed point at kappa ~ 2e25; r = 0.8 keeps the state inside the fixed-point range
    r = np.concatenate([np.full(30, 0.8), np.full(6, 0.3)])
    st_p = gi.identity_state(r, 1.0)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    modes = np.arange(30)
    want, kappa = closed_form(r, 1.0, modes)
    pr = gbs.torontonian(ctx, st, modes, "auto", "real")
    assert pr.prec == "fx"
    assert abs(pr.tor_value - want) <= 1e-12 * abs(want)
    assert pr.err_bound <= 1e-10 * abs(pr.p)
    st.free()


def test_n24_lossy_wide_fixed_point_and_fp64_agree_on_abs(ctx):
    # a lossy Haar state at N = 24: the wide fixed point against the closed-form-free
    # invariants -- tor = inc + exc exactly, abs_sum equal to the FP64 run's
    st_p = gi.uniform_squeezed_state(120, 0.7, seed=31, eta=0.6)
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    modes = gi.random_modes(120, 24, seed=31)
    pw = gbs.torontonian(ctx, st, modes, "fxw", "real")
    p64 = gbs.torontonian(ctx, st, modes, "fp64", "real")
    pf = gbs.torontonian(ctx, st, modes, "fx", "real")
    assert abs(pw.abs_sum / p64.abs_sum - 1.0) < 1e-12
    assert abs(pw.tor_value - pf.tor_value) <= 1e-12 * abs(pw.tor_value)
    st.free()


def test_auto_skips_fp64_for_large_trees_and_predicts_the_narrow_width(ctx):
    # 18 independent modes, kappa = prod (sqrt(d)+1)/(sqrt(d)-1) ~ 1e12 (the a-priori estimate is
    # exact for independent modes): FP64 cannot reach 1e-10 and a tree of 16+ modes skips it; the
    # estimate predicts the 128-bit fixed point suffices
    r = np.concatenate([np.full(18, 1.0), np.full(4, 0.5)])
    st_p = gi.identity_state(r, 1.0)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    modes = np.arange(18)
    want, kappa = closed_form(r, 1.0, modes)
    assert 1e11 < kappa < 1e13
    pr = gbs.torontonian(ctx, st, modes, "auto", "real")
    assert pr.prec == "fxn"
    assert abs(pr.tor_value - want) <= 1e-12 * abs(want)
    assert pr.err_bound <= 1e-10 * abs(pr.p)
    st.free()
