"""Full-size parity: the N = 24 Torontonian of the 200-mode workload, in the launch
configuration the benchmark times, against the oracle's stored value
(tests/golden/tor_n24_m200.txt, written by tests/golden/make_golden.py).

The inputs are regenerated from their seeds here; a different platform's
LAPACK may round the Haar unitary differently in the last bits, which moves
Tor by ~1e-13 relative (Tor is well conditioned in its matrix), far inside 1e-9.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gbs_inputs as gi
import paper_1810_00900_gb300 as gbs
from helpers import td_value

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "tor_n24_m200.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = [float(x) for x in v]
    tor = sum((Fraction(x) for x in vals["tor_components"]), Fraction(0))
    return float(tor), vals["abs_sum"][0], vals["p"][0]


@pytest.fixture(scope="module")
def ctx_state():
    from paper_1810_00900_gb300 import build
    build.build()
    ctx = gbs.Context(0)
    st_p, modes = gi.single_large_torontonian_workload(24)
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    yield ctx, st, modes
    st.free()
    ctx.close()


def test_n24_triple_double_matches_oracle(ctx_state):
    ctx, st, modes = ctx_state
    tor_ref, abs_ref, p_ref = golden()
    pr = gbs.torontonian(ctx, st, modes, "td", "real")
    assert abs(pr.tor_value - tor_ref) <= 1e-9 * abs(tor_ref)
    assert abs(pr.p - p_ref) <= 1e-9 * abs(p_ref)
    assert abs(pr.abs_sum - abs_ref) <= 1e-12 * abs_ref


@pytest.mark.parametrize("prec", ["fx", "fxw"])
def test_n24_fixed_point_matches_oracle(ctx_state, prec):
    ctx, st, modes = ctx_state
    tor_ref, abs_ref, p_ref = golden()
    pr = gbs.torontonian(ctx, st, modes, prec, "real")
    assert abs(pr.tor_value - tor_ref) <= 1e-9 * abs(tor_ref)
    assert abs(pr.p - p_ref) <= 1e-9 * abs(p_ref)
    assert abs(pr.abs_sum - abs_ref) <= 1e-12 * abs_ref
    assert pr.err_bound <= 1e-12 * abs(pr.p)


def test_n24_auto_reaches_tolerance(ctx_state):
    ctx, st, modes = ctx_state
    tor_ref, _, p_ref = golden()
    pr = gbs.torontonian(ctx, st, modes, "auto", "real")
    # kappa ~ 1e26: FP64 cannot certify 1e-9; the state bounds the tree, so the
    # fixed-point rung (before triple-double) is the one that does
    assert pr.prec == "fx"
    assert abs(pr.p - p_ref) <= 1e-9 * abs(p_ref)
    pc = gbs.torontonian(ctx, st, modes, "auto", "complex")
    assert pc.prec == "td"  # fixed point is real-basis only
    assert abs(pc.p - p_ref) <= 1e-9 * abs(p_ref)


def test_n24_fp64_throughput_configuration_sums_all_terms(ctx_state):
    # The FP64 run the benchmark times: its value is not accurate at this kappa,
    # but its sum of |terms| (no cancellation) must match the oracle's.
    ctx, st, modes = ctx_state
    _, abs_ref, _ = golden()
    for basis in ("real", "complex"):
        pr = gbs.torontonian(ctx, st, modes, "fp64", basis)
        assert abs(pr.abs_sum - abs_ref) <= 1e-12 * abs_ref
        assert pr.err_bound > abs(pr.p) * 1e-9  # honestly flagged as uncertified


@pytest.mark.parametrize("prec", ["fp64", "fp64p", "dd", "fxn"])
def test_n24_error_bound_holds_in_every_precision(ctx_state, prec):
    # the precisions that cannot certify 1e-9 at kappa ~ 1e26 still bound their own error
    ctx, st, modes = ctx_state
    _, _, p_ref = golden()
    pr = gbs.torontonian(ctx, st, modes, prec, "real")
    assert pr.prec == prec
    assert abs(pr.p - p_ref) <= pr.err_bound, (prec, pr.p, p_ref, pr.err_bound)
