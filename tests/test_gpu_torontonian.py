"""End-to-end click probabilities (gbs_build_state + gbs_torontonian) vs the oracle.

The GPU forms Sigma^-1 blocks by the closed form and the oracle by a dense numpy
inverse; the Torontonian is well conditioned in its matrix (relative change ~1e2
times the perturbation), so the two agree to ~1e-13 when both enumerations are
accurate.  The bar is the relative error 1e-9.
"""
import math

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import ref_method

pytestmark = pytest.mark.gpu
REL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def test_small_workload_all_256_patterns_sum_to_one(ctx):
    st_p, patterns = gi.small_all_patterns_workload()
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    ref = oracle.all_pattern_probabilities(st_p.U, st_p.r, st_p.eta)
    got = np.array([gbs.torontonian(ctx, st, S, "auto", "auto").p for S in patterns])
    rel = np.abs(got - ref) / ref
    assert rel.max() < REL, rel.max()
    assert abs(got.sum() - 1.0) < 1e-13
    for basis in ("real", "complex"):
        for S in (patterns[0], patterns[37], patterns[255]):
            m = int(sum(1 << j for j in S))
            pr = gbs.torontonian(ctx, st, S, "auto", basis)
            assert abs(pr.p - ref[m]) < REL * ref[m]


@pytest.mark.parametrize("N", [0, 1, 4, 9, 13, 16])
def test_large_state_patterns_auto_precision(ctx, N):
    st_p, modes24 = gi.single_large_torontonian_workload()
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    modes = modes24[:N]
    p_ref, tor_ref, kappa = oracle.click_probability(st_p.U, st_p.r, st_p.eta, modes, method=ref_method(len(modes)))
    pr = gbs.torontonian(ctx, st, modes, "auto", "real")
    assert abs(pr.p - p_ref) <= REL * abs(p_ref), (N, pr, p_ref)
    assert pr.err_bound <= REL * abs(pr.p)
    if N >= 9:
        assert pr.prec != "fp64"  # kappa is far beyond FP64 here


@pytest.mark.parametrize("prec", ["fp64", "dd", "td"])
def test_lossy_requests_complex_basis(ctx, prec):
    for i, req in enumerate(gi.batched_requests(6, seed=5, Ms=(40, 60), N_range=(3, 9))):
        U = gi.haar_unitary(req.M, req.seed)
        r = np.full(req.M, req.r)
        st = gbs.build_state(ctx, U, r, req.eta)
        p_ref, _, kappa = oracle.click_probability(U, r, req.eta, req.modes, method=ref_method(req.N))
        pr = gbs.torontonian(ctx, st, req.modes, prec, "complex")
        tol = max(REL, 8 * req.N * {"fp64": 2.0 ** -53, "dd": 2.0 ** -102, "td": 2.0 ** -152}[prec] * kappa)
        assert abs(pr.p - p_ref) <= tol * abs(p_ref) + 1e-300, (i, prec, pr.p, p_ref, kappa)
        st.free()


def test_single_mode_and_vacuum(ctx):
    st = gbs.build_state(ctx, np.eye(3), [0.7, 0.0, 1.2], 0.6)
    pr = gbs.torontonian(ctx, st, [0], "fp64")
    want = oracle.single_mode_click_probability(0.7, 0.6) * (1 - oracle.single_mode_click_probability(1.2, 0.6))
    assert abs(pr.p - want) < 1e-14
    assert gbs.torontonian(ctx, st, [1], "dd").p == 0.0
    pr0 = gbs.torontonian(ctx, st, [], "auto")
    assert abs(pr0.p - math.exp(-0.5 * oracle.logdet_sigma(oracle.sigma(oracle.covariance(np.eye(3), [0.7, 0, 1.2], 0.6))))) < 1e-15
