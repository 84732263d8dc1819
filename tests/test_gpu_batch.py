"""Batched probabilities (gbs_torontonian_batch): uneven requests in one pass.

Each request of a batch must equal the oracle (relative 1e-9 when the
precision ladder certifies it) and be bitwise identical to the same request
evaluated alone: every tree owns its plan regions and is reduced in a fixed
order that does not depend on its neighbours.
"""
import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import ref_method

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def requests(ctx, n, seed, Ms=(30, 60, 100), N_range=(1, 12)):
    reqs = gi.batched_requests(n, seed=seed, Ms=Ms, N_range=N_range)
    states, pats, params = [], [], []
    for q in reqs:
        U = gi.haar_unitary(q.M, q.seed)
        r = np.full(q.M, q.r)
        states.append(gbs.build_state(ctx, U, r, q.eta))
        pats.append(q.modes)
        params.append((U, r, q.eta))
    return states, pats, params


@pytest.mark.parametrize("basis", ["real", "complex"])
def test_batch_matches_oracle_and_single(ctx, basis):
    states, pats, params = requests(ctx, 24, seed=7)
    res = gbs.torontonian_batch(ctx, states, pats, "auto", basis)
    for i, (st, pat, (U, r, eta)) in enumerate(zip(states, pats, params)):
        p_ref, _, kappa = oracle.click_probability(U, r, eta, pat, method=ref_method(len(pat)))
        assert abs(res[i].p - p_ref) <= 1e-9 * abs(p_ref), (i, len(pat), res[i], p_ref)
        alone = gbs.torontonian(ctx, st, pat, res[i].prec, basis)
        assert alone.p == res[i].p and alone.tor == res[i].tor and alone.abs_sum == res[i].abs_sum


def test_batch_result_independent_of_neighbours(ctx):
    states, pats, _ = requests(ctx, 40, seed=11, Ms=(100, 200), N_range=(8, 16))
    full = gbs.torontonian_batch(ctx, states, pats, "fp64", "real")
    sub_idx = [3, 17, 29, 5]
    sub = gbs.torontonian_batch(ctx, [states[i] for i in sub_idx], [pats[i] for i in sub_idx], "fp64", "real")
    for j, i in enumerate(sub_idx):
        assert sub[j].tor == full[i].tor and sub[j].abs_sum == full[i].abs_sum


def test_batch_with_empty_and_tiny_patterns(ctx):
    U = gi.haar_unitary(10, 2)
    st = gbs.build_state(ctx, U, np.full(10, 0.6), 0.9)
    pats = [[], [3], [0, 9], list(range(10)), [4, 5, 6]]
    res = gbs.torontonian_batch(ctx, [st] * len(pats), pats, "auto", "auto")
    for pat, pr in zip(pats, res):
        p_ref, _, _ = oracle.click_probability(U, np.full(10, 0.6), 0.9, pat, method=ref_method(len(pat)))
        assert abs(pr.p - p_ref) <= 1e-9 * p_ref


def test_batch_fp32_diagnostic_and_td(ctx):
    states, pats, params = requests(ctx, 6, seed=3, N_range=(4, 10))
    for prec, tol in (("fp32", None), ("td", 1e-12)):
        res = gbs.torontonian_batch(ctx, states, pats, prec, "real")
        for pr, pat, (U, r, eta) in zip(res, pats, params):
            p_ref, _, kappa = oracle.click_probability(U, r, eta, pat, method=ref_method(len(pat)))
            bound = tol if tol else 8 * len(pat) * 2.0 ** -24 * kappa
            assert abs(pr.p - p_ref) <= bound * abs(p_ref) + 1e-300


def test_auto_rungs_do_not_depend_on_batch_neighbours(ctx):
    # The precision ladder of a request depends on that request alone: a 12-click request
    # (cancellation far beyond FP64) takes the same rungs and gives the bitwise same value
    # alone and batched with a 20-click request (which uses the a-priori estimate).
    st_p, modes24 = gi.single_large_torontonian_workload()
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    small, big = modes24[:12], modes24[:20]
    alone = gbs.torontonian_batch(ctx, [st], [small], "auto", "real")[0]
    mixed = gbs.torontonian_batch(ctx, [st, st], [small, big], "auto", "real")
    assert alone.prec == mixed[0].prec and alone.p == mixed[0].p and alone.tor == mixed[0].tor
    assert mixed[1].err_bound <= 1e-10 * abs(mixed[1].p)
    st.free()
