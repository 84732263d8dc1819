"""Chain-rule sampler (gbs_sample) against the oracle chain (oracle.sample_chain).

Both sides draw the coin from their own SplitMix64 with the same counter
convention, so samples must be identical except for draws with |u - p0| <
1e-9 (counted as near-ties); p0 itself must agree to 1e-10 at every step.
"""
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


def make(ctx, M, seed, r=(0.5, 1.0), eta=0.8):
    U = gi.haar_unitary(M, seed)
    rr = gi.uniform_range(seed, "squeezing", M, *r)
    st = gbs.build_state(ctx, U, rr, eta)
    Sig = oracle.sigma(oracle.covariance(U, rr, eta))
    return st, Sig


def test_forced_trajectories_p0_every_step(ctx):
    M = 7
    st, Sig = make(ctx, M, 12)
    forced = np.array([[0, 3, 6], [1, 2, 5], [4, 5, 6]], dtype=np.int32)
    pats, p0, stats, status = gbs.sample(ctx, st, 3, seed=5, N_post=3, forced_clicks=forced, want_p0=True)
    assert status == 0
    for i in range(3):
        ref = oracle.sample_chain(Sig, 5, sample=i, forced_clicks=forced[i])
        assert np.array_equal(np.nonzero(pats[i])[0], np.sort(forced[i]))
        assert np.allclose(p0[i], np.array(ref["p0"]), rtol=0, atol=1e-10), (p0[i], ref["p0"])


@pytest.mark.parametrize("prec", ["auto", "dd", "fxn", "fx", "fxw"])
def test_free_samples_match_oracle(ctx, prec):
    M = 6
    st, Sig = make(ctx, M, 21, r=(0.6, 1.1), eta=0.9)
    n = 12
    pats, p0, stats, status = gbs.sample(ctx, st, n, seed=77, prec=prec, want_p0=True)
    assert status == 0
    near = 0
    for i in range(n):
        ref = oracle.sample_chain(Sig, 77, sample=i)
        near += ref["near_ties"]
        if ref["near_ties"] == 0:
            assert np.array_equal(pats[i], ref["pattern"]), i
            assert np.allclose(p0[i], np.array(ref["p0"]), rtol=0, atol=1e-10)
    assert stats["near_ties"] == near
    assert stats["uncertified"] == 0 or prec != "auto"


def test_postselected_samples_match_oracle(ctx):
    M = 8
    st, Sig = make(ctx, M, 33, r=(0.4, 0.9), eta=0.7)
    n, N_post, attempts = 6, 3, 40
    pats, p0, stats, status = gbs.sample(ctx, st, n, seed=9, N_post=N_post, max_attempts=attempts)
    for i in range(n):
        ref = oracle.sample_chain(Sig, 9, sample=i, N_post=N_post, max_attempts=attempts)
        if ref["pattern"] is None:
            assert np.all(pats[i] == 0xFF)
        else:
            assert np.array_equal(pats[i], ref["pattern"])
            assert pats[i].sum() == N_post
    assert stats["rejections"] > 0


def test_bigger_forced_trajectory_sampled_steps(ctx):
    # 60 modes, 8 forced clicks; the oracle recomputes the conditioned state from
    # scratch at a few steps, including the last ones where most clicks are in.
    M = 60
    st, Sig = make(ctx, M, 2, r=(0.3, 0.9), eta=1.0)
    forced = gi.random_modes(M, 8, 2, stream="clicks")
    pats, p0, stats, status = gbs.sample(ctx, st, 1, seed=1, N_post=8, forced_clicks=forced[None, :], want_p0=True)
    assert status == 0
    steps = [0, 17, 45, 58, 59]
    ref = oracle.sample_chain(Sig, 1, forced_clicks=forced, steps_to_check=set(steps))
    for s in steps:
        assert abs(p0[0][s] - ref["p0"][s]) <= 1e-10, (s, p0[0][s], ref["p0"][s])
    # one tree per step once the first click is in (steps before it need none)
    assert 0 < stats["steps"] <= 2 * M
    assert np.all(np.isfinite(p0[0])) and np.all((p0[0] > 0) & (p0[0] < 1))


def test_forced_trajectory_fixed_point_equals_triple_double(ctx):
    # 40 modes, 12 forced clicks: p0 at every step in fixed point and in
    # triple-double agree far below the 5e-10 target
    M = 40
    st, Sig = make(ctx, M, 8, r=(0.4, 0.9), eta=0.9)
    forced = gi.random_modes(M, 12, 8, stream="clicks")[None, :].astype(np.int32)
    _, p_fx, s_fx, st1 = gbs.sample(ctx, st, 1, seed=3, N_post=12, forced_clicks=forced, prec="fx", want_p0=True)
    _, p_td, s_td, st2 = gbs.sample(ctx, st, 1, seed=3, N_post=12, forced_clicks=forced, prec="td", want_p0=True)
    _, p_fw, s_fw, st3 = gbs.sample(ctx, st, 1, seed=3, N_post=12, forced_clicks=forced, prec="fxw", want_p0=True)
    _, p_fn, s_fn, st4 = gbs.sample(ctx, st, 1, seed=3, N_post=12, forced_clicks=forced, prec="fxn", want_p0=True)
    assert st1 == 0 and st2 == 0 and st3 == 0 and st4 == 0
    assert np.max(np.abs(p_fx - p_td)) < 1e-20 and np.max(np.abs(p_fw - p_td)) < 1e-20
    assert np.max(np.abs(p_fn - p_td)) < 1e-15
    assert s_fx["trees"][3] > 0 and s_fx["trees"][2] == 0 and s_td["trees"][2] > 0 and s_fw["trees"][4] > 0
    assert s_fn["trees"][5] > 0


def test_forced_random_positions_equal_explicit_positions(ctx):
    # gbs_sample_forced_random draws the click positions from the seed and runs the forced chain:
    # the same as gbs_sample given those positions, and p0 at every step as the oracle's chain
    M = 40
    st, Sig = make(ctx, M, 8, r=(0.4, 0.9), eta=0.9)
    pos = gbs.draw_click_positions(M, 6, 17, 3)
    pats, p0, stats = gbs.sample_forced_random(ctx, st, 3, seed=17, n_clicks=6, want_p0=True)
    pats2, p02, _, status = gbs.sample(ctx, st, 3, seed=17, N_post=6, forced_clicks=pos, want_p0=True)
    assert status == 0 and np.array_equal(pats, pats2) and np.array_equal(p0, p02)
    for i in range(3):
        assert np.nonzero(pats[i])[0].tolist() == pos[i].tolist()
    ref = oracle.sample_chain(Sig, 17, sample=0, forced_clicks=pos[0])
    assert np.allclose(p0[0], np.array(ref["p0"]), rtol=0, atol=1e-10)
