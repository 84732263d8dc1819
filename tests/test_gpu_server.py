"""Request loop (gbs_server_start / gbs_submit / gbs_poll): continuous batching.

A served request must give exactly the result of the same request made
directly (and therefore the same alone and in any mix); late arrivals join
running work; admission respects the arena; failures are reported on the host.
"""
import time

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from paper_1810_00900_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def states(ctx):
    out = []
    for i, (M, r, eta) in enumerate(((12, 0.7, 0.8), (20, 0.6, 0.5), (9, 0.9, 1.0))):
        U = gi.haar_unitary(M, 40 + i)
        out.append((gbs.build_state(ctx, U, np.full(M, r), eta), U, np.full(M, r), eta))
    return out


def test_served_equals_direct_in_a_mix(ctx):
    sts = states(ctx)
    srv = gbs.Server(ctx, arena_bytes=64 << 20, max_active=8)
    tickets = []
    # sampling requests on two states, probability requests on all three, interleaved
    for i in range(6):
        st = sts[i % 2][0]
        tickets.append(("s", i % 2, i, srv.submit_sample(st, seed=123, sample_index=i, N_post=0)))
        pat = gi.random_modes(sts[2][0].M, 1 + i, 70 + i)
        tickets.append(("p", 2, pat, srv.submit_prob(sts[2][0], pat)))
    time.sleep(0.01)
    # late arrivals while the first ones run
    for i in range(6, 10):
        tickets.append(("s", 0, i, srv.submit_sample(sts[0][0], seed=123, sample_index=i, N_post=0)))
    results = [(kind, a, b, srv.poll(t, timeout_s=120)) for kind, a, b, t in tickets]
    stats = srv.stats()
    srv.stop()
    assert stats["completed"] == len(tickets) and stats["p99_s"] >= stats["p50_s"] > 0
    # direct evaluations
    direct = {}
    for which in (0, 1):
        st = sts[which][0]
        pats, _, _, status = gbs.sample(ctx, st, 10, seed=123)
        direct[which] = pats
    for kind, a, b, res in results:
        assert res is not None and res["status"] == 0
        if kind == "s":
            want = np.nonzero(direct[a][b])[0].tolist()
            assert res["clicks"] == want, (a, b)
        else:
            d = gbs.torontonian(ctx, sts[a][0], b, "auto", "auto")
            assert res["prob"].p == d.p and res["prob"].tor == d.tor


@pytest.mark.parametrize("width", [1, 4, 16])
def test_postselected_sampling_served_matches_oracle(ctx, width):
    # attempts run `width` at a time; the result is still the lowest accepted attempt
    M = 8
    U = gi.haar_unitary(M, 33)
    r = gi.uniform_range(33, "squeezing", M, 0.4, 0.9)
    st = gbs.build_state(ctx, U, r, 0.7)
    Sig = oracle.sigma(oracle.covariance(U, r, 0.7))
    srv = gbs.Server(ctx, arena_bytes=64 << 20, max_active=4, attempt_width=width)
    ts = [srv.submit_sample(st, seed=9, sample_index=i, N_post=3, max_attempts=40) for i in range(6)]
    ts.append(srv.submit_sample(st, seed=9, sample_index=6, N_post=7, max_attempts=3))  # exhausts its attempts
    res = [srv.poll(t, timeout_s=120) for t in ts]
    srv.stop()
    for i, rr in enumerate(res):
        ref = oracle.sample_chain(Sig, 9, sample=i, N_post=3 if i < 6 else 7, max_attempts=40 if i < 6 else 3)
        if ref["pattern"] is None:
            assert rr["status"] == _lib.EREJECT and rr["attempts"] == (40 if i < 6 else 3)
        else:
            assert rr["status"] == 0 and rr["clicks"] == np.nonzero(ref["pattern"])[0].tolist()
            assert rr["attempts"] == ref["attempts"]


def test_admission_and_failures_on_the_host(ctx):
    U = gi.haar_unitary(16, 5)
    st = gbs.build_state(ctx, U, np.full(16, 0.8), 1.0)
    # arena for exactly one 16-mode trajectory: the second request waits for the first
    one = 4 * 16 * 16 * 8 + 64 * 4 + 8 * 8 + (4 * 16 + 256) * 8
    srv = gbs.Server(ctx, arena_bytes=one + 512, max_active=8)
    t1 = srv.submit_sample(st, seed=1, sample_index=0)
    t2 = srv.submit_sample(st, seed=1, sample_index=1)
    r1 = srv.poll(t1, timeout_s=60)
    r2 = srv.poll(t2, timeout_s=60)
    assert r1["status"] == 0 and r2["status"] == 0
    assert r2["queue_s"] > 0
    # unknown and consumed tickets
    with pytest.raises(gbs.GbsError) as e:
        srv.poll(999999, timeout_s=0)
    assert e.value.status == _lib.ENOTFOUND
    with pytest.raises(gbs.GbsError):
        srv.poll(t1, timeout_s=0)
    # bad descriptors are refused at submit
    with pytest.raises(gbs.GbsError) as e:
        srv.submit_prob(st, [0, 0])
    assert e.value.status == _lib.EINVAL
    with pytest.raises(gbs.GbsError) as e:
        srv.submit_sample(st, seed=1, N_post=40)
    assert e.value.status == _lib.EINVAL
    # a request larger than the whole arena can never be admitted
    big = gbs.build_state(ctx, gi.haar_unitary(64, 6), np.full(64, 0.5), 1.0)
    with pytest.raises(gbs.GbsError) as e:
        srv.submit_sample(big, seed=1)
    assert e.value.status == _lib.ENOMEM
    # a bounded poll returns PENDING without blocking the caller
    t3 = srv.submit_sample(st, seed=2, sample_index=0)
    first = srv.poll(t3, timeout_s=0)
    final = first or srv.poll(t3, timeout_s=60)
    assert final["status"] == 0
    stats = srv.stats()
    assert stats["refused"] >= 3 and stats["last_error"] == 0
    srv.stop()
