"""FP64 with the last two tree levels summed cancellation-free (prec "fp64p") against the
oracle's exact Torontonian.  Each group of four subsets that differ only in the last two
modes contributes one value whose factors carry small relative errors, so the error is
bounded by 8 n u times the sum of the group magnitudes the kernel reports (the same
per-term model as the plain tree, applied to groups; a group's magnitude includes its
sensitivity to relative errors of its input entries), and that sum is 1e1..1e3 times
smaller than the plain tree's sum of |terms| on these states."""
from fractions import Fraction

import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import frac3, oracle_tor, real_basis_block

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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
    return oracle.sigma_inv_block(Sig, gi.random_modes(M, N, seed=seed))


def paired_error(ctx, H):
    n = H.shape[0] // 2
    G = real_basis_block(H)
    ref, ref_abs = oracle_tor(G)
    inc, exc, tor, a_p = gbs.subset_sum(ctx, G, "real", "fp64p")
    assert frac3(exc) == 0 and frac3(inc) == frac3(tor)
    err = float(abs(frac3(tor) - ref.to_fraction()))
    assert err <= 8 * n * U * a_p, (n, err, 8 * n * U * a_p)
    return err, a_p, ref_abs, float(ref.to_fraction())


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 10, 12, 14])
def test_parity_pure_haar(ctx, N):
    err, a_p, ref_abs, tor = paired_error(ctx, haar_H(N))
    if N >= 10:
        # the group magnitudes are far below the term magnitudes: the bound shrinks with them
        assert a_p * 30 <= ref_abs, (a_p, ref_abs)
        _, _, tor64, _ = gbs.subset_sum(ctx, real_basis_block(haar_H(N)), "real", "fp64")
        err64 = abs(float(frac3(tor64)) - tor)
        assert err <= err64 or err <= 1e-13 * abs(tor)


@pytest.mark.parametrize("seed,M,r,eta,N", [(31, 120, 0.7, 0.6, 12), (5, 100, 0.5, 0.5, 11), (7, 200, 1.0, 1.0, 12),
                                            (4, 400, 0.9, 0.25, 13)])
def test_parity_lossy_and_squeezed(ctx, seed, M, r, eta, N):
    err, a_p, ref_abs, tor = paired_error(ctx, haar_H(N, seed=seed, M=M, r=r, eta=eta))
    assert a_p * 10 <= ref_abs


def test_identity_closed_form(ctx):
    # independent modes: g_j = sqrt(d_j), each group is (g_a - 1)(g_b - 1) exactly (D = 0,
    # g_c = g_b) and Tor = prod (g_j - 1); a group's magnitude is (g_a-1)(g_b-1) + (g_a-1) g_b
    # + (g_b-1) g_a against the plain (g_a+1)(g_b+1), and the modes above the last two
    # contribute the same factor to both sums
    r = np.concatenate([np.linspace(0.6, 1.0, 12), np.full(4, 0.5)])
    st_p = gi.identity_state(r, 0.8)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 0.8)
    modes = np.arange(12)
    want = oracle.identity_torontonian(r, 0.8, modes)
    pr = gbs.torontonian(ctx, st, modes, "fp64p", "real")
    assert pr.prec == "fp64p"
    sc = np.exp(-0.5 * pr.logdet_sigma)
    assert abs(pr.tor_value - want) <= pr.err_bound / sc
    p64 = gbs.torontonian(ctx, st, modes, "fp64", "real")
    d = 1.0 + 0.8 * (2.0 - 0.8) * np.sinh(r[10:12]) ** 2
    ga, gb = np.sqrt(d)
    ratio = (ga + 1) * (gb + 1) / ((ga - 1) * (gb - 1) + (ga - 1) * gb + (gb - 1) * ga)
    assert abs(p64.abs_sum / pr.abs_sum / ratio - 1.0) < 1e-12
    st.free()


def test_launch_shapes_agree(ctx):
    H = haar_H(13, seed=3)
    G = real_basis_block(H)
    ref, _ = oracle_tor(G)
    saved = ctx.tuning("fp64p", "real")
    vals = []
    try:
        for sub_e, q_drop in [(0, 0), (0, 1), (5, 0), (6, 1), (7, 0)]:
            ctx.set_tuning("fp64p", "real", sub_e=sub_e, d_top=4, grid_per_sm=8, level_threads=1 << 17,
                           q_drop=q_drop, mid_e=2)
            inc, exc, tor, a_p = gbs.subset_sum(ctx, G, "real", "fp64p")
            assert abs(frac3(tor) - ref.to_fraction()) <= Fraction(8 * 13 * U * a_p)
            vals.append(frac3(tor))
    finally:
        ctx.set_tuning("fp64p", "real", **saved)
    # one shape twice: bitwise identical
    inc, exc, tor, a_p = gbs.subset_sum(ctx, G, "real", "fp64p")
    inc2, exc2, tor2, a_p2 = gbs.subset_sum(ctx, G, "real", "fp64p")
    assert frac3(tor) == frac3(tor2) and a_p == a_p2


def test_batch_of_uneven_requests(ctx):
    st_p = gi.uniform_squeezed_state(150, 0.8, seed=21)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    Sig = oracle.sigma(oracle.covariance(st_p.U, st_p.r, 1.0))
    pats = [gi.random_modes(150, n, seed=40 + n) for n in (1, 2, 4, 7, 9, 12)]
    res = gbs.torontonian_batch(ctx, [st] * len(pats), pats, "fp64p", "real")
    for m, pr in zip(pats, res):
        ref, _ = oracle_tor(oracle.sigma_inv_block(Sig, m))
        want = float(ref.to_fraction())
        assert abs(pr.tor_value - want) <= pr.err_bound / np.exp(-0.5 * pr.logdet_sigma), (len(m), pr.tor_value, want)
    st.free()


def test_refusals(ctx):
    H = haar_H(6)
    with pytest.raises(gbs.GbsError):
        gbs.subset_sum(ctx, H, "complex", "fp64p")
    st_p = gi.uniform_squeezed_state(40, 0.5, seed=2)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    with pytest.raises(gbs.GbsError):
        gbs.sample(ctx, st, 1, seed=1, prec="fp64p")
    st.free()


def test_auto_ladder_uses_the_paired_rung(ctx):
    # N = 8 of the 200-mode pure state: FP64's estimate (kappa ~ 7e10) misses 1e-5 by ~20x,
    # the grouped sum's meets it; at the default 1e-10 the miss exceeds 1e3 and AUTO goes on
    # to fixed point directly, the narrow width, since FP64 bounds |p| away from zero
    st_p = gi.uniform_squeezed_state(200, 0.8, seed=1)
    st = gbs.build_state(ctx, st_p.U, st_p.r, 1.0)
    modes = gi.random_modes(200, 8, seed=1)
    Sig = oracle.sigma(oracle.covariance(st_p.U, st_p.r, 1.0))
    ref, _ = oracle_tor(oracle.sigma_inv_block(Sig, modes))
    want = float(ref.to_fraction())
    pr = gbs.torontonian(ctx, st, modes, "auto", "real", rel_tol=1e-5)
    assert pr.prec == "fp64p"
    assert pr.err_bound <= 1e-5 * abs(pr.p)
    assert abs(pr.tor_value - want) <= 1e-5 * abs(want)
    pr2 = gbs.torontonian(ctx, st, modes, "auto", "real")
    assert pr2.prec == "fxn" and pr2.err_bound <= 1e-10 * abs(pr2.p)
    assert abs(pr2.tor_value - want) <= 1e-10 * abs(want)
    st.free()
