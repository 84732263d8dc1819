"""The autotuner and the launch shapes it chooses between change speed, not results."""
import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import frac3, oracle_tor, real_basis_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def test_launch_shapes_agree(ctx):
    st = gi.uniform_squeezed_state(150, 0.7, seed=9)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    H = real_basis_block(oracle.sigma_inv_block(Sig, gi.random_modes(150, 17, seed=9)))
    ref, ref_abs = oracle_tor(H)
    seen = []
    for sub_e in (0, 2, 3, 5, 6, 7):  # below 5: one-warp CTAs expanding several roots at once
        for d_top in (0, 4, 10):
            for grid in (0, 2):
                for q_drop, mid_e in ((0, 0), (1, 0), (0, 5), (1, 3)):
                    ctx.set_tuning("dd", "real", sub_e, d_top, grid, 1 << 17, q_drop, mid_e)
                    _, _, tor, a = gbs.subset_sum(ctx, H, "real", "dd")
                    err = abs(float(frac3(tor) - ref.to_fraction()))
                    assert err <= 8 * 17 * 2.0 ** -102 * ref_abs, (sub_e, d_top, grid, q_drop, mid_e, err)
                    seen.append(tor)
    ctx.set_tuning("dd", "real", 5, 10, 0, 1 << 18)
    # the fixed-point sums are exact and their reduction order fixed: every shape gives the same bits
    fx_seen = set()
    for sub_e in (0, 2, 4, 6):
        for d_top in (0, 8):
            for q_drop, mid_e in ((0, 0), (1, 0), (2, 0), (0, 5), (1, 2)):
                ctx.set_tuning("fx", "real", sub_e, d_top, 8, 1 << 17, q_drop, mid_e)
                _, _, tor, _ = gbs.subset_sum(ctx, H, "real", "fx")
                fx_seen.add(tuple(tor))
                assert abs(float(frac3(tor) - ref.to_fraction())) <= 8 * 17 * 2.0 ** -140 * ref_abs
    assert len(fx_seen) == 1
    ctx.set_tuning("fx", "real", 6, 6, 0, 1 << 18)
    # FP64 with several roots per shared-memory CTA: within the FP64 bound of the same input
    for sub_e in (1, 2, 3, 4):
        ctx.set_tuning("fp64", "real", sub_e, 6, 8, 1 << 17, 0, 4)
        _, _, tor, a = gbs.subset_sum(ctx, H, "real", "fp64")
        assert abs(float(frac3(tor) - ref.to_fraction())) <= 8 * 17 * 2.0 ** -53 * ref_abs + 24 * 2.0 ** -53 * a
    ctx.set_tuning("fp64", "real", 5, 8, 8, 1 << 17, 0, 4)


def test_autotune_picks_a_candidate(ctx):
    rep = ctx.autotune("fp64", "real", 14)
    assert len(rep) >= 8 and all(r["ms"] > 0 for r in rep)
    best = min(r["ms"] for r in rep)
    t = ctx.tuning("fp64", "real")
    keys = ("sub_e", "d_top", "grid_per_sm", "level_threads", "q_drop", "mid_e")
    chosen = [r for r in rep if all(r[k] == t[k] for k in keys)]
    # the report rounds to 0.1 us, so several candidates can tie with the one kept
    assert len(chosen) == 1 and chosen[0]["ms"] == best


def test_peak_probes(ctx):
    # the roofline denominators: FP64 at most 2 FMAs per clock per SM, fixed-point products
    # between a tenth of one and four per clock per SM (26 partial products of 32 x 32 bits each)
    import torch
    props = torch.cuda.get_device_properties(0)
    sms, ghz = props.multi_processor_count, 2.2
    g = ctx.measure_fp64_peak()
    assert 0 < g <= 2 * 2 * sms * ghz * 1.01
    p = ctx.measure_fx_peak()
    assert 0.1 * sms * 1.0e9 < p < 4 * sms * ghz * 1e9


def test_small_levels_every_thread_mapping(ctx):
    # Breadth-first levels of small trees, where a level has fewer than 32 nodes: with one row
    # group per node, with a few (tiles of the whole level), and with more than 8 (one group of
    # consecutive nodes per block).  Fixed point gives the same bits for every shape.
    st = gi.uniform_squeezed_state(60, 0.6, seed=21)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    for n in (5, 7, 9):
        H = real_basis_block(oracle.sigma_inv_block(Sig, gi.random_modes(60, n, seed=n)))
        ref, ref_abs = oracle_tor(H)
        seen = set()
        for level_threads in (1, 8, 64, 1 << 17):
            ctx.set_tuning("fx", "real", 0, 0, 0, level_threads, 1, 0)
            _, _, tor, _ = gbs.subset_sum(ctx, H, "real", "fx")
            seen.add(tuple(tor))
            assert abs(float(frac3(tor) - ref.to_fraction())) <= 8 * n * 2.0 ** -140 * ref_abs
            ctx.set_tuning("fp64", "real", 0, 0, 0, level_threads, 1, 0)
            _, _, tor, a = gbs.subset_sum(ctx, H, "real", "fp64")
            assert abs(float(frac3(tor) - ref.to_fraction())) <= 8 * n * 2.0 ** -53 * ref_abs + 24 * 2.0 ** -53 * a
        assert len(seen) == 1, n
    ctx.set_tuning("fx", "real", 6, 6, 0, 1 << 18)
    ctx.set_tuning("fp64", "real", 5, 8, 8, 1 << 17, 0, 4)
