"""Full-size sampler parity: the 800-mode forced-click workload the benchmark times (64
trajectories of 20 uniformly placed clicks, run together after the same launch-shape tuning),
with the no-click probability of trajectory 0 checked against the oracle at sampled steps --
the first ones, one in the middle and the last ones, where the trees span all 20 clicks.  The
oracle recomputes each sampled step from scratch (dense conditioning of the 1600 x 1600 Sigma,
then two quad-double subset trees), so it checks the GPU's running rank-2 conditioning over
the ~780 dark steps before them as well."""
import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs

pytestmark = pytest.mark.gpu


def test_m800_n20_forced_trajectories_sampled_steps():
    from paper_1810_00900_gb300 import build
    build.build()
    ctx = gbs.Context(0)
    stp, clicks = gi.chain_sampling_workload(800, 20, 64, seed=2)
    st = gbs.build_state(ctx, stp.U, stp.r, stp.eta)
    for prec in ("fxn", "fx", "fxw"):
        ctx.autotune(prec, "real", 21, n_trees=9)
    forced = np.array(clicks, dtype=np.int32)
    pats, p0, stats, status = gbs.sample(ctx, st, 64, seed=2, N_post=20, forced_clicks=forced, want_p0=True)
    assert status == 0 and stats["uncertified"] == 0
    for t in range(64):
        assert np.array_equal(np.nonzero(pats[t])[0], np.sort(forced[t]))
    assert np.all(np.isfinite(p0)) and np.all((p0 > 0) & (p0 < 1))
    Sig = oracle.sigma(oracle.covariance(stp.U, stp.r, stp.eta))
    steps = [0, 1, 400, 798, 799]
    ref = oracle.sample_chain(Sig, 2, forced_clicks=forced[0], steps_to_check=set(steps))
    for s in steps:
        assert abs(p0[0][s] - ref["p0"][s]) <= 1e-10, (s, p0[0][s], ref["p0"][s])
    st.free()
    ctx.close()
