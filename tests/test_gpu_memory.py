"""Device memory of a context: the HBM budget is enforced (GBS_ENOMEM, context still usable),
freed blocks are reused instead of returned to CUDA, and cached blocks give way when a
new allocation needs the room."""
import numpy as np
import pytest

import gbs_inputs as gi
import paper_1810_00900_gb300 as gbs
from paper_1810_00900_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_budget_cache_and_recovery():
    from paper_1810_00900_gb300 import build
    build.build()
    budget = 96 << 20
    ctx = gbs.Context(0, hbm_budget_bytes=budget)
    M = 400
    U = gi.haar_unitary(M, 3)
    r = np.full(M, 0.1)  # about 4 clicks per sample
    st = gbs.build_state(ctx, U, r, 0.9)
    pats, _, _, status = gbs.sample(ctx, st, 1, seed=1)
    assert status == 0 and ctx.bytes_in_use <= budget
    # 20 trajectories need 20 x 32 M^2 bytes = 102 MB: refused, and nothing is left behind
    with pytest.raises(gbs.GbsError) as e:
        gbs.sample(ctx, st, 20, seed=1)
    assert e.value.status == _lib.ENOMEM
    assert ctx.bytes_in_use <= budget
    pats2, _, _, status = gbs.sample(ctx, st, 1, seed=1)
    assert status == 0 and np.array_equal(pats, pats2)
    # repeated state builds reuse the freed blocks: the footprint does not grow
    st.free()
    used = []
    for i in range(8):
        s2 = gbs.build_state(ctx, U, r, 0.9)
        p = gbs.torontonian(ctx, s2, [1, 5, 9], "fp64", "real")
        assert p.p > 0
        s2.free()
        used.append(ctx.bytes_in_use)
    assert max(used[2:]) == min(used[2:]) and max(used) <= budget
    # a large request that only fits once the cache is released still succeeds
    st = gbs.build_state(ctx, U, r, 0.9)
    pats3, _, _, status = gbs.sample(ctx, st, 12, seed=1)
    assert status == 0 and np.array_equal(pats3[0], pats[0])
    st.free()
    ctx.close()
