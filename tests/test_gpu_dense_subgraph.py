"""The paper's application (Sec. IV): GBS samples of a graph-encoded state favour dense subgraphs.
On an Erdos-Renyi graph with a planted dense part, postselected click patterns must be denser, on
average, than uniformly random vertex sets of the same size, and must overlap the planted part more
(a statistical property of the sampler's output, checked with a wide margin)."""
import numpy as np
import pytest

import gbs_inputs as gi
import paper_1810_00900_gb300 as gbs

pytestmark = pytest.mark.gpu


def density(A, nodes):
    k = len(nodes)
    return A[np.ix_(nodes, nodes)].sum() / 2.0 / (k * (k - 1) / 2.0)


def test_gbs_samples_are_denser_than_uniform_subsets():
    from paper_1810_00900_gb300 import build
    build.build()
    ctx = gbs.Context(0)
    A = gi.planted_graph(60, 7, k=12)
    planted = set(gi.planted_vertices(60, 7, k=12).tolist())
    N = 6
    sp = gi.graph_state(A, 2.0 * N, 1.0)
    st = gbs.build_state(ctx, sp.U, sp.r, sp.eta)
    pats, _, _, status = gbs.sample(ctx, st, 48, seed=3, N_post=N, max_attempts=256, check=False)
    ok = [np.nonzero(p)[0] for p in pats if p[0] != 0xFF]
    assert len(ok) >= 40
    assert all(len(s) == N for s in ok)
    uni = gi.uniform_subsets(60, N, 48, seed=3)
    d_gbs = np.mean([density(A, s) for s in ok])
    d_uni = np.mean([density(A, s) for s in uni])
    assert d_gbs > d_uni + 0.1, (d_gbs, d_uni)
    f_gbs = np.mean([len(planted & set(s.tolist())) / N for s in ok])
    f_uni = np.mean([len(planted & set(s.tolist())) / N for s in uni])
    assert f_gbs > f_uni + 0.2, (f_gbs, f_uni)
    st.free()
    ctx.close()
