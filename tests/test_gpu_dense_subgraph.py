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


def test_threshold_vs_photon_number_resolving_on_small_graphs():
    # The paper's comparison of threshold and photon-number-resolving (PNR) detection for dense
    # subgraphs (Sec. IV), at sizes where every N-vertex subset can be enumerated exactly.
    # Threshold: p(S) of clicks exactly on S, from the GPU's Torontonians, element by element
    # against the oracle.  PNR: the collision-free outcome with one photon on each vertex of S,
    # |haf(B_S)|^2 / sqrt(det Sigma) with B = U tanh(R) U^T (the oracle's hafnian), which is one
    # of the outcomes the click event contains, so p(S) >= p_PNR(S) for every S.  Both
    # distributions over N-vertex sets favour dense subsets well above uniform, and the
    # threshold one does at least as well.
    import itertools
    import math
    import oracle
    from paper_1810_00900_gb300 import build
    build.build()
    ctx = gbs.Context(0)
    for M, k, seed, nbar, N in ((10, 4, 3, 1.0, 4), (12, 5, 5, 2.0, 4)):
        A = gi.planted_graph(M, seed, p=0.25, k=k, q=1.0)
        sp = gi.graph_state(A, nbar, 1.0)
        st = gbs.build_state(ctx, sp.U, sp.r, sp.eta)
        subs = [list(S) for S in itertools.combinations(range(M), N)]
        # (subsets with an isolated vertex have p = 0, which no relative bound certifies: the
        # call's status may say so, the values are still checked below)
        res = gbs.torontonian_batch(ctx, [st] * len(subs), subs, "auto", "real", check=False)
        p_gpu = np.array([r.p + r.p_lo for r in res])
        assert np.all(np.isfinite(p_gpu))
        p_orc = np.array([oracle.click_probability(sp.U, sp.r, 1.0, S)[0] for S in subs])
        scale = p_orc.max()
        assert np.all(np.abs(p_gpu - p_orc) <= 1e-9 * np.abs(p_orc) + 1e-14 * scale)
        B = sp.U @ np.diag(np.tanh(sp.r)) @ sp.U.T
        Sig = oracle.sigma(oracle.covariance(sp.U, sp.r, 1.0))
        pref = math.exp(-0.5 * oracle.logdet_sigma(Sig))
        p_pnr = np.array([abs(oracle.hafnian(B[np.ix_(S, S)])) ** 2 * pref for S in subs])
        assert np.all(p_gpu >= p_pnr - 1e-12 * scale)
        d = np.array([density(A, S) for S in subs])
        e_thr = float((np.clip(p_gpu, 0, None) * d).sum() / np.clip(p_gpu, 0, None).sum())
        e_pnr = float((p_pnr * d).sum() / p_pnr.sum())
        assert e_thr > d.mean() + 0.2 and e_pnr > d.mean() + 0.2, (e_thr, e_pnr, d.mean())
        assert e_thr >= e_pnr - 0.02, (e_thr, e_pnr)
        st.free()
    ctx.close()
