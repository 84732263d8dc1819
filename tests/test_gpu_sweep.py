"""Randomized sweep: seeded states of varied size, squeezing and loss, and click patterns of
1..12 modes, each evaluated in every precision (FP64, FP64 with the last two levels grouped,
double-double, the three fixed-point widths, triple-double) against the oracle's quad-double
Torontonian:
  * on the same input matrix (gbs_subset_sum on the oracle's real-basis block), within the
    arithmetic bound 8 n u sum|t| of each precision (sum of group magnitudes for the grouped
    FP64), u as in the error model;
  * end to end (the state's closed-form click block on the GPU), within the bound the library
    reports plus 1e-12 relative for the FP64 rounding of the two click blocks, which differ in
    the last bits (the Torontonian is well conditioned in its matrix);
  * AUTO end to end against the 1e-10 target."""
import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import frac3, oracle_tor, real_basis_block

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp64p", "dd", "fxn", "fx", "fxw", "td"]
U_OF = {"fp64": 2.0 ** -53, "fp64p": 2.0 ** -53, "dd": 2.0 ** -102, "fxn": 2.0 ** -108, "fx": 2.0 ** -140,
        "fxw": 2.0 ** -158, "td": 2.0 ** -152}


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_00900_gb300 import build
    build.build()
    c = gbs.Context(0)
    yield c
    c.close()


def case(i):
    M = (20, 60, 150)[i % 3]
    N = 1 + int(gi.uniforms(100 + i, 0, 1)[0] * 12)
    r = gi.uniform_range(100 + i, "squeezing", M, 0.2, 1.3)
    eta = float(0.3 + 0.7 * gi.uniforms(100 + i, 1, 1)[0])
    U = gi.haar_unitary(M, 100 + i)
    modes = gi.random_modes(M, N, 100 + i)
    return U, r, eta, modes


@pytest.mark.parametrize("i", range(24))
def test_every_precision_within_its_bound(ctx, i):
    U, r, eta, modes = case(i)
    st = gbs.build_state(ctx, U, r, eta)
    Sig = oracle.sigma(oracle.covariance(U, r, eta))
    ref, ref_abs = oracle_tor(oracle.sigma_inv_block(Sig, modes))
    want = float(ref.to_fraction())
    G = real_basis_block(oracle.sigma_inv_block(Sig, modes))
    gref, _ = oracle_tor(G)
    n = len(modes)
    for prec in PRECS:
        _, _, tor, a = gbs.subset_sum(ctx, G, "real", prec)
        err = abs(float(frac3(tor) - gref.to_fraction()))
        assert err <= 8 * n * U_OF[prec] * a, (i, prec, "same input", err, 8 * n * U_OF[prec] * a)
        pr = gbs.torontonian(ctx, st, modes, prec, "real")
        sc = np.exp(-0.5 * pr.logdet_sigma)
        assert abs(pr.tor_value - want) <= pr.err_bound / sc + 1e-12 * abs(want), (i, prec, pr.tor_value, want,
                                                                                   pr.err_bound / sc)
    pa = gbs.torontonian(ctx, st, modes, "auto", "real")
    assert abs(pa.tor_value - want) <= 1e-10 * abs(want), (i, pa.prec, pa.tor_value, want)
    st.free()
