"""Write the stored expected values of the full-size parity tests.

Calls only the oracle (oracle/) and the seeded input generators (gbs_inputs/).
Run from the repository root:  python tests/golden/make_golden.py [n24] [config4]
Outputs:
  tests/golden/tor_n24_m200.txt -- Tor(O_S) of the single-large-Torontonian
    workload (200 modes, r = 0.8, Haar seed 1, 24 click modes) by the oracle's
    ~212-bit decision-tree enumeration (pinned to the brute-force definition at
    N <= 16 by tests/test_oracle_pins.py), plus p = Tor / sqrt(det Sigma);
  tests/golden/batched_m400.txt -- p of the first 400-mode requests with 17, 20
    and 22 clicks of the 4096-request uneven workload (gbs_inputs.batched_requests),
    the same enumeration.
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gbs_inputs as gi  # noqa: E402
import oracle  # noqa: E402


def n24():
    st, modes = gi.single_large_torontonian_workload(24)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    H = oracle.sigma_inv_block(Sig, modes)
    t0 = time.time()
    tor, asum = oracle.torontonian(H, "tree")
    dt = time.time() - t0
    ld = oracle.logdet_sigma(Sig)
    p = float(tor) * math.exp(-0.5 * ld)
    with open(os.path.join(HERE, "tor_n24_m200.txt"), "w") as f:
        f.write("# Torontonian of the N=24 pattern of the 200-mode r=0.8 Haar (seed 1) pure state.\n")
        f.write("# Written by tests/golden/make_golden.py (oracle decision tree, ~212-bit), %.0f s.\n" % dt)
        f.write("# modes: %s\n" % " ".join(str(int(m)) for m in modes))
        f.write("tor_components %r %r %r %r\n" % tor.c)
        f.write("abs_sum %r\n" % asum)
        f.write("logdet_sigma %r\n" % ld)
        f.write("p %r\n" % p)
        f.write("kappa %r\n" % (asum / abs(float(tor))))


# (index in the 4096-request workload, M, N) of the requests batched_m400.txt holds
def config4_picks(Ns=(17, 20, 22), M=400):
    picks = []
    reqs = gi.batched_requests(4096)
    for N in Ns:
        i = next(j for j, q in enumerate(reqs) if q.M == M and q.N == N)
        picks.append(i)
    return picks


def config4():
    reqs = gi.batched_requests(4096)
    with open(os.path.join(HERE, "batched_m400.txt"), "w") as f:
        f.write("# 400-mode requests of the 4096-request uneven workload (gbs_inputs.batched_requests(4096)):\n")
        f.write("# index N eta r p tor_components(4) abs_sum logdet_sigma; written by tests/golden/make_golden.py\n")
        f.write("# (oracle decision tree, ~212-bit)\n")
        for i in config4_picks():
            q = reqs[i]
            U = gi.haar_unitary(q.M, q.seed)
            r = np.full(q.M, q.r)
            Sig = oracle.sigma(oracle.covariance(U, r, q.eta))
            H = oracle.sigma_inv_block(Sig, q.modes)
            t0 = time.time()
            tor, asum = oracle.torontonian(H, "tree")
            ld = oracle.logdet_sigma(Sig)
            p = float(tor) * math.exp(-0.5 * ld)
            f.write("%d %d %r %r %r %r %r %r %r %r %r\n" % ((i, q.N, q.eta, q.r, p) + tor.c + (asum, ld)))
            f.flush()
            print("request %d (N=%d) %.0f s" % (i, q.N, time.time() - t0))


if __name__ == "__main__":
    which = sys.argv[1:] or ["n24", "config4"]
    if "n24" in which:
        n24()
    if "config4" in which:
        config4()
