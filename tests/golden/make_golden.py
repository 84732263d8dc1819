"""Write the stored expected values of the full-size parity tests.

Calls only the oracle (oracle/) and the seeded input generators (gbs_inputs/).
Run from the repository root:  python tests/golden/make_golden.py
Output: tests/golden/tor_n24_m200.txt -- Tor(O_S) of the single-large-Torontonian
workload (200 modes, r = 0.8, Haar seed 1, 24 click modes) by the oracle's
~212-bit decision-tree enumeration (pinned to the brute-force definition at
N <= 12 by tests/test_oracle_pins.py), plus p = Tor / sqrt(det Sigma).
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gbs_inputs as gi  # noqa: E402
import oracle  # noqa: E402


def main():
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


if __name__ == "__main__":
    main()
