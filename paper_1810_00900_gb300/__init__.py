"""GB300-native exact threshold-detector Gaussian Boson Sampling.

Click probabilities via Torontonians (the 2^N subset determinants enumerated on
the GPU by a decision tree of shared-prefix Schur complements) and chain-rule
click sampling, behind the C ABI in include/gbs.h.  This package is the thin
Python binding; importing it does not touch the GPU.
"""
from ._lib import (  # noqa: F401
    BASIS, PREC, Context, Server, GbsError, Prob, State, build_state, draw_click_positions, header_functions, load,
    sample, sample_forced_random, sigma_inv_block, state_from_V, subset_sum, torontonian, torontonian_batch,
)
