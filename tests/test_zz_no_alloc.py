"""gbs_subset_sum_static, the entry point that allocates nothing, against
gbs_subset_sum and against the oracle.

Callers that cannot let a library call cudaMalloc / cudaFree (cudaFree stalls
the whole device; their memory belongs to another allocator or a fixed pool)
pass their own device buffers to gbs_subset_sum_static, which keeps its
intermediate data in the library's static device array.  Here the caller's
buffers come from PyTorch's allocator.  Calls in a row (of different sizes, up
to the stated maximum of 19 modes and down to the one-level leaf cases) check
that reusing the array, which still holds the previous call's data, changes
nothing; the tolerance is the FP64 one of tests/test_gpu_tree.py.  A matrix
that is not positive definite is reported in the status word.
"""
import numpy as np
import pytest

import gbs_inputs as gi
import oracle
import paper_1810_00900_gb300 as gbs
from helpers import frac3, oracle_tor, real_basis_block
from paper_1810_00900_gb300 import _lib

pytestmark = pytest.mark.gpu


def real_block(N, seed):
    st = gi.uniform_squeezed_state(120, 0.7, seed=seed, eta=0.8)
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    return real_basis_block(oracle.sigma_inv_block(Sig, gi.random_modes(120, N, seed=seed)))


def test_static_entry_point_matches_allocating_entry_point():
    import torch
    from paper_1810_00900_gb300 import build
    build.build()
    ctx = gbs.Context(0)
    stream = torch.cuda.Stream()
    for n, seed in ((17, 1), (11, 5), (19, 2), (3, 4), (1, 6)):
        G = real_block(n, seed)
        inc, exc, tor, asum = gbs.subset_sum(ctx, G, "real", "fp64")
        ref, ref_abs = oracle_tor(G)
        G_dev = torch.from_numpy(G).to("cuda")
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = _lib.subset_sum_static(G_dev.data_ptr(), n, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert st == 0
        o = out.cpu().numpy()
        assert o[7] == 0.0  # status: every pivot positive definite
        tol = 8 * n * 2.0 ** -53 * asum
        assert abs((o[0] + o[1]) - (tor[0] + tor[1])) <= tol
        assert abs((o[2] + o[3]) - (inc[0] + inc[1])) <= tol
        assert abs((o[4] + o[5]) - (exc[0] + exc[1])) <= tol
        assert abs(o[6] - asum) <= 1e-12 * asum
        # and against the oracle (the plain definition up to 14 modes, its tree beyond)
        assert abs(float(frac3((o[0], o[1], 0.0)) - ref.to_fraction())) <= tol
        assert abs(o[6] - ref_abs) <= 1e-12 * ref_abs
    # a matrix that is not positive definite (one diagonal entry negated): the status
    # word says so; the call itself succeeds
    G = real_block(9, 3)
    G[4, 4] = -G[4, 4]
    G_dev = torch.from_numpy(G).to("cuda")
    torch.cuda.synchronize()
    assert _lib.subset_sum_static(G_dev.data_ptr(), 9, out.data_ptr(), stream.cuda_stream) == 0
    stream.synchronize()
    assert out.cpu().numpy()[7] == 3.0
    # beyond the stated maximum: rejected before anything is queued
    assert _lib.subset_sum_static(G_dev.data_ptr(), 20, out.data_ptr(), stream.cuda_stream) == _lib.EINVAL
    ctx.close()
