"""CPU ORACLE -- test infrastructure only.

A plain, slow, independent CPU implementation of what the GPU path computes,
used to check it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product package never does, and nothing here imports the product.

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from .gbs_oracle import *  # noqa: F401,F403
from ._native import build, lib_path  # noqa: F401
