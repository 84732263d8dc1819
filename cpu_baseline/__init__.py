"""Same-precision CPU baseline of the subset enumeration (bench comparator only).

A plain FP64 decision tree (fp64_tree.cpp) on the host cores with OpenMP over
subtrees.  It shares no code with the CUDA library (paper_1810_00900_gb300) or
with the oracle (oracle/); bench.py times it single-core and on all cores beside
the GPU kernels, on the same input matrix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fp64_tree.cpp")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcputree.so")
_lib = None


def build() -> str:
    os.makedirs(OUT, exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["g++", "-O3", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC], check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.cpu_tree_fp64.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.cpu_tree_fp64.restype = ctypes.c_int
        L.cpu_tree_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().cpu_tree_max_threads())


def torontonian_fp64(G: np.ndarray, threads: int = 0, split: int = 10):
    """(Tor, sum of |terms|, seconds) of a 2n x 2n real symmetric block in plain FP64.

    threads <= 0 uses every host core; `split` modes are decided by an outer loop
    over 2^split prefixes that the threads share."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    n = G.shape[0] // 2
    tor, asum, sec = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib().cpu_tree_fp64(n, G.ctypes.data_as(dp), int(threads), int(min(split, n)), ctypes.byref(tor),
                             ctypes.byref(asum), ctypes.byref(sec))
    if st == 1:
        raise np.linalg.LinAlgError("a pivot block is not positive definite")
    if st != 0:
        raise ValueError("bad arguments")
    return tor.value, asum.value, sec.value
