"""Build and load the oracle's C core (oracle/tor_oracle.c). Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tor_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_handle = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile tor_oracle.c with plain gcc; strict IEEE evaluation (no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib() -> ctypes.CDLL:
    global _handle
    if _handle is None:
        build()
        h = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        for name in ("orc_sum_bruteforce", "orc_sum_tree"):
            f = getattr(h, name)
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int,
                          ctypes.c_int, dp, dp]
        h.orc_qd_op.restype = None
        h.orc_qd_op.argtypes = [ctypes.c_int, dp, dp, dp]
        h.orc_qd_normalize.restype = None
        h.orc_qd_normalize.argtypes = [dp, ctypes.c_int, dp]
        h.orc_det.restype = None
        h.orc_det.argtypes = [ctypes.c_int, dp, dp, dp]
        _handle = h
    return _handle


def nthreads() -> int:
    return max(1, os.cpu_count() or 1)
