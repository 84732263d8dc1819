"""ctypes binding of libgbs (include/gbs.h): argument marshalling only.

Every computation behind these functions runs in the library's CUDA kernels.
There is no CPU fallback: if the shared library is missing, loading fails
loudly (build it with ``paper_1810_00900_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes
import os
import re
import weakref
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbs.so")
HEADER = os.path.join(HERE, "..", "include", "gbs.h")

OK, EINVAL, ENOMEM, ENOTPD, EPRECISION, EREJECT, ETIMEDOUT, ECUDA, PENDING, ENOTFOUND = range(10)
PREC = {"auto": 0, "fp64": 1, "dd": 2, "td": 3, "fp32": 4, "fx": 5, "fxw": 6, "fp64p": 7, "fxn": 8}
PREC_NAME = {v: k for k, v in PREC.items()}
BASIS = {"auto": 0, "real": 1, "complex": 2}
BASIS_NAME = {v: k for k, v in BASIS.items()}


class GbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("gbs status %d: %s" % (status, msg))
        self.status = status


class gbs_prob(ctypes.Structure):
    _fields_ = [
        ("p_hi", ctypes.c_double), ("p_lo", ctypes.c_double), ("tor", ctypes.c_double * 3),
        ("abs_sum", ctypes.c_double), ("kappa", ctypes.c_double), ("err_bound", ctypes.c_double),
        ("logdet_sigma", ctypes.c_double), ("prec_used", ctypes.c_int), ("basis_used", ctypes.c_int),
        ("status", ctypes.c_int),
    ]


class gbs_sample_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("escalations", ctypes.c_longlong),
                ("near_ties", ctypes.c_longlong), ("rejections", ctypes.c_longlong), ("seconds", ctypes.c_double),
                ("trees", ctypes.c_longlong * 6), ("tree_seconds", ctypes.c_double * 6),
                ("cond_seconds", ctypes.c_double), ("uncertified", ctypes.c_longlong)]


class gbs_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("state", ctypes.c_void_p), ("N", ctypes.c_int),
                ("modes", ctypes.POINTER(ctypes.c_int)), ("seed", ctypes.c_uint64), ("sample_index", ctypes.c_int),
                ("max_attempts", ctypes.c_int), ("prec", ctypes.c_int), ("basis", ctypes.c_int),
                ("rel_tol", ctypes.c_double)]


class gbs_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("kind", ctypes.c_int), ("prob", gbs_prob), ("n_clicks", ctypes.c_int),
                ("clicks", ctypes.c_int * 64), ("attempts", ctypes.c_int), ("latency_s", ctypes.c_double),
                ("queue_s", ctypes.c_double)]


class gbs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("refused", ctypes.c_longlong),
                ("active", ctypes.c_longlong), ("queued", ctypes.c_longlong), ("p50_s", ctypes.c_double),
                ("p99_s", ctypes.c_double), ("mean_s", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("arena_bytes", ctypes.c_size_t), ("arena_in_use", ctypes.c_size_t),
                ("last_error", ctypes.c_int)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


def header_functions() -> list[str]:
    """Names of the functions declared in include/gbs.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(gbs_\w+)\s*\(", txt, flags=re.M)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgbs.so is not built (%s); call paper_1810_00900_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "gbs_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]),
        "gbs_ctx_destroy": (None, [_vp]),
        "gbs_ctx_set_stream": (ctypes.c_int, [_vp, _vp]),
        "gbs_ctx_last_error": (ctypes.c_char_p, [_vp]),
        "gbs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "gbs_ctx_bytes_in_use": (ctypes.c_size_t, [_vp]),
        "gbs_ctx_launch_count": (ctypes.c_longlong, [_vp]),
        "gbs_ctx_enable_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gbs_ctx_kernel_time": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
        "gbs_ctx_host_gaps": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
        "gbs_draw_click_positions": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _ip]),
        "gbs_sample_forced_random": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_uint8), _dp,
                                                    ctypes.POINTER(gbs_sample_stats)]),
        "gbs_measure_fp64_peak": (ctypes.c_int, [_vp, _dp]),
        "gbs_measure_fx_peak": (ctypes.c_int, [_vp, _dp]),
        "gbs_build_state": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, ctypes.POINTER(_vp)]),
        "gbs_state_from_V": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(_vp)]),
        "gbs_state_free": (None, [_vp]),
        "gbs_state_info": (ctypes.c_int, [_vp, _ip, _dp]),
        "gbs_sigma_inv_block": (ctypes.c_int, [_vp, _vp, _ip, ctypes.c_int, ctypes.c_int, _dp]),
        "gbs_torontonian": (ctypes.c_int, [_vp, _vp, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.POINTER(gbs_prob)]),
        "gbs_torontonian_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), _ip, _ip, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_double, ctypes.POINTER(gbs_prob)]),
        "gbs_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_char_p, ctypes.c_size_t]),
        "gbs_get_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip, _ip,
                                          ctypes.POINTER(ctypes.c_longlong), _ip, _ip]),
        "gbs_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int]),
        "gbs_sample": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _ip,
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_uint8), _dp,
                                      ctypes.POINTER(gbs_sample_stats)]),
        "gbs_server_start": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
        "gbs_server_stop": (ctypes.c_int, [_vp]),
        "gbs_submit": (ctypes.c_int, [_vp, ctypes.POINTER(gbs_request), ctypes.POINTER(ctypes.c_uint64)]),
        "gbs_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(gbs_result), ctypes.c_int64]),
        "gbs_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(gbs_server_stats)]),
        "gbs_subset_sum": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]),
        "gbs_subset_sum_static": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


class Context:
    """A libgbs context on one CUDA device (owns a stream and a workspace)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.L = load()
        h = _vp()
        st = self.L.gbs_ctx_create(ctypes.byref(h), device, hbm_budget_bytes)
        if st:
            raise GbsError(st, "gbs_ctx_create failed (device %d)" % device)
        self.h = h
        # states must be freed before their context; close() frees the live ones
        self._states = weakref.WeakSet()

    def check(self, st: int):
        if st:
            raise GbsError(st, self.L.gbs_ctx_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            for st in list(self._states):
                st.free()
            self.L.gbs_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream_handle: int):
        self.check(self.L.gbs_ctx_set_stream(self.h, _vp(stream_handle)))

    @property
    def bytes_in_use(self) -> int:
        return int(self.L.gbs_ctx_bytes_in_use(self.h))

    @property
    def launch_count(self) -> int:
        return int(self.L.gbs_ctx_launch_count(self.h))

    def enable_timing(self, on: bool = True):
        self.check(self.L.gbs_ctx_enable_timing(self.h, 1 if on else 0))

    def measure_fp64_peak(self) -> float:
        """Measured FP64 rate of the device in GFLOP/s."""
        g = ctypes.c_double()
        self.check(self.L.gbs_measure_fp64_peak(self.h, ctypes.byref(g)))
        return g.value

    def measure_fx_peak(self) -> float:
        """Measured rate of 192-bit fixed-point products (the FX entry type) in products/s."""
        g = ctypes.c_double()
        self.check(self.L.gbs_measure_fx_peak(self.h, ctypes.byref(g)))
        return g.value

    def autotune(self, prec: str = "fp64", basis: str = "real", n: int = 22, n_trees: int = 1):
        """Time candidate launch shapes on a batch of n_trees trees of n, n-1, ... modes and keep the
        fastest; returns the timings."""
        import json
        buf = ctypes.create_string_buffer(1 << 18)
        self.check(self.L.gbs_autotune(self.h, PREC[prec], BASIS[basis], int(n), int(n_trees), buf, len(buf)))
        return json.loads(buf.value.decode() or "[]")

    def tuning(self, prec: str = "fp64", basis: str = "real") -> dict:
        a, b, c, e, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        d = ctypes.c_longlong()
        self.check(self.L.gbs_get_tuning(self.h, PREC[prec], BASIS[basis], ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(c), ctypes.byref(d), ctypes.byref(e), ctypes.byref(f)))
        return {"sub_e": a.value, "d_top": b.value, "grid_per_sm": c.value, "level_threads": d.value,
                "q_drop": e.value, "mid_e": f.value}

    def set_tuning(self, prec: str = "fp64", basis: str = "real", sub_e: int = 5, d_top: int = 10,
                   grid_per_sm: int = 0, level_threads: int = 1 << 18, q_drop: int = 0, mid_e: int = 0):
        self.check(self.L.gbs_set_tuning(self.h, PREC[prec], BASIS[basis], sub_e, d_top, grid_per_sm,
                                         level_threads, q_drop, mid_e))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        self.check(self.L.gbs_ctx_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def host_gaps(self):
        """(seconds, waits) of host gaps since the last call (gbs_ctx_host_gaps)."""
        s = ctypes.c_double()
        n = ctypes.c_longlong()
        self.check(self.L.gbs_ctx_host_gaps(self.h, ctypes.byref(s), ctypes.byref(n)))
        return s.value, n.value


class State:
    def __init__(self, ctx: Context, h, M: int):
        self.ctx, self.h, self.M = ctx, h, M
        ctx._states.add(self)

    def free(self):
        # a state of a closed context was already freed by Context.close()
        if self.h and getattr(self.ctx, "h", None):
            self.ctx.L.gbs_state_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def logdet_sigma(self) -> float:
        m = ctypes.c_int()
        ld = ctypes.c_double()
        self.ctx.check(self.ctx.L.gbs_state_info(self.h, ctypes.byref(m), ctypes.byref(ld)))
        return ld.value


def build_state(ctx: Context, U, r, eta: float = 1.0, want_V: bool = False):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    r = np.ascontiguousarray(r, dtype=np.float64)
    M = r.shape[0]
    if U.shape != (M, M):
        raise ValueError("U must be M x M")
    V = np.empty((2 * M, 2 * M), dtype=np.complex128) if want_V else None
    h = _vp()
    ctx.check(ctx.L.gbs_build_state(ctx.h, M, _p(U.view(np.float64)), _p(r), float(eta),
                                    _p(V.view(np.float64)) if want_V else None, ctypes.byref(h)))
    st = State(ctx, h, M)
    return (st, V) if want_V else st


def state_from_V(ctx: Context, V) -> State:
    V = np.ascontiguousarray(V, dtype=np.complex128)
    M = V.shape[0] // 2
    h = _vp()
    ctx.check(ctx.L.gbs_state_from_V(ctx.h, M, _p(V.view(np.float64)), ctypes.byref(h)))
    return State(ctx, h, M)


def sigma_inv_block(ctx: Context, st: State, modes, basis: str = "complex") -> np.ndarray:
    m = np.ascontiguousarray(modes, dtype=np.int32)
    N = m.size
    real = basis == "real"
    out = np.zeros((2 * N, 2 * N), dtype=np.float64 if real else np.complex128)
    ctx.check(ctx.L.gbs_sigma_inv_block(ctx.h, st.h, _i(m) if N else None, N, BASIS[basis],
                                        _p(out.view(np.float64)) if N else _p(np.zeros(1))))
    return out


@dataclass
class Prob:
    p: float
    p_lo: float
    tor: tuple
    abs_sum: float
    kappa: float
    err_bound: float
    logdet_sigma: float
    prec: str
    basis: str

    @property
    def tor_value(self) -> float:
        return self.tor[0] + (self.tor[1] + self.tor[2])


def torontonian(ctx: Context, st: State, modes, prec: str = "auto", basis: str = "auto",
                rel_tol: float = 0.0) -> Prob:
    m = np.ascontiguousarray(modes, dtype=np.int32)
    out = gbs_prob()
    ctx.check(ctx.L.gbs_torontonian(ctx.h, st.h, _i(m) if m.size else None, int(m.size), PREC[prec], BASIS[basis],
                                    float(rel_tol), ctypes.byref(out)))
    return Prob(out.p_hi, out.p_lo, tuple(out.tor), out.abs_sum, out.kappa, out.err_bound, out.logdet_sigma,
                PREC_NAME[out.prec_used], BASIS_NAME[out.basis_used])


def _prob(out: gbs_prob) -> "Prob":
    return Prob(out.p_hi, out.p_lo, tuple(out.tor), out.abs_sum, out.kappa, out.err_bound, out.logdet_sigma,
                PREC_NAME[out.prec_used], BASIS_NAME[out.basis_used])


def torontonian_batch(ctx: Context, states, patterns, prec: str = "auto", basis: str = "auto",
                      rel_tol: float = 0.0, check: bool = True, return_status: bool = False):
    """Click probabilities of many (state, pattern) requests in one batch (with return_status:
    also the call's gbs_status, e.g. GBS_EPRECISION when some request stayed above rel_tol)."""
    n = len(patterns)
    if len(states) != n:
        raise ValueError("one state per pattern")
    hs = (_vp * max(n, 1))(*[s.h for s in states])
    Ns = np.array([len(p) for p in patterns], dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.int32) for p in patterns])
                                if n and Ns.sum() else np.zeros(1, dtype=np.int32), dtype=np.int32)
    outs = (gbs_prob * max(n, 1))()
    st = ctx.L.gbs_torontonian_batch(ctx.h, n, hs, _i(flat), _i(Ns) if n else None, PREC[prec], BASIS[basis],
                                     float(rel_tol), outs)
    if check:
        ctx.check(st)
    res = [_prob(outs[i]) for i in range(n)]
    return (res, st) if return_status else res


def sample(ctx: Context, st: State, n_samples: int, seed: int, N_post: int = 0, max_attempts: int = 1,
           forced_clicks=None, prec: str = "auto", want_p0: bool = False, check: bool = True):
    """Chain-rule samples (gbs_sample): returns (patterns uint8 [n, M], p0 [n, M] or None, stats dict, status)."""
    M = st.M
    pats = np.zeros((n_samples, M), dtype=np.uint8)
    p0 = np.zeros((n_samples, M)) if want_p0 else None
    fc = None
    if forced_clicks is not None:
        fc = np.ascontiguousarray(forced_clicks, dtype=np.int32).reshape(n_samples, N_post)
    stats = gbs_sample_stats()
    status = ctx.L.gbs_sample(ctx.h, st.h, n_samples, ctypes.c_uint64(seed & ((1 << 64) - 1)), N_post, max_attempts,
                              _i(fc) if fc is not None else None, PREC[prec],
                              pats.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _p(p0) if want_p0 else None,
                              ctypes.byref(stats))
    if check and status not in (0, EREJECT):
        ctx.check(status)
    sd = {f: getattr(stats, f) for f, _ in gbs_sample_stats._fields_}
    sd["trees"] = list(sd["trees"])
    sd["tree_seconds"] = list(sd["tree_seconds"])
    return pats, p0, sd, status


def draw_click_positions(M: int, n_clicks: int, seed: int, n_samples: int) -> np.ndarray:
    """The seed-drawn forced click positions (gbs_draw_click_positions; host only)."""
    out = np.zeros((max(n_samples, 0), n_clicks), dtype=np.int32)
    st = load().gbs_draw_click_positions(int(M), int(n_clicks), ctypes.c_uint64(seed & ((1 << 64) - 1)),
                                         int(n_samples), _i(out) if out.size else None)
    if st != OK:
        raise GbsError(st, "gbs_draw_click_positions")
    return out


def sample_forced_random(ctx: Context, st: State, n_samples: int, seed: int, n_clicks: int, prec: str = "auto",
                         want_p0: bool = False):
    """Forced-outcome samples with seed-drawn click positions (gbs_sample_forced_random):
    (patterns, p0 or None, stats dict)."""
    M = st.M
    pats = np.zeros((n_samples, M), dtype=np.uint8)
    p0 = np.zeros((n_samples, M)) if want_p0 else None
    stats = gbs_sample_stats()
    ctx.check(ctx.L.gbs_sample_forced_random(ctx.h, st.h, n_samples, ctypes.c_uint64(seed & ((1 << 64) - 1)),
                                             n_clicks, PREC[prec], pats.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                             _p(p0) if want_p0 else None, ctypes.byref(stats)))
    sd = {f: getattr(stats, f) for f, _ in gbs_sample_stats._fields_}
    sd["trees"] = list(sd["trees"])
    sd["tree_seconds"] = list(sd["tree_seconds"])
    return pats, p0, sd


class Server:
    """The context's request loop (gbs_server_start / gbs_submit / gbs_poll)."""

    def __init__(self, ctx: Context, arena_bytes: int = 4 << 30, max_active: int = 64, attempt_width: int = 1):
        self.ctx = ctx
        ctx.check(ctx.L.gbs_server_start(ctx.h, int(arena_bytes), int(max_active), int(attempt_width)))
        self._keep = {}

    def submit_prob(self, st: State, modes, prec: str = "auto", basis: str = "auto", rel_tol: float = 0.0) -> int:
        m = np.ascontiguousarray(modes, dtype=np.int32)
        r = gbs_request(kind=0, state=st.h, N=int(m.size), modes=_i(m) if m.size else None, seed=0,
                        sample_index=0, max_attempts=1, prec=PREC[prec], basis=BASIS[basis], rel_tol=rel_tol)
        t = ctypes.c_uint64()
        self.ctx.check(self.ctx.L.gbs_submit(self.ctx.h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def submit_sample(self, st: State, seed: int, sample_index: int = 0, N_post: int = 0, max_attempts: int = 1,
                      prec: str = "auto") -> int:
        r = gbs_request(kind=1, state=st.h, N=int(N_post), modes=None, seed=seed & ((1 << 64) - 1),
                        sample_index=int(sample_index), max_attempts=int(max_attempts), prec=PREC[prec], basis=1,
                        rel_tol=0.0)
        t = ctypes.c_uint64()
        self.ctx.check(self.ctx.L.gbs_submit(self.ctx.h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_s: float = -1.0):
        """None while pending; else a dict with the result."""
        out = gbs_result()
        us = -1 if timeout_s < 0 else int(timeout_s * 1e6)
        st = self.ctx.L.gbs_poll(self.ctx.h, ctypes.c_uint64(ticket), ctypes.byref(out), ctypes.c_int64(us))
        if st == PENDING:
            return None
        if st != OK:
            raise GbsError(st, "gbs_poll")
        res = {"status": out.status, "kind": out.kind, "latency_s": out.latency_s, "queue_s": out.queue_s,
               "attempts": out.attempts}
        if out.kind == 0:
            res["prob"] = _prob(out.prob)
        else:
            res["clicks"] = sorted(out.clicks[i] for i in range(out.n_clicks))
        return res

    def stats(self) -> dict:
        s = gbs_server_stats()
        self.ctx.check(self.ctx.L.gbs_server_stats_get(self.ctx.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in gbs_server_stats._fields_}

    def stop(self):
        if self.ctx.h:
            self.ctx.L.gbs_server_stop(self.ctx.h)


def subset_sum(ctx: Context, G, basis: str = "complex", prec: str = "fp64"):
    """Signed subset sum of an explicit matrix (see gbs_subset_sum): (inc, exc, tor, abs_sum)."""
    real = basis == "real"
    G = np.ascontiguousarray(G, dtype=np.float64 if real else np.complex128)
    n = G.shape[0] // 2
    inc, exc, tor = np.zeros(3), np.zeros(3), np.zeros(3)
    a = ctypes.c_double()
    ctx.check(ctx.L.gbs_subset_sum(ctx.h, n, _p(G.view(np.float64)), BASIS[basis], PREC[prec], _p(inc), _p(exc),
                                   _p(tor), ctypes.byref(a)))
    return inc, exc, tor, a.value


def subset_sum_static(G_dev_ptr: int, n: int, out_dev_ptr: int, stream_ptr: int = 0) -> int:
    """gbs_subset_sum_static on caller-owned device buffers (raw device addresses).
    Queues the work on `stream_ptr` and returns the status code without waiting."""
    L = load()
    return int(L.gbs_subset_sum_static(_vp(G_dev_ptr), int(n), _vp(out_dev_ptr), _vp(stream_ptr)))
