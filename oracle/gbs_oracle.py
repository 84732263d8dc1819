"""CPU ORACLE -- test infrastructure only (see oracle/__init__.py).

Threshold-detector Gaussian Boson Sampling quantities, written from the paper
(Gupt, Arrazola, Quesada, Bromley, "Classical benchmarking of Gaussian Boson
Sampling on the Titan supercomputer", arXiv:1810.00900) and plain definitions.

Conventions
-----------
* Complex basis (a_1..a_M, a_1^+..a_M^+), covariance V with vacuum V = I/2 and
  Sigma = V + I/2 (vacuum Sigma = I).  The paper's real basis
  (x_1, p_1, ..., x_M, p_M) with hbar = 2 (Sec. II, Eq. 1, vacuum V = I) is
  related per mode by a = (x + i p)/2.
* A mode subset A is addressed through its rows {j, j+M : j in A}, taken
  mode-interleaved (a_j, a_j^+) in the order of A.
* Vacuum probability of modes A: 1/sqrt(det Sigma_A) -- the paper's Eq. (5),
  q = 2/sqrt(det(V_B + 1)), for zero means, rewritten with Sigma.
* Click pattern S (clicks on S, vacuum on the other modes):
      p(S) = sum_{W subset S} (-1)^|W| / sqrt(det Sigma_{W u S^c})
  (each click detector is 1 - |0><0|, expanded), which the identity
  det Sigma_B = det Sigma * det((Sigma^-1)_{B^c}) turns into
      p(S) = Tor(O_S) / sqrt(det Sigma),
      Tor(O_S) = sum_{Z subset S} (-1)^(|S|-|Z|) / sqrt(det((Sigma^-1)_Z)),
  with O = I - Sigma^-1, so that 1 - O_Z = (Sigma^-1)_Z.

The subset sums run in the C core (tor_oracle.c) in ~212-bit arithmetic; the
matrices they start from are formed here in FP64 with numpy.
"""
from __future__ import annotations

import ctypes
import math
from fractions import Fraction
from itertools import product as _iproduct

import numpy as np

from . import _native

__all__ = [
    "QD", "symplectic", "covariance", "sigma", "mode_rows", "sigma_inv_block",
    "logdet_sigma", "to_real_basis", "from_real_basis", "subset_sum", "torontonian",
    "click_probability", "click_probability_sigma_form", "vacuum_probability",
    "single_mode_click_probability", "identity_torontonian", "mixture_pattern_probability",
    "hafnian", "pnr_click_probability", "conditioned_sigma", "no_click_probability",
    "sample_chain", "splitmix_uniform", "memory_gb", "all_pattern_probabilities",
    "qd_op", "qd_normalize", "det_qd",
]


# ------------------------------------------------------------- qd values --

class QD:
    """A value held as an unevaluated sum of doubles (as returned by the C core)."""

    __slots__ = ("c",)

    def __init__(self, comps):
        self.c = tuple(float(x) for x in comps)

    def __float__(self):
        return float(self.to_fraction())

    def to_fraction(self) -> Fraction:
        return sum((Fraction(x) for x in self.c), Fraction(0))

    def __repr__(self):
        return "QD(%r)" % (self.c,)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def qd_op(op: str, a, b=(0.0, 0.0, 0.0, 0.0)) -> QD:
    codes = {"add": 0, "mul": 1, "div": 2, "rsqrt": 3, "sub": 4}
    x = np.ascontiguousarray(a, dtype=np.float64)
    y = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(4)
    _native.lib().orc_qd_op(codes[op], _dp(x), _dp(y), _dp(out))
    return QD(out)


def qd_normalize(terms) -> QD:
    t = np.ascontiguousarray(terms, dtype=np.float64)
    out = np.zeros(4)
    _native.lib().orc_qd_normalize(_dp(t), int(t.size), _dp(out))
    return QD(out)


def det_qd(A: np.ndarray):
    """Determinant of a complex matrix by elimination with partial pivoting, in qd."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    d = A.shape[0]
    re, im = np.zeros(4), np.zeros(4)
    _native.lib().orc_det(d, _dp(A.view(np.float64)), _dp(re), _dp(im))
    return QD(re), QD(im)


# ------------------------------------------------------------------ state --

def symplectic(U: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Complex-basis Bogoliubov matrix of squeezers R = diag(r) followed by U:
    S = [[U ch R, U sh R], [U* sh R, U* ch R]]."""
    ch = np.cosh(r)
    sh = np.sinh(r)
    top = np.hstack([U * ch[None, :], U * sh[None, :]])
    bot = np.hstack([U.conj() * sh[None, :], U.conj() * ch[None, :]])
    return np.vstack([top, bot])


def covariance(U: np.ndarray, r, eta: float = 1.0) -> np.ndarray:
    """V = S S^+ / 2, then loss V -> eta V + (1 - eta) I/2 (transmissivity eta)."""
    r = np.asarray(r, dtype=np.float64)
    S = symplectic(np.asarray(U, dtype=np.complex128), r)
    V = 0.5 * (S @ S.conj().T)
    V = 0.5 * (V + V.conj().T)  # Hermitian by definition; drop the rounding asymmetry
    M = r.shape[0]
    return eta * V + (1.0 - eta) * 0.5 * np.eye(2 * M)


def sigma(V: np.ndarray) -> np.ndarray:
    return V + 0.5 * np.eye(V.shape[0])


def mode_rows(modes, M: int) -> np.ndarray:
    """Row indices {j, j+M} of the modes, mode-interleaved."""
    modes = np.asarray(modes, dtype=np.int64)
    out = np.empty(2 * modes.size, dtype=np.int64)
    out[0::2] = modes
    out[1::2] = modes + M
    return out


def sigma_inv_block(Sig: np.ndarray, modes) -> np.ndarray:
    """(Sigma^-1)_S, 2N x 2N, mode-interleaved, from a dense FP64 inverse."""
    M = Sig.shape[0] // 2
    ix = mode_rows(modes, M)
    Si = np.linalg.inv(Sig)
    Si = 0.5 * (Si + Si.conj().T)
    return np.ascontiguousarray(Si[np.ix_(ix, ix)])


def logdet_sigma(Sig: np.ndarray) -> float:
    sign, ld = np.linalg.slogdet(Sig)
    return float(ld)


def _real_basis_map(M: int) -> np.ndarray:
    """W with (a, a^+) = W (x_1, p_1, ..., x_M, p_M), a = (x + i p)/2 (hbar = 2)."""
    W = np.zeros((2 * M, 2 * M), dtype=np.complex128)
    for j in range(M):
        W[j, 2 * j] = 0.5
        W[j, 2 * j + 1] = 0.5j
        W[j + M, 2 * j] = 0.5
        W[j + M, 2 * j + 1] = -0.5j
    return W


def to_real_basis(V: np.ndarray) -> np.ndarray:
    """The paper's real covariance (Eq. 1, hbar = 2) of a complex-basis V."""
    M = V.shape[0] // 2
    Wi = np.linalg.inv(_real_basis_map(M))
    Vr = Wi @ V @ Wi.conj().T
    return np.ascontiguousarray(Vr.real)


def from_real_basis(Vr: np.ndarray) -> np.ndarray:
    M = Vr.shape[0] // 2
    W = _real_basis_map(M)
    return W @ Vr @ W.conj().T


# ------------------------------------------------------------ subset sums --

def subset_sum(G: np.ndarray, free, fixed=(), sign: str = "tor", method: str = "auto", nthreads=None):
    """sum_{W subset free} sign(W) det(G_{W u fixed})^(-1/2) in ~212-bit arithmetic.

    G is 2n x 2n complex Hermitian PD with mode i on rows 2i, 2i+1.  sign "tor"
    is (-1)^(|free|-|W|), sign "incl" is (-1)^|W|.  Returns (QD sum, sum of |terms|).
    method: "bruteforce" (every subset by its own LU), "tree" (Schur decision
    tree), "auto" (bruteforce up to 10 free modes, tree beyond).
    """
    G = np.ascontiguousarray(G, dtype=np.complex128)
    n = G.shape[0] // 2
    F = np.ascontiguousarray(free, dtype=np.int32)
    X = np.ascontiguousarray(fixed, dtype=np.int32)
    if F.size and (F.min() < 0 or F.max() >= n):
        raise ValueError("free mode out of range")
    if X.size and (X.min() < 0 or X.max() >= n):
        raise ValueError("fixed mode out of range")
    if method == "auto":
        method = "bruteforce" if F.size <= 10 else "tree"
    fn = {"bruteforce": _native.lib().orc_sum_bruteforce, "tree": _native.lib().orc_sum_tree}[method]
    out = np.zeros(4)
    asum = np.zeros(1)
    Fb = F if F.size else np.zeros(1, dtype=np.int32)
    Xb = X if X.size else np.zeros(1, dtype=np.int32)
    st = fn(n, _dp(G.view(np.float64)), int(F.size), _ip(Fb), int(X.size), _ip(Xb),
            0 if sign == "tor" else 1, int(nthreads or _native.nthreads()), _dp(out), _dp(asum))
    if st == 1:
        raise np.linalg.LinAlgError("a principal minor is not positive")
    if st != 0:
        raise ValueError("bad arguments")
    return QD(out), float(asum[0])


def torontonian(H: np.ndarray, method: str = "auto", nthreads=None):
    """Tor(O_S) from H = (Sigma^-1)_S: returns (QD value, sum of |terms|)."""
    n = H.shape[0] // 2
    return subset_sum(H, range(n), (), "tor", method, nthreads)


def click_probability(U, r, eta, modes, method="auto"):
    """p(S) = Tor(O_S) / sqrt(det Sigma).  Returns (p, Tor as QD, kappa = sum|t| / |Tor|)."""
    Sig = sigma(covariance(U, r, eta))
    H = sigma_inv_block(Sig, modes)
    tor, asum = torontonian(H, method)
    t = float(tor)
    p = t * math.exp(-0.5 * logdet_sigma(Sig))
    kappa = asum / abs(t) if t != 0.0 else math.inf
    return p, tor, kappa


def click_probability_sigma_form(V: np.ndarray, modes, method="bruteforce") -> float:
    """p(S) = sum_{W subset S} (-1)^|W| / sqrt(det Sigma_{W u S^c})  (no inverse)."""
    Sig = sigma(V)
    M = Sig.shape[0] // 2
    order = list(range(M))
    ix = mode_rows(order, M)
    G = Sig[np.ix_(ix, ix)]  # mode-interleaved, mode j on rows 2j, 2j+1
    S = sorted(int(j) for j in modes)
    Sc = [j for j in range(M) if j not in set(S)]
    val, _ = subset_sum(G, S, Sc, "incl", method)
    return float(val)


def vacuum_probability(Sig: np.ndarray, modes) -> float:
    """The paper's Eq. (5) for zero means: 1/sqrt(det Sigma_A)."""
    M = Sig.shape[0] // 2
    ix = mode_rows(modes, M)
    sub = Sig[np.ix_(ix, ix)]
    return 1.0 / math.sqrt(np.linalg.det(sub).real)


def all_pattern_probabilities(U, r, eta=1.0, method="auto"):
    """p(S) for all 2^M patterns, S given by the bits of the index (bit j = mode j)."""
    M = len(r)
    Sig = sigma(covariance(U, r, eta))
    Si = np.linalg.inv(Sig)
    Si = 0.5 * (Si + Si.conj().T)
    pref = math.exp(-0.5 * logdet_sigma(Sig))
    out = []
    for m in range(1 << M):
        modes = [j for j in range(M) if (m >> j) & 1]
        ix = mode_rows(modes, M)
        H = np.ascontiguousarray(Si[np.ix_(ix, ix)])
        tor, _ = torontonian(H, method, nthreads=1) if modes else (QD((1.0, 0, 0, 0)), 1.0)
        out.append(float(tor) * pref)
    return np.array(out)


# ------------------------------------------------------------ closed forms --

def single_mode_click_probability(r: float, eta: float = 1.0) -> float:
    """Click probability of one lossy squeezed mode: 1 - (1 + eta(2-eta) sinh^2 r)^(-1/2).

    det Sigma of a single mode is d+ d- with d+- = (eta e^{+-2r} + 2 - eta)/2, which
    equals 1 + eta (2 - eta) sinh^2 r; with eta = 1 this is 1 - 1/cosh r."""
    return 1.0 - (1.0 + eta * (2.0 - eta) * math.sinh(r) ** 2) ** -0.5


def identity_torontonian(r, eta, modes) -> float:
    """Tor(O_S) for independent modes: prod_{j in S} (sqrt(det Sigma_j) - 1)."""
    r = np.asarray(r, dtype=np.float64)
    out = 1.0
    for j in modes:
        dj = 1.0 + eta * (2.0 - eta) * math.sinh(r[j]) ** 2
        out *= math.sqrt(dj) - 1.0
    return out


# ----------------------------------------- the paper's mixture algorithm --

def mixture_pattern_probability(Vr: np.ndarray, clicks) -> float:
    """Probability of a full click pattern by the paper's Sec. II update rule.

    Vr is the paper's real covariance (x_1, p_1, ..., x_l, p_l), hbar = 2, zero
    means.  Modes are measured from the last one down (the paper starts at the
    l-th mode).  The state is a list of (a_k, V_k).  For the measured mode B
    each term has q_k = 2 / sqrt(det(V_B + 1)) (Eq. 5 with zero means) and the
    no-click update V_A' = V_A - V_AB (V_B + 1)^-1 V_AB^T (Eq. 4a); p = sum a_k q_k
    is the no-click probability.  A click keeps both V_A (weight a_k/(1-p)) and
    V_A' (weight -a_k q_k/(1-p)) (Eq. 6); no click keeps V_A' with a_k q_k / p
    (Eq. 7).  The pattern probability is the product of the branch probabilities.
    """
    clicks = set(int(j) for j in clicks)
    ell = Vr.shape[0] // 2
    comps = [(1.0, np.array(Vr, dtype=np.float64))]
    prob = 1.0
    for mode in range(ell - 1, -1, -1):
        new = []
        qs = []
        for a, V in comps:
            A = V[:-2, :-2]
            AB = V[:-2, -2:]
            B = V[-2:, -2:]
            Binv = np.linalg.inv(B + np.eye(2))
            q = 2.0 / math.sqrt(np.linalg.det(B + np.eye(2)))
            Ap = A - AB @ Binv @ AB.T
            qs.append((a, q, A, Ap))
        p = sum(a * q for a, q, _, _ in qs)
        if mode in clicks:
            prob *= 1.0 - p
            for a, q, A, Ap in qs:
                new.append((a / (1.0 - p), A))
                new.append((-a * q / (1.0 - p), Ap))
        else:
            prob *= p
            for a, q, A, Ap in qs:
                new.append((a * q / p, Ap))
        comps = new
    return prob


# -------------------------------------------------- photon-number brute force --

def hafnian(A: np.ndarray) -> complex:
    """Hafnian by expansion along the first row over perfect matchings (memoised on the row set)."""
    n = A.shape[0]
    if n % 2:
        return 0.0
    memo = {}

    def rec(mask: int) -> complex:
        if mask == 0:
            return 1.0
        if mask in memo:
            return memo[mask]
        i = (mask & -mask).bit_length() - 1
        rest = mask & ~(1 << i)
        tot = 0.0
        m = rest
        while m:
            j = (m & -m).bit_length() - 1
            m &= m - 1
            tot += A[i, j] * rec(rest & ~(1 << j))
        memo[mask] = tot
        return tot

    return rec((1 << n) - 1)


def pnr_click_probability(U, r, clicks, n_max: int):
    """Click-pattern probability of a pure state summed from photon-number probabilities.

    P(n) = |haf(B_n)|^2 / (prod n_j! sqrt(det Sigma)), B = U tanh(R) U^T, for every
    n with n_j >= 1 on the clicked modes, n_j = 0 elsewhere and sum n <= n_max.
    Returns (truncated sum, total probability of all n with sum n <= n_max), so the
    truncation error is at most 1 - total.
    """
    U = np.asarray(U, dtype=np.complex128)
    r = np.asarray(r, dtype=np.float64)
    M = r.shape[0]
    B = U @ np.diag(np.tanh(r)) @ U.T
    Sig = sigma(covariance(U, r, 1.0))
    pref = math.exp(-0.5 * logdet_sigma(Sig))
    clicks = set(int(j) for j in clicks)
    total = 0.0
    part = 0.0
    for n in _iproduct(range(n_max + 1), repeat=M):
        s = sum(n)
        if s > n_max or s % 2:
            continue
        idx = [j for j in range(M) for _ in range(n[j])]
        Bn = B[np.ix_(idx, idx)] if idx else np.zeros((0, 0))
        h = hafnian(Bn) if idx else 1.0
        fac = 1.0
        for j in range(M):
            fac *= math.factorial(n[j])
        p = abs(h) ** 2 * pref / fac
        total += p
        if all((n[j] >= 1) == (j in clicks) for j in range(M)):
            part += p
    return part, total


# ---------------------------------------------------------------- sampler --

GAMMA = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def splitmix_uniform(seed: int, sample: int, step: int, attempt: int = 0) -> float:
    """The sampler's coin: output n = 1 + step + 2^20 (attempt + 2^12 sample) of the
    SplitMix64 stream with state ``seed`` (Steele et al. 2014), top 53 bits / 2^53."""
    n = 1 + step + (1 << 20) * (attempt + (1 << 12) * sample)
    z = (seed + n * GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    z ^= z >> 31
    return (z >> 11) * 2.0 ** -53


def conditioned_sigma(Sig: np.ndarray, noclick, keep) -> np.ndarray:
    """Sigma of the modes ``keep`` after projecting the modes ``noclick`` on vacuum:
    Sigma_T - Sigma_TU Sigma_U^-1 Sigma_UT (the paper's Eq. 4a written with Sigma),
    mode-interleaved in the order of ``keep``; recomputed from scratch."""
    M = Sig.shape[0] // 2
    it = mode_rows(keep, M)
    S_T = Sig[np.ix_(it, it)]
    if len(noclick) == 0:
        return np.ascontiguousarray(S_T)
    iu = mode_rows(noclick, M)
    S_U = Sig[np.ix_(iu, iu)]
    S_TU = Sig[np.ix_(it, iu)]
    out = S_T - S_TU @ np.linalg.solve(S_U, S_TU.conj().T)
    return np.ascontiguousarray(0.5 * (out + out.conj().T))


def no_click_probability(Sig: np.ndarray, clicks, noclicks, k: int):
    """P(no click at k | clicks on S, no clicks on U), measured so far.

    = sum_W (-1)^|W| det(Sigma'_{W u k})^-1/2 / sum_W (-1)^|W| det(Sigma'_W)^-1/2 over
    W subset S, with Sigma' the state conditioned on vacuum at U (Eqs. 5-7 in closed
    form).  Returns (p0, numerator QD, denominator QD).
    """
    S = [int(j) for j in clicks]
    G = conditioned_sigma(Sig, list(noclicks), S + [int(k)])
    m = len(S)
    den, _ = subset_sum(G, range(m), (), "incl")
    num, _ = subset_sum(G, range(m), (m,), "incl")
    return float(num.to_fraction() / den.to_fraction()), num, den


def sample_chain(Sig: np.ndarray, seed: int, sample: int = 0, forced_clicks=None, N_post: int = 0,
                 max_attempts: int = 1, steps_to_check=None):
    """One chain-rule sample, modes measured from the last to the first.

    forced_clicks: the paper's forced-outcome benchmark (the coin is replaced by a
    preset outcome); the no-click probability is still evaluated at every step.
    Otherwise u = splitmix_uniform(seed, sample, step, attempt) and the mode stays
    dark iff u < p0.  N_post > 0 rejects a trajectory as soon as it can no longer
    end with exactly N_post clicks and retries with the next attempt index.
    Returns dict(pattern, p0 list, u list, attempts, near_ties).
    """
    M = Sig.shape[0] // 2
    forced = None if forced_clicks is None else set(int(j) for j in forced_clicks)
    for attempt in range(max_attempts):
        S, U, p0s, us = [], [], [], []
        ok = True
        near = 0
        for step, k in enumerate(range(M - 1, -1, -1)):
            if steps_to_check is not None and step not in steps_to_check and forced is not None:
                # forced outcome without evaluating p0 at this step
                (S if k in forced else U).append(k)
                p0s.append(None)
                us.append(None)
                continue
            p0, _, _ = no_click_probability(Sig, S, U, k)
            p0s.append(p0)
            if forced is not None:
                click = k in forced
                us.append(None)
            else:
                u = splitmix_uniform(seed, sample, step, attempt)
                us.append(u)
                if abs(u - p0) < 1e-9:
                    near += 1
                click = not (u < p0)
            (S if click else U).append(k)
            if N_post and forced is None:
                if len(S) > N_post or len(S) + k < N_post:
                    ok = False
                    break
        if ok:
            pat = np.zeros(M, dtype=np.uint8)
            pat[S] = 1
            return dict(pattern=pat, p0=p0s, u=us, attempts=attempt + 1, near_ties=near)
    return dict(pattern=None, p0=p0s, u=us, attempts=max_attempts, near_ties=near)


# ------------------------------------------------------------ memory model --

def memory_gb(ell: int, m: int, k: int, eta: float = 2.0) -> float:
    """The paper's Eq. (memory): eta 2^(m-24) (ell-k)^2 GB to store 2^m quad covariances."""
    return eta * 2.0 ** (m - 24) * (ell - k) ** 2
