"""Seeded synthetic inputs for threshold Gaussian Boson Sampling workloads.

This module is shared by the CPU oracle (``oracle/``) and the GPU path
(``paper_1810_00900_gb300``), and by the benchmark.  It holds *none* of the
method's arithmetic: it only draws the physical parameters of a state
(interferometer U, squeezing r, transmissivity eta), click patterns, forced
click positions, graphs and request streams.  Everything that turns those
parameters into covariances, probabilities or samples lives on either side of
the boundary, separately.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the n-th output
(n = 1, 2, ...) of the stream with state ``seed`` is ``mix(seed + n * GAMMA)``.
Each named input stream gets its own 64-bit seed derived from the workload
seed, so that e.g. the unitary and the click pattern of one workload are
independent.

Workloads mirror the paper's benchmark inputs: Haar-random interferometers
(Sec. III, "unitaries drawn from the Haar measure"), uniform or random
squeezing (the paper uses 8 dB, r ~ 0.921), losses given as transmissivity
(Sec. IV: 1.2 / 3 / 6 dB), and planted dense-subgraph graphs (Sec. IV A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

# Stream identifiers: one independent SplitMix64 stream per kind of input.
STREAMS = {
    "unitary": 1,
    "squeezing": 2,
    "modes": 3,
    "eta": 4,
    "graph": 5,
    "clicks": 6,
    "arrivals": 7,
    "requests": 8,
    "uniform-subsets": 9,
}


def mix64(z: int) -> int:
    """SplitMix64 output function (finaliser) on a Python int."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def stream_seed(seed: int, stream: str) -> int:
    """64-bit seed of the named stream of workload ``seed``."""
    return mix64((seed & MASK64) * GAMMA + STREAMS[stream] * 0xD1B54A32D192ED03)


def u64_block(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start+1 .. start+count`` of the SplitMix64 stream ``seed``."""
    n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + n * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each output times 2^-53."""
    return (u64_block(seed, start, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform on consecutive uniform pairs."""
    pairs = (count + 1) // 2
    u = uniforms(seed, 0, 2 * pairs)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def haar_unitary(M: int, seed: int) -> np.ndarray:
    """Haar-random M x M unitary (F. Mezzadri, Notices AMS 54, 2007).

    QR of a complex Gaussian matrix with entries (g1 + i g2)/sqrt(2), then each
    column of Q is multiplied by the phase of the matching diagonal entry of R,
    which makes the distribution exactly Haar.  The Gaussians are drawn from
    the "unitary" stream of ``seed``, row-major, real part first.
    """
    g = normals(stream_seed(seed, "unitary"), 2 * M * M).reshape(M, M, 2)
    Z = (g[..., 0] + 1j * g[..., 1]) / math.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R)
    ph = d / np.abs(d)
    return np.ascontiguousarray(Q * ph[None, :])


def uniform_range(seed: int, stream: str, count: int, lo: float, hi: float, start: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniforms(stream_seed(seed, stream), start, count)


def random_modes(M: int, N: int, seed: int, stream: str = "modes", start: int = 0) -> np.ndarray:
    """N distinct modes out of M, uniformly at random (partial Fisher-Yates), sorted."""
    if not 0 <= N <= M:
        raise ValueError("need 0 <= N <= M")
    u = uniforms(stream_seed(seed, stream), start, N)
    perm = list(range(M))
    for i in range(N):
        j = i + int(u[i] * (M - i))
        perm[i], perm[j] = perm[j], perm[i]
    return np.array(sorted(perm[:N]), dtype=np.int32)


def db_to_eta(db: float) -> float:
    """Transmissivity for a loss given in dB (eta = 10^(-dB/10))."""
    return 10.0 ** (-db / 10.0)


def db_to_r(db: float) -> float:
    """Squeezing parameter for a squeezing level in dB (r = dB / (20 log10 e))."""
    return db / (20.0 * math.log10(math.e))


@dataclass
class StateParams:
    """Physical parameters of a lossy squeezed-vacuum + interferometer state."""

    U: np.ndarray  # M x M complex unitary
    r: np.ndarray  # M squeezing parameters
    eta: float = 1.0  # transmissivity in (0, 1]

    @property
    def M(self) -> int:
        return int(self.r.shape[0])


def uniform_squeezed_state(M: int, r: float, seed: int, eta: float = 1.0) -> StateParams:
    return StateParams(haar_unitary(M, seed), np.full(M, float(r)), float(eta))


def identity_state(r, eta: float = 1.0) -> StateParams:
    """Independent squeezed modes (identity interferometer)."""
    r = np.asarray(r, dtype=np.float64)
    return StateParams(np.eye(r.shape[0], dtype=np.complex128), r.copy(), float(eta))


# ---------------------------------------------------------------- workloads --

def small_all_patterns_workload():
    """8 modes, r = 0.5 in every mode, Haar unitary seed 0, no loss; all 256 patterns."""
    st = uniform_squeezed_state(8, 0.5, seed=0)
    patterns = [np.array([j for j in range(8) if (m >> j) & 1], dtype=np.int32) for m in range(256)]
    return st, patterns


def single_large_torontonian_workload(N: int = 24):
    """200 modes, r = 0.8, Haar unitary seed 1, no loss; one N-click pattern on random modes."""
    st = uniform_squeezed_state(200, 0.8, seed=1)
    return st, random_modes(200, N, seed=1)


# Mode counts of the paper's walltime benchmark (Table II): l modes for m clicks.
# the paper's Table II sizes, then two rows past its largest one with l = 2 m^2
WALLTIME_MODES = {10: 200, 12: 288, 14: 392, 16: 512, 18: 624, 20: 800, 22: 968, 24: 1152}


def walltime_workload(m: int, seed: int = 10):
    """The paper's walltime benchmark (Sec. III B, Table II) for m clicks: l modes
    (WALLTIME_MODES), 8 dB squeezing in every mode, Haar unitary (seed + m), no loss,
    and the worst-case click positions -- the first m measured modes (l-1 .. l-m, the
    measurement runs from the last mode down) -- as forced outcomes."""
    M = WALLTIME_MODES[m]
    st = StateParams(haar_unitary(M, seed + m), np.full(M, db_to_r(8.0)), 1.0)
    return st, np.arange(M - 1, M - 1 - m, -1, dtype=np.int64)


def walltime_random_positions(m: int, count: int, seed: int = 10) -> np.ndarray:
    """count sets of m click positions drawn uniformly from the WALLTIME_MODES[m] modes (the
    paper's random-position runs beside the worst case)."""
    M = WALLTIME_MODES[m]
    return np.array([random_modes(M, m, seed + m, stream="clicks", start=i * m) for i in range(count)])


def chain_sampling_workload(M: int = 800, n_clicks: int = 20, n_traj: int = 64, seed: int = 2):
    """M modes, r ~ U[0.3, 0.9] per mode, Haar unitary, no loss, plus n_traj forced
    click-position sets of n_clicks modes each (drawn uniformly, the paper's forced-outcome
    benchmark of Sec. III B)."""
    U = haar_unitary(M, seed)
    r = uniform_range(seed, "squeezing", M, 0.3, 0.9)
    clicks = [random_modes(M, n_clicks, seed, stream="clicks", start=t * n_clicks) for t in range(n_traj)]
    return StateParams(U, r, 1.0), clicks


@dataclass
class TorRequest:
    M: int
    N: int
    r: float
    eta: float
    seed: int
    modes: np.ndarray = field(repr=False)


def batched_requests(n_req: int = 4096, seed: int = 3, Ms=(100, 200, 400), N_range=(8, 22),
                     r_range=(0.4, 1.0), eta_range=(0.25, 1.0)):
    """Mixed Torontonian requests: N ~ U{N_range}, M ~ U(Ms), r ~ U[r_range], eta ~ U[eta_range].

    Request i uses Haar seed ``seed * 1_000_003 + i`` and its own click modes.
    """
    s = stream_seed(seed, "requests")
    u = uniforms(s, 0, 4 * n_req).reshape(n_req, 4)
    out = []
    for i in range(n_req):
        N = N_range[0] + int(u[i, 0] * (N_range[1] - N_range[0] + 1))
        M = Ms[int(u[i, 1] * len(Ms))]
        r = r_range[0] + (r_range[1] - r_range[0]) * u[i, 2]
        eta = eta_range[0] + (eta_range[1] - eta_range[0]) * u[i, 3]
        rs = seed * 1_000_003 + i
        out.append(TorRequest(M, N, float(r), float(eta), rs, random_modes(M, N, rs)))
    return out


def planted_graph(n: int, seed: int, p: float = 0.1, k: int = 20, q: float = 0.9) -> np.ndarray:
    """Erdos-Renyi G(n, p) adjacency with a planted dense part of k vertices at edge probability q."""
    s = stream_seed(seed, "graph")
    u = uniforms(s, 0, n * n).reshape(n, n)
    A = (u < p).astype(np.float64)
    planted = random_modes(n, k, seed, stream="graph", start=n * n)
    for a in planted:
        for b in planted:
            A[a, b] = 1.0 if u[b, a] < q else A[a, b]
    A = np.triu(A, 1)
    A = A + A.T
    return A


def planted_vertices(n: int, seed: int, k: int = 20) -> np.ndarray:
    """The k vertices planted_graph(n, seed, k=k) made dense."""
    return random_modes(n, k, seed, stream="graph", start=n * n)


def uniform_subsets(n: int, size: int, count: int, seed: int) -> np.ndarray:
    """count subsets of `size` vertices out of n, uniformly at random (the baseline of random search)."""
    return np.array([random_modes(n, size, seed, stream="uniform-subsets", start=i * size) for i in range(count)])


def graph_state(A: np.ndarray, mean_photons: float, eta: float = 1.0) -> StateParams:
    """Encode a graph into a GBS state (the encoding the paper uses for dense subgraphs, Sec. IV,
    after its Ref. on GBS and graphs): Takagi factorisation c A = U diag(tanh r) U^T of the scaled
    adjacency matrix, with c chosen by bisection so that the mean photon number sum_j sinh^2 r_j
    equals mean_photons, then uniform loss eta.

    For real symmetric A = O diag(mu) O^T the Takagi factors are lambda = |mu| and U = O diag(phase),
    phase_j = 1 (mu_j >= 0) or i (mu_j < 0), so that U diag(lambda) U^T = A.
    """
    mu, O = np.linalg.eigh(np.asarray(A, dtype=np.float64))
    lam = np.abs(mu)
    U = O * np.where(mu >= 0, 1.0, 1j)[None, :]
    lmax = lam.max()

    def nbar(c):
        t = c * lam
        return float(np.sum(t * t / (1.0 - t * t)))

    lo, hi = 0.0, (1.0 - 1e-12) / lmax
    if nbar(hi) < mean_photons:
        raise ValueError("mean photon number out of reach for this graph")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if nbar(mid) < mean_photons:
            lo = mid
        else:
            hi = mid
    c = 0.5 * (lo + hi)
    return StateParams(np.ascontiguousarray(U), np.arctanh(c * lam), float(eta))


def served_stream_workload(n_req: int, seed: int = 5, rate_hz: float = 200.0, n_graphs: int = 4):
    """Requests of the served dense-subgraph stream: Poisson arrival times, and per request a
    graph (Erdos-Renyi n in [100, 200], p = 0.1, planted 20-vertex part at p = 0.9), a loss
    eta in {1, 0.5, 0.25} and a postselected click count N in [8, 20]; the state of request
    (graph, eta, N) has mean photon number 2N.  Returns (arrivals, [(graph, eta, N)], graphs)."""
    s = stream_seed(seed, "requests")
    u = uniforms(s, 0, 3 * n_req + n_graphs).reshape(-1)
    graphs = [planted_graph(100 + int(u[3 * n_req + g] * 101), seed * 97 + g) for g in range(n_graphs)]
    reqs = []
    for i in range(n_req):
        g = int(u[3 * i] * n_graphs)
        eta = (1.0, 0.5, 0.25)[int(u[3 * i + 1] * 3)]
        N = 8 + int(u[3 * i + 2] * 13)
        reqs.append((g, eta, N))
    return poisson_arrivals(rate_hz, n_req, seed), reqs, graphs


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    u = uniforms(stream_seed(seed, "arrivals"), 0, n)
    return np.cumsum(-np.log(1.0 - u) / rate_hz)
