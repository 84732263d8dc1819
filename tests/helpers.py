"""Test helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def real_basis_block(H: np.ndarray) -> np.ndarray:
    """Mode-interleaved complex (a_j, a_j^+) matrix -> the (x_j, p_j) matrix q^+ H q,
    q = [[1, i], [1, -i]] / sqrt(2) per mode (a unitary change of basis: same minors)."""
    n = H.shape[0] // 2
    q = np.array([[1, 1j], [1, -1j]]) / np.sqrt(2)
    Q = np.kron(np.eye(n), q)
    R = Q.conj().T @ H @ Q
    assert np.abs(R.imag).max() < 1e-12 * max(1.0, np.abs(R).max())
    R = R.real
    return np.ascontiguousarray(0.5 * (R + R.T))


def td_value(x) -> float:
    return float(x[0]) + (float(x[1]) + float(x[2]))


def frac3(x):
    from fractions import Fraction
    return Fraction(float(x[0])) + Fraction(float(x[1])) + Fraction(float(x[2]))


# Parity references: the oracle's plain definition (O1: every subset by its own
# LU, ~212-bit) up to BRUTE_N modes, its decision tree (O2) beyond; O2 itself
# is pinned to O1 up to 16 modes by the CPU tests.
BRUTE_N = 14
_TOR_CACHE = {}


def ref_method(n: int) -> str:
    return "bruteforce" if n <= BRUTE_N else "tree"


def oracle_tor(G):
    """(Tor as the oracle's QD value, sum of |terms|) of a 2n x 2n block, cached per matrix."""
    import oracle
    G = np.ascontiguousarray(G, dtype=np.complex128)
    key = (G.shape, G.tobytes())
    if key not in _TOR_CACHE:
        _TOR_CACHE[key] = oracle.torontonian(G, ref_method(G.shape[0] // 2))
    return _TOR_CACHE[key]
