"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the method's arithmetic: it only draws numbers.
Random numbers come from xoshiro256** streams (Blackman & Vigna, 2018) seeded
by SplitMix64 (Steele, Lea & Flood, 2014), run as many independent lanes in
lock-step so that numpy can vectorise them; normals use the Box-Muller
transform; Haar-distributed orthogonal matrices come from the QR factors of a
Gaussian matrix with diag(R) made positive (Mezzadri, 2007).

Seeds follow the scheme ``BASE_SEED + workload_index * 0x1000 + instance``.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x2604039600000000
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def workload_seed(workload_index: int, instance: int = 0) -> int:
    return (BASE_SEED + workload_index * 0x1000 + instance) & 0xFFFFFFFFFFFFFFFF


def _splitmix64(state: int, count: int) -> list[int]:
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        out.append(z ^ (z >> 31))
    return out


def _rotl(x: np.ndarray, k: int) -> np.ndarray:
    return (x << np.uint64(k)) | (x >> np.uint64(64 - k))


class Xoshiro:
    """``lanes`` independent xoshiro256** generators advanced in lock-step."""

    def __init__(self, seed: int, lanes: int = 1024):
        words = _splitmix64(seed & 0xFFFFFFFFFFFFFFFF, 4 * lanes)
        s = np.array(words, dtype=np.uint64).reshape(lanes, 4)
        self.s0, self.s1, self.s2, self.s3 = (s[:, i].copy() for i in range(4))
        self.lanes = lanes

    def _step(self) -> np.ndarray:
        with np.errstate(over="ignore"):
            result = _rotl(self.s1 * np.uint64(5), 7) * np.uint64(9)
            t = self.s1 << np.uint64(17)
            self.s2 ^= self.s0
            self.s3 ^= self.s1
            self.s1 ^= self.s2
            self.s0 ^= self.s3
            self.s2 ^= t
            self.s3 = _rotl(self.s3, 45)
        return result

    def u64(self, n: int) -> np.ndarray:
        steps = -(-n // self.lanes)
        out = np.empty((steps, self.lanes), dtype=np.uint64)
        for i in range(steps):
            out[i] = self._step()
        return out.reshape(-1)[:n]

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (pairs from two uniforms)."""
        m = -(-n // 2)
        u1 = 1.0 - self.uniform(m)            # in (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(2.0 * np.pi * u2)
        z[1::2] = r * np.sin(2.0 * np.pi * u2)
        return z[:n]


def gaussian(seed: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    return Xoshiro(seed, lanes=min(4096, max(64, n // 64))).normal(n).reshape(shape)


def haar_orthogonal(seed: int, n: int) -> np.ndarray:
    """Haar-distributed n x n orthogonal matrix (QR of a Gaussian, diag(R) > 0)."""
    G = gaussian(seed, (n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def spectrum(kind: str, n: int, chi: int) -> np.ndarray:
    """The two prescribed spectra of the isolated-SVD workload:
    'exp': s_k = exp(-k / (0.1 chi)), 'pow': s_k = (k+1)^-1.5, k = 0..n-1."""
    k = np.arange(n, dtype=np.float64)
    if kind == "exp":
        return np.exp(-k / (0.1 * chi))
    if kind == "pow":
        return (k + 1.0) ** -1.5
    raise ValueError(kind)


def svd_test_matrix(seed: int, m: int, n: int, s: np.ndarray) -> np.ndarray:
    """A = U[:, :r] diag(s) V[:, :r]^T with Haar U (m x m), V (n x n), r = len(s)."""
    r = len(s)
    U = haar_orthogonal(seed, m)[:, :r]
    V = haar_orthogonal(seed + 1, n)[:, :r]
    return (U * s[None, :]) @ V.T


def initial_mps_entries(seed: int, N: int, chi_init: int, d: int = 2) -> np.ndarray:
    """Gaussian entries of the initial MPS, site after site, each site a
    chi_{i} x d x chi_{i+1} block with chi_i = min(chi_init, d^i, d^(N-i))."""
    chi = [min(chi_init, d ** i, d ** (N - i)) for i in range(N + 1)]
    total = sum(chi[i] * d * chi[i + 1] for i in range(N))
    return gaussian(seed, (total,))


def uneven_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), e.g. chi of the uneven SVD batch."""
    u = Xoshiro(seed, lanes=64).u64(count)
    return (lo + (u % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def uniform_range(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * Xoshiro(seed, lanes=64).uniform(count)


def brickwork_circuit(seed: int, N: int, n_layers: int):
    """A hardware-efficient circuit on N qubits: layer l holds two-qubit gates
    on the pairs (q, q+1) with q = l mod 2, l mod 2 + 2, ...; each gate is a
    CNOT (control q) after single-qubit RY rotations on both qubits, with
    angles uniform in [0, 2 pi) from the seeded generator.  Real gates, as
    4 x 4 matrices G[(s1' s2')][(s1 s2)], index 2 s1 + s2, s1 = qubit q.
    Returns [(positions, gates (n x 4 x 4))] per layer."""
    rng = Xoshiro(seed, lanes=64)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.float64)
    layers = []
    for l in range(n_layers):
        pos = list(range(l % 2, N - 1, 2))
        ang = rng.uniform(2 * len(pos)) * 2.0 * np.pi
        gates = []
        for g in range(len(pos)):
            a, b = ang[2 * g] / 2.0, ang[2 * g + 1] / 2.0
            ry_a = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
            ry_b = np.array([[np.cos(b), -np.sin(b)], [np.sin(b), np.cos(b)]])
            gates.append(cnot @ np.kron(ry_a, ry_b))
        layers.append((np.array(pos, dtype=np.int32), np.array(gates).reshape(len(pos), 4, 4)))
    return layers
