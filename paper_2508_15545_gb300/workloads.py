"""Seeded synthetic inputs: circuits, random states, random matrices, Hamiltonians.

This module is shared by the CUDA path, the oracle, the tests and the bench. It
holds none of the simulation arithmetic: it only draws random numbers and writes
gate LISTS (kind, qubits, angles). Each side turns a gate record into a matrix
with its own code.

Conventions
-----------
* Qubit q is bit q of the amplitude index (little-endian). The paper's pairing
  rule (Sec. III-A, Eq. 5) pairs index i with i XOR 2^k for a gate on qubit k.
* A gate record is a ``Gate`` named tuple:
  ``kind``   one of ``GATE_KINDS``;
  ``target`` the qubit the 2x2 matrix acts on (for ``swap``: the first qubit);
  ``target2`` the second qubit of ``swap``, else -1;
  ``ctrl``   control qubit (the gate acts where that bit is 1), or -1;
  ``theta``  three angles (unused ones are 0);
  ``param``  three parameter indices, one per angle, -1 when not trainable;
  ``matrix`` four complex numbers (row-major U00, U01, U10, U11) for ``matrix``.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): uniform doubles take the top 53
bits; normal deviates use the Box-Muller transform.
"""
from __future__ import annotations

import math
from typing import List, NamedTuple, Sequence, Tuple

import numpy as np

GATE_KINDS = ("h", "x", "y", "z", "s", "sdg", "t", "tdg",
              "rx", "ry", "rz", "p", "u3", "matrix", "swap")
PARAMETRIC = {"rx": 1, "ry": 1, "rz": 1, "p": 1, "u3": 3}

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


class Gate(NamedTuple):
    kind: str
    target: int
    target2: int = -1
    ctrl: int = -1
    theta: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    param: Tuple[int, int, int] = (-1, -1, -1)
    matrix: Tuple[complex, complex, complex, complex] | None = None


class SplitMix64:
    """SplitMix64 stream; ``next_block(k)`` returns the next k outputs as uint64."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_block(self, count: int) -> np.ndarray:
        k = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + count * int(_GAMMA)) & _MASK64
        return z

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.next_block(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, count: int, sigma: float = 1.0) -> np.ndarray:
        """Box-Muller normal deviates N(0, sigma^2)."""
        m = (count + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return sigma * z[:count]

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + np.floor(self.uniform(count) * span).astype(np.int64)


def config_seed(config: int, index: int = 0) -> int:
    """Seed of circuit ``index`` of workload ``config``: (1000 + config) in the
    high 32 bits, the circuit index in the low 32 bits."""
    return ((1000 + config) << 32) | (index & 0xFFFFFFFF)


# ----------------------------------------------------------------------------
# circuits
# ----------------------------------------------------------------------------
def brickwork_pairs(n: int, layer: int) -> List[Tuple[int, int]]:
    """CNOT pairs of one brickwork layer: even layers (0,1),(2,3)...; odd layers
    (1,2),(3,4)...; pairs past the last qubit are dropped. Control = first."""
    start = layer % 2
    return [(a, a + 1) for a in range(start, n - 1, 2)]


def random_circuit(n: int, layers: int, seed: int) -> List[Gate]:
    """Random-circuit recipe: each layer applies U3(theta, phi, lambda) to every
    qubit (angles uniform in [0, 2 pi), drawn qubit by qubit, three per qubit),
    then CNOT on the layer's brickwork pairs."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    for layer in range(layers):
        ang = rng.uniform(3 * n) * (2.0 * math.pi)
        for q in range(n):
            th = (float(ang[3 * q]), float(ang[3 * q + 1]), float(ang[3 * q + 2]))
            gates.append(Gate("u3", q, theta=th))
        for c, t in brickwork_pairs(n, layer):
            gates.append(Gate("x", t, ctrl=c))
    return gates


def ansatz_circuit(n: int, layers: int, seed: int, sigma: float = 0.5,
                   ry_first: bool = True) -> Tuple[List[Gate], int]:
    """Hardware-efficient ansatz: per layer RY(theta_q) on every qubit, then
    RZ(phi_q) on every qubit, then CZ(i, (i+1) mod n) for i = 0..n-1. Angles are
    N(0, sigma^2). Parameter index = layer*2n + q for RY, layer*2n + n + q for RZ.
    Returns (gates, number of parameters). For n = 2 the ring's two CZs cancel."""
    rng = SplitMix64(seed)
    angles = rng.normal(2 * n * layers, sigma)
    gates: List[Gate] = []
    for layer in range(layers):
        base = layer * 2 * n
        rot = [("ry", base), ("rz", base + n)]
        if not ry_first:
            rot.reverse()
        for kind, off in rot:
            for q in range(n):
                gates.append(Gate(kind, q, theta=(float(angles[off + q]), 0.0, 0.0),
                                  param=(off + q, -1, -1)))
        for i in range(n):
            gates.append(Gate("z", (i + 1) % n, ctrl=i))
    return gates, 2 * n * layers


def with_params(gates: Sequence[Gate], params: Sequence[float]) -> List[Gate]:
    """Copy of ``gates`` whose trainable angles are replaced by ``params``."""
    out = []
    for g in gates:
        if any(p >= 0 for p in g.param):
            th = tuple(float(params[p]) if p >= 0 else g.theta[i] for i, p in enumerate(g.param))
            out.append(g._replace(theta=th))
        else:
            out.append(g)
    return out


def qft_circuit(n: int, with_swaps: bool = True) -> List[Gate]:
    """Quantum Fourier transform on n qubits (little-endian), written so that
    the output is sum_k exp(2 pi i j k / 2^n) |k> / 2^(n/2) for input |j>: for
    a = n-1 down to 0, H on a then CP(pi / 2^(a-b)) controlled by b for b = a-1
    down to 0; finally SWAP(a, n-1-a) for a < n/2."""
    gates: List[Gate] = []
    for a in range(n - 1, -1, -1):
        gates.append(Gate("h", a))
        for b in range(a - 1, -1, -1):
            gates.append(Gate("p", a, ctrl=b, theta=(math.pi / (1 << (a - b)), 0.0, 0.0)))
    if with_swaps:
        for a in range(n // 2):
            gates.append(Gate("swap", a, target2=n - 1 - a))
    return gates


def ghz_circuit(n: int) -> List[Gate]:
    """H on qubit 0, then CNOT(q, q+1) for q = 0..n-2."""
    return [Gate("h", 0)] + [Gate("x", q + 1, ctrl=q) for q in range(n - 1)]


def uneven_batch(count: int, seed: int, n_lo: int = 16, n_hi: int = 28,
                 d_lo: int = 10, d_hi: int = 60) -> List[Tuple[int, int, int]]:
    """(n, depth, circuit seed) triples: n uniform in [n_lo, n_hi], depth uniform
    in [d_lo, d_hi]; each circuit follows ``random_circuit``."""
    rng = SplitMix64(seed)
    ns = rng.integers(n_lo, n_hi, count)
    ds = rng.integers(d_lo, d_hi, count)
    return [(int(ns[i]), int(ds[i]), seed * 1000003 + i) for i in range(count)]


def random_gate_list(n: int, count: int, seed: int, kinds: Sequence[str] = GATE_KINDS,
                     ctrl_prob: float = 0.3) -> List[Gate]:
    """Random mix of gate kinds on random qubits (tests: every kind, every
    target, random controls)."""
    rng = SplitMix64(seed)
    out: List[Gate] = []
    for _ in range(count):
        u = rng.uniform(8)
        kind = kinds[int(u[0] * len(kinds)) % len(kinds)]
        t = int(u[1] * n) % n
        th = tuple(float(x) for x in (rng.uniform(3) * 2 * math.pi - math.pi))
        if kind == "swap":
            if n < 2:
                continue
            t2 = (t + 1 + int(u[2] * (n - 1)) % (n - 1)) % n
            out.append(Gate("swap", t, target2=t2))
            continue
        ctrl = -1
        if n >= 2 and u[3] < ctrl_prob:
            ctrl = (t + 1 + int(u[4] * (n - 1)) % (n - 1)) % n
        mat = None
        if kind == "matrix":
            mat = tuple(complex(x) for x in random_unitary(rng).reshape(-1))
        out.append(Gate(kind, t, ctrl=ctrl, theta=th, matrix=mat))
    return out


# ----------------------------------------------------------------------------
# states, matrices, Hamiltonians
# ----------------------------------------------------------------------------
def random_unitary(rng: SplitMix64) -> np.ndarray:
    """2x2 Haar-random unitary: QR of a complex Gaussian matrix, with the phases
    of R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    z = rng.normal(8).reshape(2, 2, 2)
    a = z[0] + 1j * z[1]
    q, r = np.linalg.qr(a)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_matrix_2x2(seed: int) -> np.ndarray:
    return random_unitary(SplitMix64(seed))


def random_state(n: int, seed: int, normalize: bool = True) -> np.ndarray:
    """Complex Gaussian vector of 2^n amplitudes (complex128), unit norm."""
    rng = SplitMix64(seed)
    z = rng.normal(2 << n)
    psi = z[0::2] + 1j * z[1::2]
    if normalize:
        psi /= np.sqrt(np.vdot(psi, psi).real)
    return psi


def ansatz_hamiltonian(n: int, periodic: bool = False, hx: float = 0.5):
    """H = sum_{i} Z_i Z_{i+1} + hx * sum_i X_i as (coeff, x_mask, z_mask) terms.
    Open chain (n-1 ZZ terms) unless ``periodic``."""
    terms = []
    last = n if periodic else n - 1
    for i in range(last):
        j = (i + 1) % n
        terms.append((1.0, 0, (1 << i) | (1 << j)))
    for i in range(n):
        terms.append((hx, 1 << i, 0))
    return terms


def layer_count_gates(n: int, layers: int) -> int:
    """Gate count of ``random_circuit(n, layers)``."""
    return sum(n + len(brickwork_pairs(n, l)) for l in range(layers))
