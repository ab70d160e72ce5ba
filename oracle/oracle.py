"""Python face of the CPU oracle (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` leg may
import this module. It loads ``liboracle.so`` (plain C, complex128, built from
``qv_oracle.c`` by ``build_oracle()``) and shares no code with the CUDA path.

Gradients here are computed by re-simulation only: the exact parameter-shift
rule and central finite differences. Neither uses the adjoint method.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Iterable, List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_KIND = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "sdg": 5, "t": 6, "tdg": 7,
         "rx": 8, "ry": 9, "rz": 10, "p": 11, "u3": 12, "matrix": 13, "swap": 14}


class OrcGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32),
                ("target2", ctypes.c_int32), ("ctrl", ctypes.c_int32),
                ("theta", ctypes.c_double * 3), ("m", ctypes.c_double * 8)]


def build_oracle(force: bool = False, openmp: bool = True, out: str | None = None) -> str:
    """Compile qv_oracle.c with gcc (plain -O2, no -ffast-math) into
    liboracle.so, or into ``out``. ``openmp`` splits the pair loops over
    threads (same arithmetic per pair; the serial build gives the same bits)."""
    lib = out or _LIB
    if force or out or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared"] + (["-fopenmp"] if openmp else [])
        subprocess.check_call(cmd + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


_lib = None


def load(path: str):
    """Load an oracle library at ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    c128p = ctypes.c_void_p
    L.orc_gate_matrix.argtypes = [ctypes.POINTER(OrcGate), c128p]
    L.orc_gate_matrix.restype = ctypes.c_int
    L.orc_apply_1q.argtypes = [c128p, ctypes.c_int, ctypes.c_int, c128p]
    L.orc_apply_controlled.argtypes = [c128p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c128p]
    L.orc_apply_swap.argtypes = [c128p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.orc_run.argtypes = [c128p, ctypes.c_int, ctypes.POINTER(OrcGate), ctypes.c_int64]
    L.orc_run.restype = ctypes.c_int64
    L.orc_basis.argtypes = [c128p, ctypes.c_int, ctypes.c_uint64]
    L.orc_permute.argtypes = [c128p, c128p, ctypes.c_int, ctypes.c_void_p]
    L.orc_norm2.argtypes = [c128p, ctypes.c_int]
    L.orc_norm2.restype = ctypes.c_double
    L.orc_expect_z.argtypes = [c128p, ctypes.c_int, ctypes.c_void_p]
    L.orc_expect_pauli.argtypes = [c128p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
    L.orc_expect_pauli.restype = ctypes.c_double
    L.orc_apply_pauli_sum.argtypes = [c128p, c128p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_set_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build_oracle())
    return _lib


def set_threads(nthreads: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: keep the current number);
    returns the number in effect (1 for a serial build)."""
    return int(lib().orc_set_threads(int(nthreads)))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check_state(psi: np.ndarray) -> int:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("oracle states are contiguous complex128 arrays")
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


def to_orc_gates(gates: Sequence) -> ctypes.Array:
    arr = (OrcGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        o = arr[i]
        o.kind = _KIND[g.kind]
        o.target = g.target
        o.target2 = g.target2
        o.ctrl = g.ctrl
        for e in range(3):
            o.theta[e] = g.theta[e]
        if g.matrix is not None:
            for e, z in enumerate(g.matrix):
                o.m[2 * e] = complex(z).real
                o.m[2 * e + 1] = complex(z).imag
    return arr


# ----------------------------------------------------------------------------
# state construction and gate application
# ----------------------------------------------------------------------------
def basis(n: int, j: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().orc_basis(_ptr(psi), n, j)
    return psi


def gate_matrix(g) -> np.ndarray:
    U = np.zeros(4, dtype=np.complex128)
    arr = to_orc_gates([g])
    if lib().orc_gate_matrix(arr, _ptr(U)):
        raise ValueError("no matrix for gate kind %r" % (g.kind,))
    return U.reshape(2, 2)


def apply_1q(psi: np.ndarray, target: int, U) -> np.ndarray:
    """Eq. 5 in place on ``psi``; returns psi."""
    n = _check_state(psi)
    if not 0 <= target < n:
        raise ValueError("target out of range")
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(4))
    lib().orc_apply_1q(_ptr(psi), n, target, _ptr(Uc))
    return psi


def apply_controlled(psi: np.ndarray, ctrl: int, target: int, U) -> np.ndarray:
    n = _check_state(psi)
    if not (0 <= target < n and 0 <= ctrl < n and ctrl != target):
        raise ValueError("bad control/target")
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(4))
    lib().orc_apply_controlled(_ptr(psi), n, ctrl, target, _ptr(Uc))
    return psi


def apply_swap(psi: np.ndarray, a: int, b: int) -> np.ndarray:
    n = _check_state(psi)
    lib().orc_apply_swap(_ptr(psi), n, a, b)
    return psi


def run(n: int, gates: Sequence, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply ``gates`` in order to ``psi`` (default |0...0>), in place; returns psi."""
    if psi is None:
        psi = basis(n, 0)
    if _check_state(psi) != n:
        raise ValueError("state size does not match n")
    if len(gates) == 0:
        return psi
    arr = to_orc_gates(gates)
    bad = lib().orc_run(_ptr(psi), n, arr, len(gates))
    if bad:
        raise ValueError("bad gate at index %d: %r" % (bad - 1, gates[bad - 1]))
    return psi


def permute(psi: np.ndarray, perm: Sequence[int]) -> np.ndarray:
    """out[pi(i)] = psi[i] where bit q of i moves to bit perm[q]."""
    n = _check_state(psi)
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    if sorted(p.tolist()) != list(range(n)):
        raise ValueError("not a permutation")
    out = np.empty_like(psi)
    lib().orc_permute(_ptr(psi), _ptr(out), n, _ptr(p))
    return out


# ----------------------------------------------------------------------------
# reductions
# ----------------------------------------------------------------------------
def norm2(psi: np.ndarray) -> float:
    return lib().orc_norm2(_ptr(psi), _check_state(psi))


def expect_z(psi: np.ndarray) -> np.ndarray:
    n = _check_state(psi)
    out = np.zeros(n)
    lib().orc_expect_z(_ptr(psi), n, _ptr(out))
    return out


def expect_pauli(psi: np.ndarray, xmask: int, zmask: int) -> float:
    return lib().orc_expect_pauli(_ptr(psi), _check_state(psi), xmask, zmask)


def expect_terms(psi: np.ndarray, terms: Iterable[Tuple[float, int, int]]) -> float:
    """<psi|H|psi> for H = sum coeff * P(xmask, zmask)."""
    return float(sum(c * expect_pauli(psi, x, z) for c, x, z in terms))


def apply_pauli_sum(psi: np.ndarray, terms: Sequence[Tuple[float, int, int]]) -> np.ndarray:
    n = _check_state(psi)
    c = np.array([t[0] for t in terms], dtype=np.float64)
    x = np.array([t[1] for t in terms], dtype=np.uint64)
    z = np.array([t[2] for t in terms], dtype=np.uint64)
    out = np.empty_like(psi)
    lib().orc_apply_pauli_sum(_ptr(psi), _ptr(out), n, _ptr(c), _ptr(x), _ptr(z), len(terms))
    return out


def sample(psi: np.ndarray, u) -> np.ndarray:
    """Born-rule measurement in the computational basis by inverse CDF: for
    each uniform u in [0, 1), the smallest i with p_0 + ... + p_i > u * sum p,
    p_i = re_i^2 + im_i^2 (FP64). A target that rounds to the total takes the
    last outcome with nonzero probability."""
    p = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    cdf = np.cumsum(p)
    total = cdf[-1]
    idx = np.searchsorted(cdf, np.asarray(u, dtype=np.float64) * total, side="right")
    last = int(np.nonzero(p)[0][-1])
    return np.minimum(idx, last).astype(np.uint64)


# ----------------------------------------------------------------------------
# gradients by re-simulation
# ----------------------------------------------------------------------------
def energy(n: int, gates: Sequence, terms, psi0: np.ndarray | None = None) -> float:
    psi = run(n, gates, None if psi0 is None else psi0.copy())
    return expect_terms(psi, terms)


def _shifted(gates: Sequence, gi: int, slot: int, delta: float) -> List:
    g = gates[gi]
    th = list(g.theta)
    th[slot] += delta
    out = list(gates)
    out[gi] = g._replace(theta=tuple(th))
    return out


def _occurrences(gates: Sequence, nparams: int):
    occ = [[] for _ in range(nparams)]
    for gi, g in enumerate(gates):
        for slot, p in enumerate(g.param):
            if p >= 0:
                occ[p].append((gi, slot))
    return occ


_ROTATION_ANGLE = {"rx": (0,), "ry": (0,), "rz": (0,), "u3": (0,)}
_D1 = (math.sqrt(2.0) + 1.0) / (4.0 * math.sqrt(2.0))
_D2 = (math.sqrt(2.0) - 1.0) / (4.0 * math.sqrt(2.0))


def param_shift_grad(n: int, gates: Sequence, terms, nparams: int, psi0: np.ndarray | None = None) -> np.ndarray:
    """d<H>/d theta_p by parameter-shift rules, summed over every gate using p
    (circuit started from psi0, default |0...0>).

    Each angle enters the circuit as exp(-i theta G) for a fixed generator G.
    When the eigenvalues of G differ only by 0 or 1 -- any uncontrolled angle
    here (RX, RY, RZ, P, U3 up to a global phase), and a controlled P or the
    phi / lambda angles of a controlled U3, whose generator is a projector --
    E(theta) is a + b cos(theta) + c sin(theta) and
        dE = (E(theta + pi/2) - E(theta - pi/2)) / 2
    is exact. A controlled rotation angle (RX, RY, RZ, U3 theta with a control)
    has G = |1><1| (x) sigma/2 with eigenvalues {-1/2, 0, 1/2}: E then holds
    frequencies 1/2 and 1, and the four-term rule
        dE = d1 (E(+pi/2) - E(-pi/2)) - d2 (E(+3pi/2) - E(-3pi/2)),
        d1 = (sqrt 2 + 1) / (4 sqrt 2), d2 = (sqrt 2 - 1) / (4 sqrt 2)
    is exact (it reproduces d/dtheta of sin(w theta) for w = 1/2 and 1 and
    annihilates the cosines; Wierichs et al., "General parameter-shift rules
    for quantum gradients", Quantum 6, 677 (2022))."""
    g = np.zeros(nparams)
    for p, uses in enumerate(_occurrences(gates, nparams)):
        for gi, slot in uses:
            gt = gates[gi]
            E = lambda d: energy(n, _shifted(gates, gi, slot, d), terms, psi0)
            if gt.ctrl >= 0 and slot in _ROTATION_ANGLE.get(gt.kind, ()):
                g[p] += _D1 * (E(math.pi / 2) - E(-math.pi / 2)) - _D2 * (E(1.5 * math.pi) - E(-1.5 * math.pi))
            else:
                g[p] += 0.5 * (E(math.pi / 2) - E(-math.pi / 2))
    return g


def finite_diff_grad(n: int, gates: Sequence, terms, nparams: int, h: float = 1e-3,
                     psi0: np.ndarray | None = None) -> np.ndarray:
    """Central differences (E(theta_p + h) - E(theta_p - h)) / (2h), shifting
    every gate that uses parameter p together."""
    g = np.zeros(nparams)
    for p, uses in enumerate(_occurrences(gates, nparams)):
        if not uses:
            continue
        gp, gm = list(gates), list(gates)
        for gi, slot in uses:
            gp = _shifted(gp, gi, slot, h)
            gm = _shifted(gm, gi, slot, -h)
        g[p] = (energy(n, gp, terms, psi0) - energy(n, gm, terms, psi0)) / (2 * h)
    return g
