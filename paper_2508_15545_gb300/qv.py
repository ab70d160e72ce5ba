"""ctypes binding of libqv.so (include/qv.h). Function names match the C ABI;
this module only marshals arguments. Device memory and streams may come from
PyTorch (``StateVector`` wraps a torch tensor with ``qv_wrap``).

Importing raises if libqv.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqv.so")

QV_C64, QV_C128 = 0, 1
QV_OK, QV_ERR_ARG, QV_ERR_OOM, QV_ERR_CUDA, QV_ERR_TIMEOUT, QV_ERR_UNSUPPORTED = range(6)
QV_MODE_AUTO, QV_MODE_PLAIN, QV_MODE_FUSED = 0, 1, 2
QV_PLAN_NO_FUSION = 1
QV_PLAN_INTERPRET = 2
QV_PLAN_NO_PAIRS = 4
QV_PLAN_TENSOR = 8
QV_PLAN_AUTOTUNE = 16
QV_PLAN_HOST_IN_PLACE = 32
QV_ALLOC_HOST = 1
QV_SWEEP_AUTO, QV_SWEEP_PER_GATE, QV_SWEEP_TILES, QV_SWEEP_COMPILED = 0, 1, 2, 3
STATUS_NAMES = {0: "QV_OK", 1: "QV_ERR_ARG", 2: "QV_ERR_OOM", 3: "QV_ERR_CUDA",
                4: "QV_ERR_TIMEOUT", 5: "QV_ERR_UNSUPPORTED"}
KIND = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "sdg": 5, "t": 6, "tdg": 7,
        "rx": 8, "ry": 9, "rz": 10, "p": 11, "u3": 12, "matrix": 13, "swap": 14}


class QvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class qv_c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class qv_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32), ("target2", ctypes.c_int32),
                ("ctrl", ctypes.c_int32), ("param", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32),
                ("theta", ctypes.c_double * 3), ("u", qv_c128 * 4)]


class qv_plan_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_bits", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("window_bits", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class qv_tc_stage(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("nstages", ctypes.c_int32), ("tile_qubit", ctypes.c_int32 * 12),
                ("in_reg", ctypes.c_int32 * 4), ("in_thr", ctypes.c_int32 * 8),
                ("out_reg", ctypes.c_int32 * 4), ("out_thr", ctypes.c_int32 * 8),
                ("has_matrix", ctypes.c_int32), ("ext", ctypes.c_int32), ("m", (qv_c128 * 256) * 2)]


class qv_dist_step(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("global_bit", ctypes.c_int32), ("peer", ctypes.c_int32),
                ("send_upper", ctypes.c_int32), ("gate_begin", ctypes.c_uint64), ("gate_end", ctypes.c_uint64)]


QV_DIST_LOCAL, QV_DIST_EXCHANGE = 0, 1


class qv_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


KERNEL_CLASSES = ("basis", "pair", "diag", "swap", "fused", "reduce", "pauli", "adjoint", "batch", "verify")


class qv_pauli_term(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64)]


_H = ctypes.c_void_p  # qv_state*


class qv_batch_item(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("gates", ctypes.POINTER(qv_gate)), ("ngates", ctypes.c_size_t)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libqv.so not built (run paper_2508_15545_gb300.build.build()); "
                          "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    P = ctypes.c_void_p
    sig = {
        "qv_create": [ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(_H)],
        "qv_create_ex": [ctypes.c_int, ctypes.c_int, P, ctypes.c_int32, ctypes.POINTER(_H)],
        "qv_wrap": [P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(_H)],
        "qv_destroy": [_H],
        "qv_set_stream": [_H, P],
        "qv_info": [_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(P)],
        "qv_set_basis": [_H, ctypes.c_uint64],
        "qv_get_state": [_H, P, ctypes.c_size_t],
        "qv_set_state": [_H, P, ctypes.c_size_t],
        "qv_apply_1q": [_H, ctypes.c_int, ctypes.POINTER(qv_c128)],
        "qv_apply_controlled": [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_c128)],
        "qv_apply_circuit": [_H, ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(qv_plan_opts)],
        "qv_permute_qubits": [_H, ctypes.POINTER(ctypes.c_int32)],
        "qv_plan_info": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                         ctypes.POINTER(qv_plan_opts), ctypes.POINTER(ctypes.c_int32)],
        "qv_plan_cost": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                         ctypes.POINTER(qv_plan_opts), ctypes.POINTER(ctypes.c_double)],
        "qv_plan_source": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                           ctypes.POINTER(qv_plan_opts), ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t,
                           ctypes.POINTER(ctypes.c_size_t)],
        "qv_plan_compile": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                            ctypes.POINTER(qv_plan_opts), ctypes.POINTER(ctypes.c_int64)],
        "qv_dist_plan": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                         ctypes.c_int32, ctypes.POINTER(qv_dist_step), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(ctypes.c_int32)],
        "qv_plan_tc_stage": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qv_gate), ctypes.c_size_t,
                             ctypes.POINTER(qv_plan_opts), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(qv_tc_stage)],
        "qv_norm2": [_H, ctypes.POINTER(ctypes.c_double)],
        "qv_expect_z": [_H, P, P, ctypes.POINTER(ctypes.c_double)],
        "qv_expect_pauli": [_H, ctypes.POINTER(qv_pauli_term), ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)],
        "qv_zsums_noalloc": [P, ctypes.c_int, ctypes.c_int, P, P],
        "qv_apply_pauli": [_H, ctypes.POINTER(qv_pauli_term), ctypes.c_size_t, _H],
        "qv_adjoint_grad": [_H, ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(qv_pauli_term),
                            ctypes.c_size_t, ctypes.c_size_t, P, ctypes.POINTER(ctypes.c_double)],
        "qv_adjoint_grad_ex": [_H, ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(qv_pauli_term),
                            ctypes.c_size_t, ctypes.c_size_t, P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32],
        "qv_autotune": [_H, ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(qv_plan_opts),
                        ctypes.POINTER(ctypes.c_int32)],
        "qv_autotune_ex": [_H, ctypes.POINTER(qv_gate), ctypes.c_size_t, ctypes.POINTER(qv_plan_opts),
                           ctypes.POINTER(ctypes.c_int32)],
        "qv_batch_create": [ctypes.POINTER(qv_batch_item), ctypes.c_size_t, ctypes.POINTER(qv_pauli_term),
                            ctypes.c_size_t, ctypes.POINTER(qv_plan_opts), ctypes.POINTER(ctypes.c_void_p)],
        "qv_batch_run": [ctypes.c_void_p, P],
        "qv_batch_destroy": [ctypes.c_void_p],
        "qv_apply_batch": [ctypes.POINTER(qv_batch_item), ctypes.c_size_t, ctypes.POINTER(qv_pauli_term),
                           ctypes.c_size_t, ctypes.POINTER(qv_plan_opts), P],
        "qv_verify_qft": [_H, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)],
        "qv_sync": [_H],
        "qv_default_tile_bits": [ctypes.c_int, ctypes.c_int, ctypes.c_int32],
        "qv_sample": [_H, P, ctypes.c_size_t, P],
        "qv_get_amplitudes": [_H, P, ctypes.c_size_t, P],
        "qv_wait_selftest": [_H, ctypes.c_uint32],
        "qv_distance": [_H, _H, ctypes.POINTER(ctypes.c_double)],
        "qv_profile": [_H, ctypes.c_int],
        "qv_profile_read": [_H, ctypes.POINTER(qv_kernel_stat), ctypes.c_int],
        "qv_transfer_bytes": [_H, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.qv_batch_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    L.qv_batch_info.restype = ctypes.c_int32
    L.qv_last_error.argtypes = []
    L.qv_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(status: int):
    if status != QV_OK:
        raise QvError(status, lib.qv_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    """Accepts None, an int (cudaStream_t) or a torch.cuda.Stream."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def c128_array(U) -> ctypes.Array:
    U = np.asarray(U, dtype=np.complex128).reshape(4)
    arr = (qv_c128 * 4)()
    for e in range(4):
        arr[e].re = U[e].real
        arr[e].im = U[e].imag
    return arr


def gates_to_c(gates: Sequence) -> ctypes.Array:
    """workloads.Gate records -> qv_gate[]."""
    arr = (qv_gate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        o = arr[i]
        o.kind = KIND[g.kind]
        o.target = g.target
        o.target2 = g.target2
        o.ctrl = g.ctrl
        for e in range(3):
            o.param[e] = g.param[e]
            o.theta[e] = g.theta[e]
        if g.matrix is not None:
            for e, z in enumerate(g.matrix):
                o.u[e].re = complex(z).real
                o.u[e].im = complex(z).imag
    return arr


def terms_to_c(terms: Sequence[Tuple[float, int, int]]) -> ctypes.Array:
    arr = (qv_pauli_term * max(1, len(terms)))()
    for i, (c, x, z) in enumerate(terms):
        arr[i].coeff = c
        arr[i].xmask = x
        arr[i].zmask = z
    return arr


def plan_opts(mode: int = QV_MODE_AUTO, tile_bits: int = 0, flags: int = 0) -> qv_plan_opts:
    o = qv_plan_opts()
    o.mode = mode
    o.tile_bits = tile_bits
    o.flags = flags
    return o


# ----------------------------------------------------------------------------
# C ABI, one Python function per entry point
# ----------------------------------------------------------------------------
def qv_create(n: int, dtype: int = QV_C64, stream=None, flags: int = 0) -> int:
    """New |0...0> state; flags = QV_ALLOC_HOST keeps it in mapped host memory."""
    h = _H()
    if flags:
        _check(lib.qv_create_ex(n, dtype, _stream_ptr(stream), flags, ctypes.byref(h)))
    else:
        _check(lib.qv_create(n, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qv_wrap(dev_ptr: int, n: int, dtype: int = QV_C64, stream=None) -> int:
    h = _H()
    _check(lib.qv_wrap(dev_ptr, n, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qv_destroy(h: int):
    _check(lib.qv_destroy(h))


def qv_set_stream(h: int, stream):
    _check(lib.qv_set_stream(h, _stream_ptr(stream)))


def qv_info(h: int):
    n, dt, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(lib.qv_info(h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p)))
    return n.value, dt.value, p.value


def qv_set_basis(h: int, j: int):
    _check(lib.qv_set_basis(h, j))


def qv_get_state(h: int) -> np.ndarray:
    n, dt, _ = qv_info(h)
    out = np.empty(1 << n, dtype=np.complex64 if dt == QV_C64 else np.complex128)
    _check(lib.qv_get_state(h, out.ctypes.data, out.nbytes))
    return out


def qv_set_state(h: int, psi: np.ndarray):
    n, dt, _ = qv_info(h)
    a = np.ascontiguousarray(psi, dtype=np.complex64 if dt == QV_C64 else np.complex128)
    _check(lib.qv_set_state(h, a.ctypes.data, a.nbytes))


def qv_apply_1q(h: int, target: int, U):
    _check(lib.qv_apply_1q(h, target, c128_array(U)))


def qv_apply_controlled(h: int, ctrl: int, target: int, U):
    _check(lib.qv_apply_controlled(h, ctrl, target, c128_array(U)))


def qv_apply_circuit(h: int, gates, mode: int = QV_MODE_AUTO, tile_bits: int = 0, flags: int = 0):
    """``gates``: a sequence of workloads.Gate or a prebuilt qv_gate array
    (``gates_to_c``) with its length as ``(array, count)``."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    opts = plan_opts(mode, tile_bits, flags)
    _check(lib.qv_apply_circuit(h, arr, ng, ctypes.byref(opts)))


def qv_default_tile_bits(n: int, dtype: int = QV_C64, flags: int = 0) -> int:
    """Tile size (log2 amplitudes) fused mode uses when none is given."""
    return int(lib.qv_default_tile_bits(n, dtype, flags))


def qv_plan_info(n: int, dtype: int, gates, tile_bits: int = 0, flags: int = 0) -> dict:
    """Fused-mode plan of ``gates`` (host only): passes, stages, transposes, ops."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    out = (ctypes.c_int32 * 4)()
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
    _check(lib.qv_plan_info(n, dtype, arr, ng, ctypes.byref(opts), out))
    return {"passes": out[0], "stages": out[1], "transposes": out[2], "ops": out[3]}


def qv_plan_cost(n: int, dtype: int, gates, tile_bits: int = 0, flags: int = 0) -> dict:
    """Algorithmic cost of the fused plan (host only): HBM bytes and floating-point operations."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    out = (ctypes.c_double * 2)()
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
    _check(lib.qv_plan_cost(n, dtype, arr, ng, ctypes.byref(opts), out))
    return {"bytes": out[0], "flops": out[1]}


def qv_plan_source(n: int, dtype: int, gates, pass_index: int, tile_bits: int = 0, flags: int = 0) -> str:
    """CUDA source of compiled fused pass ``pass_index`` (host only)."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
    ln = ctypes.c_size_t()
    _check(lib.qv_plan_source(n, dtype, arr, ng, ctypes.byref(opts), pass_index, None, 0, ctypes.byref(ln)))
    buf = ctypes.create_string_buffer(ln.value + 1)
    _check(lib.qv_plan_source(n, dtype, arr, ng, ctypes.byref(opts), pass_index, buf, ln.value + 1,
                              ctypes.byref(ln)))
    return buf.value.decode()


def qv_plan_compile(n: int, dtype: int, gates, tile_bits: int = 0, flags: int = 0) -> dict:
    """Compiles every pass of the fused plan with NVRTC (host only, no GPU)."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
    out = (ctypes.c_int64 * 4)()
    _check(lib.qv_plan_compile(n, dtype, arr, ng, ctypes.byref(opts), out))
    return {"passes": int(out[0]), "source_bytes": int(out[1]), "max_registers": int(out[2]),
            "spilling_passes": int(out[3])}


def qv_plan_tc_stage(n: int, gates, pass_index: int, stage: int, tile_bits: int = 0, flags: int = 0) -> dict:
    """Stage ``stage`` of pass ``pass_index`` of the tensor-core plan (host only):
    layouts (tile positions of register and thread bits), the physical qubit of
    every tile position, and the stage's 16x16 matrices."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags | QV_PLAN_TENSOR)
    o = qv_tc_stage()
    _check(lib.qv_plan_tc_stage(n, QV_C64, arr, ng, ctypes.byref(opts), pass_index, stage, ctypes.byref(o)))
    k = int(o.k)
    m = np.array([[complex(o.m[v][e].re, o.m[v][e].im) for e in range(256)] for v in range(2)]).reshape(2, 16, 16)
    return {"k": k, "nstages": int(o.nstages), "tile_qubit": list(o.tile_qubit)[:k],
            "in_reg": list(o.in_reg), "in_thr": list(o.in_thr)[:k - 4],
            "out_reg": list(o.out_reg), "out_thr": list(o.out_thr)[:k - 4],
            "has_matrix": bool(o.has_matrix), "ext": int(o.ext), "m": m}


QV_DIST_RESTORE = 1


def qv_dist_plan(n: int, global_bits: int, rank: int, gates, restore: bool = False):
    """Schedule of ``gates`` on ``rank`` of 2^global_bits ranks (Eq. 9; host
    only): (steps, local gate array, final_perm). steps: list of dicts with
    kind 'local' (begin, end into the local gate array) or 'exchange' (peer,
    global_bit, send_upper)."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    ns, nl = ctypes.c_size_t(), ctypes.c_size_t()
    fl = QV_DIST_RESTORE if restore else 0
    _check(lib.qv_dist_plan(n, global_bits, rank, arr, ng, fl, None, 0, ctypes.byref(ns), None, 0, ctypes.byref(nl),
                            None))
    st = (qv_dist_step * max(1, ns.value))()
    lg = (qv_gate * max(1, nl.value))()
    perm = (ctypes.c_int32 * n)()
    _check(lib.qv_dist_plan(n, global_bits, rank, arr, ng, fl, st, ns.value, ctypes.byref(ns), lg, nl.value,
                            ctypes.byref(nl), perm))
    steps = []
    for k in range(ns.value):
        x = st[k]
        if x.kind == QV_DIST_LOCAL:
            steps.append({"kind": "local", "begin": int(x.gate_begin), "end": int(x.gate_end)})
        else:
            steps.append({"kind": "exchange", "peer": int(x.peer), "global_bit": int(x.global_bit),
                          "send_upper": bool(x.send_upper)})
    return steps, (lg, nl.value), list(perm)


def qv_permute_qubits(h: int, perm: Sequence[int]):
    arr = (ctypes.c_int32 * max(1, len(perm)))(*perm)
    _check(lib.qv_permute_qubits(h, arr))


def qv_norm2(h: int) -> float:
    out = ctypes.c_double()
    _check(lib.qv_norm2(h, ctypes.byref(out)))
    return out.value


def qv_expect_z(h: int, weights: Optional[Sequence[float]] = None):
    """Returns (per-qubit <Z_q> as numpy array, weighted total)."""
    n, _, _ = qv_info(h)
    per = np.zeros(n)
    tot = ctypes.c_double()
    w = None
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.size != n:
            raise ValueError("weights must have n entries")
    _check(lib.qv_expect_z(h, None if w is None else w.ctypes.data, per.ctypes.data, ctypes.byref(tot)))
    return per, tot.value


def qv_expect_pauli(h: int, terms: Sequence[Tuple[float, int, int]]) -> float:
    out = ctypes.c_double()
    _check(lib.qv_expect_pauli(h, terms_to_c(terms), len(terms), ctypes.byref(out)))
    return out.value


def qv_apply_pauli(h: int, terms, out_h: int):
    """out_h <- H |psi_h> (same n, dtype and stream)."""
    _check(lib.qv_apply_pauli(h, terms_to_c(terms), len(terms), out_h))


def qv_adjoint_grad(h: int, gates, terms, nparams: int, sweep_mode: int = QV_SWEEP_AUTO):
    """Adjoint-method gradient of <H> over the circuit ``gates`` applied to the
    handle's current state. Returns (grad as numpy array, <H>). ``sweep_mode``
    is one of QV_SWEEP_* (per gate, shared-memory tiles, compiled passes)."""
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        arr, ng = gates
    else:
        arr, ng = gates_to_c(gates), len(gates)
    grad = np.zeros(max(1, nparams))
    e = ctypes.c_double()
    _check(lib.qv_adjoint_grad_ex(h, arr, ng, terms_to_c(terms), len(terms), nparams, grad.ctypes.data,
                                  ctypes.byref(e), sweep_mode))
    return grad[:nparams], e.value


def qv_zsums_noalloc(dev_amp: int, n: int, dtype: int, stream, dev_out: int):
    """Allocation-free Z sums into the caller's device buffer of n + 1 doubles
    (see include/qv.h); asynchronous on ``stream``."""
    _check(lib.qv_zsums_noalloc(dev_amp, n, dtype, _stream_ptr(stream), dev_out))


def qv_autotune(h: int, gates, flags: int = 0) -> int:
    """Times the fused path for every tile size on this circuit, remembers the
    fastest for (n, dtype, engine) and returns it. Leaves the state at |0...0>."""
    arr, ng = _gate_array(gates)
    opts = plan_opts(QV_MODE_FUSED, 0, flags)
    best = ctypes.c_int32()
    _check(lib.qv_autotune(h, arr, ng, ctypes.byref(opts), ctypes.byref(best)))
    return best.value


def qv_autotune_ex(h: int, gates, flags: int = 0):
    """Like qv_autotune, also over the schedule variants; returns (tile bits, plan flags)."""
    arr, ng = _gate_array(gates)
    opts = plan_opts(QV_MODE_FUSED, 0, flags)
    out = (ctypes.c_int32 * 2)()
    _check(lib.qv_autotune_ex(h, arr, ng, ctypes.byref(opts), out))
    return int(out[0]), int(out[1])


def qv_batch_info(b) -> list:
    """Per launch group of a batch: dict of tile_bits, circuits, qubits, compiled, l2_group, chunk_tiles."""
    n = lib.qv_batch_info(b, None, 0)
    if n < 0:
        raise QvError(QV_ERR_ARG, "bad batch")
    out = (ctypes.c_int32 * max(1, 6 * n))()
    lib.qv_batch_info(b, out, n)
    keys = ("tile_bits", "circuits", "qubits", "compiled", "l2_group", "chunk_tiles")
    return [dict(zip(keys, [int(out[6 * g + i]) for i in range(6)])) for g in range(n)]


def qv_apply_batch(items, terms=None, tile_bits: int = 0, flags: int = 0) -> np.ndarray:
    """One-shot batch (qv_apply_batch): runs every (state, circuit) pair from
    |0...0> and returns <H> per state (zeros without terms)."""
    count = len(items)
    arrs = [_gate_array(g) for _, g in items]
    c_items = (qv_batch_item * max(1, count))()
    for k, ((h, _), (arr, ng)) in enumerate(zip(items, arrs)):
        c_items[k].state = h
        c_items[k].gates = ctypes.cast(arr, ctypes.POINTER(qv_gate))
        c_items[k].ngates = ng
    terms = list(terms or [])
    opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
    out = np.zeros(max(1, count))
    _check(lib.qv_apply_batch(c_items, count, terms_to_c(terms), len(terms), ctypes.byref(opts),
                              out.ctypes.data if terms else None))
    return out[:count]


class Batch:
    """qv_batch_create / qv_batch_run / qv_batch_destroy: many (state, circuit)
    pairs in one graph-captured persistent launch, plus <H> per state."""

    def __init__(self, items, terms=None, tile_bits: int = 0, flags: int = 0):
        self.count = len(items)
        arrs = [_gate_array(g) for _, g in items]
        c_items = (qv_batch_item * self.count)()
        for k, ((h, _), (arr, ng)) in enumerate(zip(items, arrs)):
            c_items[k].state = h
            c_items[k].gates = ctypes.cast(arr, ctypes.POINTER(qv_gate))
            c_items[k].ngates = ng
        terms = list(terms or [])
        opts = plan_opts(QV_MODE_FUSED, tile_bits, flags)
        b = ctypes.c_void_p()
        _check(lib.qv_batch_create(c_items, self.count, terms_to_c(terms), len(terms), ctypes.byref(opts),
                                   ctypes.byref(b)))
        self.b = b.value
        self.has_h = len(terms) > 0

    def run(self) -> np.ndarray:
        out = np.zeros(self.count)
        _check(lib.qv_batch_run(self.b, out.ctypes.data if self.has_h else None))
        return out

    def info(self) -> list:
        return qv_batch_info(self.b)

    def close(self):
        if self.b:
            _check(lib.qv_batch_destroy(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gate_array(gates):
    if isinstance(gates, tuple) and len(gates) == 2 and isinstance(gates[1], int):
        return gates
    return gates_to_c(gates), len(gates)


def qv_verify_qft(h: int, j: int) -> float:
    """||psi - QFT|j>||_2 from the closed form, computed on the GPU."""
    d = ctypes.c_double()
    _check(lib.qv_verify_qft(h, j, ctypes.byref(d)))
    return d.value


def qv_sample(h: int, u) -> np.ndarray:
    """Outcomes for the uniforms u in [0, 1) (inverse-CDF sampling of |a|^2)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(max(1, u.size), dtype=np.uint64)
    _check(lib.qv_sample(h, u.ctypes.data, u.size, out.ctypes.data))
    return out[:u.size]


def qv_get_amplitudes(h: int, idx) -> np.ndarray:
    """Amplitudes at the given indices (complex64 or complex128 as the state)."""
    _, dt, _ = qv_info(h)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros(max(1, idx.size), dtype=np.complex64 if dt == QV_C64 else np.complex128)
    _check(lib.qv_get_amplitudes(h, idx.ctypes.data, idx.size, out.ctypes.data))
    return out[:idx.size]


def qv_sync(h: int):
    _check(lib.qv_sync(h))


def qv_wait_selftest(h: int, limit: int):
    """Runs the bounded device wait into its timeout; raises QvError (QV_ERR_TIMEOUT)."""
    _check(lib.qv_wait_selftest(h, limit))


def qv_distance(a: int, b: int) -> float:
    """||psi_a - psi_b||_2 (FP64), any mix of dtypes."""
    d = ctypes.c_double()
    _check(lib.qv_distance(a, b, ctypes.byref(d)))
    return d.value


def qv_profile(h: int, timing: bool = False):
    _check(lib.qv_profile(h, 1 if timing else 0))


def qv_profile_read(h: int) -> dict:
    """{class name: (launches, device ms, algorithmic bytes)}"""
    arr = (qv_kernel_stat * len(KERNEL_CLASSES))()
    _check(lib.qv_profile_read(h, arr, len(KERNEL_CLASSES)))
    return {name: (int(arr[k].launches), float(arr[k].ms), float(arr[k].bytes))
            for k, name in enumerate(KERNEL_CLASSES)}


def qv_transfer_bytes(h: int):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.qv_transfer_bytes(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def qv_last_error() -> str:
    return lib.qv_last_error().decode(errors="replace")


# ----------------------------------------------------------------------------
# torch-owned state
# ----------------------------------------------------------------------------
class StateVector:
    """A 2^n state held in a torch CUDA tensor and driven through the C ABI on
    torch's current stream (or ``stream``)."""

    def __init__(self, n: int, dtype: int = QV_C64, stream=None, basis: int = 0):
        import torch
        self.n = n
        self.dtype = dtype
        tdt = torch.complex64 if dtype == QV_C64 else torch.complex128
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        self.h = qv_wrap(self.tensor.data_ptr(), n, dtype, self.stream)
        qv_set_basis(self.h, basis)

    def close(self):
        if self.h:
            qv_destroy(self.h)
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

    def apply(self, gates, mode: int = QV_MODE_AUTO, tile_bits: int = 0):
        qv_apply_circuit(self.h, gates, mode, tile_bits)
        return self

    def numpy(self) -> np.ndarray:
        return qv_get_state(self.h)

    def expect_z(self, weights=None):
        return qv_expect_z(self.h, weights)

    def expect_pauli(self, terms) -> float:
        return qv_expect_pauli(self.h, terms)

    def norm2(self) -> float:
        return qv_norm2(self.h)
