"""The OpenMP build of the oracle gives the same bits as the serial build.

The parallel loops split the index range of Eq. 5 (Sec. III-A) over threads;
every pair is still updated once with the same arithmetic, so the state may not
differ in a single bit. <Z_q> runs its independent sums on separate threads,
each in index order, so it is bit-identical too."""
import os

import numpy as np

from oracle import oracle as O
from paper_2508_15545_gb300 import workloads as W


def _run(L, n, gates):
    psi = np.zeros(1 << n, dtype=np.complex128)
    L.orc_basis(psi.ctypes.data, n, 0)
    arr = O.to_orc_gates(gates)
    assert L.orc_run(psi.ctypes.data, n, arr, len(gates)) == 0
    return psi


def test_openmp_and_serial_builds_bit_identical(tmp_path):
    serial = O.load(O.build_oracle(openmp=False, out=str(tmp_path / "liboracle_serial.so")))
    par = O.lib()
    threads = par.orc_set_threads(max(2, os.cpu_count() or 2))
    assert threads >= 2
    assert serial.orc_set_threads(8) == 1
    n = 20
    gates = W.random_circuit(n, 4, W.config_seed(0, 7)) + W.random_gate_list(n, 60, seed=31)
    a = _run(serial, n, gates)
    b = _run(par, n, gates)
    assert a.view(np.uint64).tobytes() == b.view(np.uint64).tobytes()
    za, zb = np.zeros(n), np.zeros(n)
    serial.orc_expect_z(a.ctypes.data, n, za.ctypes.data)
    par.orc_expect_z(b.ctypes.data, n, zb.ctypes.data)
    assert za.tobytes() == zb.tobytes()
    perm = np.array(np.random.RandomState(3).permutation(n), dtype=np.int32)
    pa, pb = np.empty_like(a), np.empty_like(b)
    serial.orc_permute(a.ctypes.data, pa.ctypes.data, n, perm.ctypes.data)
    par.orc_permute(b.ctypes.data, pb.ctypes.data, n, perm.ctypes.data)
    assert pa.tobytes() == pb.tobytes()
