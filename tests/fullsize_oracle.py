"""Oracle states for the full-size parity tests, computed on the host cores
while the rest of the GPU suite runs.

The oracle (plain complex128 Eq. 5 loops, OpenMP over the pairs) needs about
four minutes for the 30-qubit, 1,780-gate circuit and eight for the 64-circuit
uneven batch on 16 cores. A background thread starts at the end of collection
when a test marked ``oracle_fullsize`` is selected and a GPU is present; the
oracle's C calls release the GIL, so the GPU tests keep running meanwhile.
Tests take each finished state with ``take(key)`` (which waits for it)."""
from __future__ import annotations

import os
import threading
import time

from paper_2508_15545_gb300 import workloads as W

RANDOM30 = ("random30", 30, 40)  # key, qubits, layers (seed: workload 1)
UNEVEN_COUNT = 64


def uneven_spec():
    """(n, depth, seed) of the 64 uneven-batch circuits (workload 4)."""
    return W.uneven_batch(UNEVEN_COUNT, W.config_seed(4))


def jobs():
    out = [(("uneven", i), n, W.random_circuit(n, d, s)) for i, (n, d, s) in enumerate(uneven_spec())]
    key, n, layers = RANDOM30
    out.append((key, n, W.random_circuit(n, layers, W.config_seed(1))))
    return out


class FullSizeOracle:
    def __init__(self, job_list):
        self.jobs = job_list
        self.done = {}
        self.err = None
        self.threads = 0
        self.cv = threading.Condition()
        self.thread = threading.Thread(target=self._run, name="oracle-fullsize", daemon=True)
        self.thread.start()

    def _run(self):
        try:
            from oracle import oracle as O
            self.threads = O.set_threads(len(os.sched_getaffinity(0)))
            for key, n, gates in self.jobs:
                t0 = time.perf_counter()
                psi = O.run(n, gates)
                with self.cv:
                    self.done[key] = (psi, time.perf_counter() - t0)
                    self.cv.notify_all()
        except BaseException as e:  # noqa: BLE001 -- reported by take()
            with self.cv:
                self.err = e
                self.cv.notify_all()

    def take(self, key, timeout: float = 1500.0):
        """(oracle state, seconds it took); waits until it is computed."""
        with self.cv:
            ok = self.cv.wait_for(lambda: key in self.done or self.err is not None, timeout)
            if self.err is not None:
                raise RuntimeError("oracle thread failed: %r" % (self.err,))
            if not ok:
                raise TimeoutError("oracle state %r not ready after %.0f s" % (key, timeout))
            return self.done.pop(key)


_instance = None


def start():
    global _instance
    if _instance is None:
        _instance = FullSizeOracle(jobs())
    return _instance


def get():
    return _instance if _instance is not None else start()
