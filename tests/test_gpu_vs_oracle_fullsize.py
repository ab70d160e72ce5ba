"""Full-size parity against the FP64 oracle.

The two workloads whose sizes the other tests only sample, compared element by
element with the oracle's complex128 state (Eq. 3 gate by gate with the
pairing rule of Eq. 5; the method reaches that state exactly up to rounding):

* the 30-qubit, 40-layer, 1,780-gate random circuit the bench times, in the
  bench's launch configuration (fused passes, default tile size), as a
  complex64 state (||dpsi||_2 <= 1e-5) and as a complex128 state (<= 1e-12);
* every member of the 64-circuit uneven batch (16..28 qubits, depth 10..60)
  run in one persistent launch, complex64, ||dpsi||_2 <= 1e-5 each.

The oracle states come from a background thread started at the end of
collection (tests/fullsize_oracle.py), so the host cores compute them while
the other GPU tests run."""
import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from tests import fullsize_oracle as F

pytestmark = [pytest.mark.gpu, pytest.mark.oracle_fullsize]


def l2_distance(got: np.ndarray, ref: np.ndarray, chunk: int = 1 << 24) -> float:
    """||got - ref||_2 in FP64, in chunks (no state-sized temporaries)."""
    assert got.shape == ref.shape
    acc = 0.0
    for i in range(0, got.size, chunk):
        d = got[i:i + chunk].astype(np.complex128) - ref[i:i + chunk]
        acc += float(np.vdot(d, d).real)
    return acc ** 0.5


def test_uneven_batch_64_circuits_vs_oracle(qvlib, cuda, fullsize_oracle):
    """Every member of the uneven batch (one persistent launch per tile size)
    against the oracle, at the complex64 tolerance."""
    qv = qvlib
    spec = F.uneven_spec()
    circuits = [W.random_circuit(n, d, seed) for n, d, seed in spec]
    states = [qv.qv_create(n, qv.QV_C64) for n, _, _ in spec]
    try:
        b = qv.Batch(list(zip(states, circuits)))
        b.run()
        worst = 0.0
        for i, ((n, d, _), h) in enumerate(zip(spec, states)):
            got = qv.qv_get_state(h)
            ref, _ = fullsize_oracle.take(("uneven", i))
            err = l2_distance(got, ref)
            del got, ref
            worst = max(worst, err)
            assert err <= 1e-5, (i, n, d, err)
        b.close()
        print("uneven batch: worst ||dpsi||_2 = %.3e over %d circuits" % (worst, len(spec)))
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_random_circuit_30_qubits_vs_oracle(qvlib, cuda, fullsize_oracle):
    """The bench circuit at full size: fused complex64 and complex128 states
    against the oracle's complex128 state."""
    qv = qvlib
    torch = cuda
    key, n, layers = F.RANDOM30
    gates = W.random_circuit(n, layers, W.config_seed(1))
    assert len(gates) == 1780
    free, _ = torch.cuda.mem_get_info()
    if free < (24 << n) + (4 << 30):
        pytest.skip("needs 28 GiB of free device memory")
    h = qv.qv_create(n, qv.QV_C64)
    try:
        qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_FUSED)
        got64 = qv.qv_get_state(h)
    finally:
        qv.qv_destroy(h)
    h = qv.qv_create(n, qv.QV_C128)
    try:
        qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_FUSED)
        got128 = qv.qv_get_state(h)
    finally:
        qv.qv_destroy(h)
    ref, secs = fullsize_oracle.take(key)
    e64 = l2_distance(got64, ref)
    del got64
    e128 = l2_distance(got128, ref)
    print("30 qubits, 1780 gates: ||dpsi||_2 complex64 %.3e, complex128 %.3e (oracle %.0f s on %d threads)"
          % (e64, e128, secs, fullsize_oracle.threads))
    assert e64 <= 1e-5
    assert e128 <= 1e-12
