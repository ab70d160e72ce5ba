"""States in host memory staged through device windows (the sliding window of
Sec. III-B, Eq. 6, with HBM as the fast memory): the whole state in one window,
or chunks of it streamed through two windows with half-chunk exchanges (the
split schedule of Sec. III-D, Eq. 9); against the oracle."""
import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run_host(qv, n, gates, psi, window_bits=0, flags=0, dtype=0):
    h = qv.qv_create(n, dtype, flags=qv.QV_ALLOC_HOST)
    try:
        qv.qv_set_state(h, psi)
        qv.qv_profile(h, timing=False)          # transfer counters from here on
        opts = qv.plan_opts(qv.QV_MODE_FUSED, 0, flags)
        opts.window_bits = window_bits
        import ctypes
        arr = qv.gates_to_c(gates)
        qv._check(qv.lib.qv_apply_circuit(h, arr, len(gates), ctypes.byref(opts)))
        qv.qv_sync(h)
        moved = qv.qv_transfer_bytes(h)
        return qv.qv_get_state(h), moved
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,wb", [(16, 16), (16, 14), (18, 15), (20, 18)])
def test_host_state_through_windows(qvlib, orc, cuda, n, wb, dtype):
    """Every gate kind (controls on chunk qubits, SWAPs, diagonals), a random
    circuit and a QFT: one window (wb = n) or 2^(n - wb) chunks."""
    qv = qvlib
    gates = W.random_gate_list(n, 120, seed=300 + n + wb, ctrl_prob=0.4) + \
        W.random_circuit(n, 4, W.config_seed(0, n)) + W.qft_circuit(n)
    psi = W.random_state(n, 7 + n)
    got, _ = run_host(qv, n, gates, psi, wb, dtype=dtype)
    want = orc.run(n, gates, psi.copy())
    assert np.linalg.norm(got.astype(np.complex128) - want) <= (1e-5 if dtype == 0 else 1e-12)


def test_host_state_window_traffic_and_in_place(qvlib, orc, cuda):
    """One window: the state crosses the host link once each way per call; in
    place (QV_PLAN_HOST_IN_PLACE) every pass reads and writes it there; both
    give the oracle's state."""
    qv = qvlib
    n = 18
    gates = W.random_circuit(n, 10, W.config_seed(0, 18))
    psi = W.random_state(n, 3)
    want = orc.run(n, gates, psi.copy())
    got, (h2d, d2h) = run_host(qv, n, gates, psi, n)
    assert np.linalg.norm(got.astype(np.complex128) - want) <= 1e-5
    state = 8 << n
    assert h2d - state < 1 << 16 and d2h == state    # the state in once (+ gate coefficients), out once
    got2, _ = run_host(qv, n, gates, psi, 0, qv.QV_PLAN_HOST_IN_PLACE)
    assert np.linalg.norm(got2.astype(np.complex128) - want) <= 1e-5


def test_window_bits_checked(qvlib, cuda):
    qv = qvlib
    import ctypes
    h = qv.qv_create(14, 0, flags=qv.QV_ALLOC_HOST)
    try:
        for wb in (9, 15):
            opts = qv.plan_opts(qv.QV_MODE_FUSED, 0, 0)
            opts.window_bits = wb
            arr = qv.gates_to_c(W.random_circuit(14, 1, 1))
            st = qv.lib.qv_apply_circuit(h, arr, 14, ctypes.byref(opts))
            assert st == qv.QV_ERR_ARG
    finally:
        qv.qv_destroy(h)
