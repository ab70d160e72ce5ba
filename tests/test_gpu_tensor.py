"""Parity of the tensor-core fused passes (QV_PLAN_TENSOR: one 16x16 complex
matrix per stage applied with tcgen05 in split TF32) against the oracle, through
the C ABI. Tolerance: ||dpsi||_2 <= 1e-5 for complex64 (depth <= 200)."""
import math

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dist(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b))


def run_tc(qv, n, gates, psi=None, basis=0, tile_bits=11, host=False):
    h = qv.qv_create(n, qv.QV_C64, flags=qv.QV_ALLOC_HOST if host else 0)
    try:
        if psi is not None:
            qv.qv_set_state(h, psi)
        else:
            qv.qv_set_basis(h, basis)
        qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_FUSED, tile_bits=tile_bits, flags=qv.QV_PLAN_TENSOR)
        qv.qv_sync(h)
        return qv.qv_get_state(h)
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("k", [11, 12])
@pytest.mark.parametrize("n", [11, 12, 13, 16, 19])
def test_tensor_random_gate_kinds(qvlib, orc, cuda, n, k):
    """Every gate kind, random controls inside and outside the tile, SWAPs;
    n = k is a single tile (no tile index bits)."""
    if k > n:
        pytest.skip("tile larger than the state")
    qv = qvlib
    gates = W.random_gate_list(n, 180, seed=5000 + 100 * n + k, ctrl_prob=0.4)
    psi = W.random_state(n, 17 * n + k)
    got = run_tc(qv, n, gates, psi=psi, tile_bits=k)
    assert dist(got, orc.run(n, gates, psi.copy())) <= 1e-5


@pytest.mark.parametrize("k", [11, 12])
def test_tensor_random_circuit(qvlib, orc, cuda, k):
    qv = qvlib
    for n, layers in ((16, 20), (21, 12)):
        gates = W.random_circuit(n, layers, W.config_seed(0, n))
        got = run_tc(qv, n, gates, tile_bits=k)
        assert dist(got, orc.run(n, gates)) <= 1e-5, n


@pytest.mark.parametrize("n", [12, 15])
def test_tensor_qft_closed_form(qvlib, cuda, n):
    """QFT with its final SWAPs (relabels) against e^{2 pi i j k / 2^n} / 2^{n/2}."""
    qv = qvlib
    N = 1 << n
    gates = W.qft_circuit(n)
    k = np.arange(N)
    for j in (1, N - 1, (3 * N) // 7):
        want = np.exp(2j * np.pi * ((j * k) % N) / N) / math.sqrt(N)
        for tb in (11, 12):
            assert dist(run_tc(qv, n, gates, basis=j, tile_bits=tb), want) <= 1e-5, (j, tb)


def test_tensor_ansatz_and_diagonals(qvlib, orc, cuda):
    """RY, RZ and CZ rings (diagonal gates with controls anywhere)."""
    qv = qvlib
    n = 14
    gates, _ = W.ansatz_circuit(n, 6, W.config_seed(2, 3))
    for tb in (11, 12):
        assert dist(run_tc(qv, n, gates, tile_bits=tb), orc.run(n, gates)) <= 1e-5


def test_tensor_matches_fp32_passes_24q(qvlib, orc, cuda):
    """24 qubits, 30 layers: the tensor-core passes, the FP32 compiled passes and
    the oracle agree; the norm stays 1."""
    qv = qvlib
    n = 24
    gates = W.random_circuit(n, 30, W.config_seed(0, 24))
    want = orc.run(n, gates)
    h = qv.qv_create(n, qv.QV_C64)
    try:
        for tb in (11, 12):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_FUSED, tile_bits=tb, flags=qv.QV_PLAN_TENSOR)
            qv.qv_sync(h)
            assert abs(qv.qv_norm2(h) - 1.0) <= 1e-5
            assert dist(qv.qv_get_state(h), want) <= 1e-5, tb
    finally:
        qv.qv_destroy(h)


def test_tensor_host_memory_state(qvlib, orc, cuda):
    qv = qvlib
    n = 17
    gates = W.random_gate_list(n, 120, seed=99, ctrl_prob=0.3)
    psi = W.random_state(n, 5)
    got = run_tc(qv, n, gates, psi=psi, tile_bits=12, host=True)
    assert dist(got, orc.run(n, gates, psi.copy())) <= 1e-5


def test_tensor_new_angles_replan(qvlib, orc, cuda):
    """The handle's plan cache: the same structure with new angles gives the new state."""
    qv = qvlib
    n = 15
    h = qv.qv_create(n, qv.QV_C64)
    try:
        for seed in (1, 2, 1):
            gates = W.random_circuit(n, 6, W.config_seed(0, 700 + seed))
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_FUSED, tile_bits=11, flags=qv.QV_PLAN_TENSOR)
            assert dist(qv.qv_get_state(h), orc.run(n, gates)) <= 1e-5, seed
    finally:
        qv.qv_destroy(h)


def test_tensor_rejects_unsupported(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(12, qv.QV_C128)
    try:
        with pytest.raises(qv.QvError):
            qv.qv_apply_circuit(h, W.random_circuit(12, 2, 1), mode=qv.QV_MODE_FUSED, tile_bits=11,
                                flags=qv.QV_PLAN_TENSOR)
    finally:
        qv.qv_destroy(h)
    h = qv.qv_create(12, qv.QV_C64)
    try:
        with pytest.raises(qv.QvError):
            qv.qv_apply_circuit(h, W.random_circuit(12, 2, 1), mode=qv.QV_MODE_FUSED, tile_bits=10,
                                flags=qv.QV_PLAN_TENSOR)
        # the handle stays usable
        qv.qv_apply_circuit(h, W.random_circuit(12, 2, 1), mode=qv.QV_MODE_FUSED, tile_bits=11,
                            flags=qv.QV_PLAN_TENSOR)
        assert abs(qv.qv_norm2(h) - 1.0) <= 1e-5
    finally:
        qv.qv_destroy(h)
