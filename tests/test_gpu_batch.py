"""Batched circuits in one graph-captured persistent launch, and the tile-size
autotuner, against the oracle."""
import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


# flags 0: one plan structure -> compiled persistent kernel; 2: interpreting kernel
@pytest.mark.parametrize("flags", [0, 2])
def test_batch_ansatz_energies(qvlib, orc, cuda, flags):
    """Parameter sets of the hardware-efficient ansatz (RY, RZ, CZ ring) with
    H = sum Z Z + 0.5 sum X: <H> per set, two replays of the same graph."""
    qv = qvlib
    n, layers, count = 12, 4, 12
    terms = W.ansatz_hamiltonian(n)
    circuits = [W.ansatz_circuit(n, layers, W.config_seed(2, c))[0] for c in range(count)]
    states = [qv.qv_create(n, 0) for _ in range(count)]
    b = qv.Batch(list(zip(states, circuits)), terms, flags=flags)
    want = np.array([orc.energy(n, g, terms) for g in circuits])
    for rep in range(2):
        got = b.run()
        assert np.max(np.abs(got - want)) <= 2e-5, rep
    psi = qv.qv_get_state(states[3])
    assert np.linalg.norm(psi.astype(complex) - orc.run(n, circuits[3])) <= 1e-5
    b.close()
    for h in states:
        qv.qv_destroy(h)


def test_apply_batch_one_shot(qvlib, orc, cuda):
    """qv_apply_batch (create, one run, destroy in one call) gives the oracle's
    <H> per state and leaves each state as the oracle's."""
    qv = qvlib
    n, layers, count = 11, 3, 5
    terms = W.ansatz_hamiltonian(n)
    circuits = [W.ansatz_circuit(n, layers, W.config_seed(2, 40 + c))[0] for c in range(count)]
    states = [qv.qv_create(n, 0) for _ in range(count)]
    got = qv.qv_apply_batch(list(zip(states, circuits)), terms)
    want = np.array([orc.energy(n, g, terms) for g in circuits])
    assert np.max(np.abs(got - want)) <= 2e-5
    for h, g in zip(states, circuits):
        assert np.linalg.norm(qv.qv_get_state(h).astype(complex) - orc.run(n, g)) <= 1e-5
    for h in states:
        qv.qv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_uneven_sizes(qvlib, orc, cuda, dtype):
    """Random circuits of uneven qubit counts and depths, several tile sizes."""
    qv = qvlib
    spec = [(10, 5), (14, 9), (11, 3), (17, 12), (12, 7), (16, 4), (13, 10), (15, 6)]
    circuits = [W.random_circuit(n, d, seed=900 + k) for k, (n, d) in enumerate(spec)]
    states = [qv.qv_create(n, dtype) for n, _ in spec]
    for tb in (0, 10):
        b = qv.Batch(list(zip(states, circuits)), tile_bits=tb)
        b.run()
        for (n, _), h, g in zip(spec, states, circuits):
            got = qv.qv_get_state(h)
            assert np.linalg.norm(got.astype(complex) - orc.run(n, g)) <= (1e-5 if dtype == 0 else 1e-12), (n, tb)
        b.close()
    for h in states:
        qv.qv_destroy(h)


def test_batch_rejects_bad_items(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(12, 0)
    small = qv.qv_create(6, 0)
    g = W.random_circuit(12, 2, 1)
    with pytest.raises(qv.QvError):
        qv.Batch([(h, g), (h, g)])                  # same state twice
    with pytest.raises(qv.QvError):
        qv.Batch([(small, W.random_circuit(6, 2, 1))])   # below the smallest tile
    with pytest.raises(qv.QvError):
        qv.Batch([(h, g)], terms=[(1.0, 1 << 13, 0)])    # term on a qubit >= n
    qv.qv_destroy(h)
    qv.qv_destroy(small)


def test_autotune_picks_a_tile_and_keeps_results_exact(qvlib, orc, cuda):
    qv = qvlib
    n = 18
    g = W.random_circuit(n, 6, seed=5)
    h = qv.qv_create(n, 0)
    best = qv.qv_autotune(h, g)
    assert best in (10, 11, 12)
    assert np.abs(qv.qv_get_state(h)[0] - 1) < 1e-7          # left at |0...0>
    qv.qv_apply_circuit(h, g, mode=qv.QV_MODE_FUSED)           # tile_bits = 0: tuned value
    assert np.linalg.norm(qv.qv_get_state(h).astype(complex) - orc.run(n, g)) <= 1e-5
    qv.qv_destroy(h)


def test_bounded_wait_reports_timeout(qvlib, orc, cuda):
    """The batch kernel's dependency wait, run into its limit on a counter
    nothing increments, reports QV_ERR_TIMEOUT through the status word; the
    handle, its stream and later kernels keep working."""
    qv = qvlib
    n = 12
    h = qv.qv_create(n, 0)
    for limit in (0, 1000):
        with pytest.raises(qv.QvError) as e:
            qv.qv_wait_selftest(h, limit)
        assert e.value.status == qv.QV_ERR_TIMEOUT
        qv.qv_sync(h)   # reported once, then cleared
    with pytest.raises(qv.QvError) as e:
        qv.qv_wait_selftest(h, (1 << 24) + 1)
    assert e.value.status == qv.QV_ERR_ARG
    gates = W.random_circuit(n, 6, W.config_seed(0, 7))
    qv.qv_apply_circuit(h, gates)
    psi = qv.qv_get_state(h)
    assert np.linalg.norm(psi.astype(complex) - orc.run(n, gates)) <= 1e-5
    qv.qv_destroy(h)
