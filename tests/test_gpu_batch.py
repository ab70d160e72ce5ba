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


def test_batch_compiled_many_sets(qvlib, orc, cuda):
    """Forty parameter sets of one ansatz (one plan structure, the compiled
    kernel): energies equal the oracle's on sampled sets and the one-by-one GPU
    path on all of them; the batch reports its launch group."""
    qv = qvlib
    n, layers, count = 18, 6, 40
    terms = W.ansatz_hamiltonian(n)
    circuits = [W.ansatz_circuit(n, layers, W.config_seed(2, 300 + c))[0] for c in range(count)]
    states = [qv.qv_create(n, 0) for _ in range(count)]
    try:
        b = qv.Batch(list(zip(states, circuits)), terms)
        info = b.info()
        assert len(info) == 1 and info[0]["compiled"] == 1 and info[0]["circuits"] == count
        assert info[0]["qubits"] == n and info[0]["chunk_tiles"] == 32
        e = b.run()
        for c in (0, 23, count - 1):
            assert e[c] == pytest.approx(orc.energy(n, circuits[c], terms), abs=2e-5), c
        h = qv.qv_create(n, 0)
        for c in range(count):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, circuits[c])
            assert e[c] == pytest.approx(qv.qv_expect_pauli(h, terms), abs=2e-5), c
        qv.qv_destroy(h)
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_batch_autotunes_each_qubit_count(qvlib, orc, cuda):
    """QV_PLAN_AUTOTUNE at batch creation tunes every qubit count once; the
    batch then runs with the tuned tile sizes and gives the oracle's states."""
    qv = qvlib
    spec = [(13, 6), (15, 5), (13, 4), (16, 3)]
    circuits = [W.random_circuit(n, d, seed=1300 + k) for k, (n, d) in enumerate(spec)]
    states = [qv.qv_create(n, 0) for n, _ in spec]
    try:
        b = qv.Batch(list(zip(states, circuits)), flags=qv.QV_PLAN_AUTOTUNE)
        for g in b.info():
            assert g["tile_bits"] == qv.qv_default_tile_bits(g["qubits"], 0)
        b.run()
        for (n, _), h, g in zip(spec, states, circuits):
            assert np.linalg.norm(qv.qv_get_state(h).astype(complex) - orc.run(n, g)) <= 1e-5, n
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_autotune_schedule_variants(qvlib, orc, cuda):
    """The autotuner over tile sizes and schedule variants (pair operations on
    or off, tensor-core stages): it reports one of them, and the next fused call
    with no tile size or engine flags uses it and gives the oracle's state."""
    qv = qvlib
    n = 17
    g = W.random_circuit(n, 8, seed=17)
    h = qv.qv_create(n, 0)
    try:
        k, fl = qv.qv_autotune_ex(h, g)
        assert k in (10, 11, 12) and fl in (0, qv.QV_PLAN_NO_PAIRS, qv.QV_PLAN_TENSOR)
        assert not (fl == qv.QV_PLAN_TENSOR and k < 11)
        assert qv.qv_default_tile_bits(n, 0) == k
        qv.qv_apply_circuit(h, g, mode=qv.QV_MODE_FUSED)
        assert np.linalg.norm(qv.qv_get_state(h).astype(complex) - orc.run(n, g)) <= 1e-5
    finally:
        qv.qv_destroy(h)


def test_batch_large_member_runs_its_own_passes(qvlib, orc, cuda):
    """A member that fills the GPU alone (24 qubits: 2^13 tiles per pass) runs
    on its own compiled fused passes inside the batch graph; the small members
    stay in the persistent queue. Every state equals the oracle's, <H> too."""
    qv = qvlib
    spec = [(24, 4), (12, 5), (13, 3)]
    circuits = [W.random_circuit(n, d, seed=2400 + k) for k, (n, d) in enumerate(spec)]
    terms = [(1.0, 0, 0b11), (0.5, 0b1, 0)]
    states = [qv.qv_create(n, 0) for n, _ in spec]
    try:
        b = qv.Batch(list(zip(states, circuits)), terms)
        info = b.info()
        big = [g for g in info if g["compiled"] == 2]
        assert len(big) == 1 and big[0]["qubits"] == 24 and big[0]["circuits"] == 1
        for rep in range(2):
            e = b.run()
            for (n, _), h, g, ek in zip(spec, states, circuits, e):
                want = orc.run(n, g)
                assert np.linalg.norm(qv.qv_get_state(h).astype(complex) - want) <= 1e-5, (n, rep)
                assert ek == pytest.approx(orc.expect_terms(want, terms), abs=2e-5), (n, rep)
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_batch_members_on_side_streams(qvlib, orc, cuda):
    """Members whose passes have at least 2^8 tiles run on their own compiled
    passes, spread over the batch graph's side streams: twenty parameter sets of
    a 19-qubit ansatz (2^8 tiles of 2^11 amplitudes per pass). Energies equal
    the oracle's on sampled sets and the one-by-one GPU path on all of them,
    over two replays."""
    qv = qvlib
    n, layers, count = 19, 3, 20
    terms = W.ansatz_hamiltonian(n)
    circuits = [W.ansatz_circuit(n, layers, W.config_seed(2, 500 + c))[0] for c in range(count)]
    states = [qv.qv_create(n, 0) for _ in range(count)]
    try:
        b = qv.Batch(list(zip(states, circuits)), terms, tile_bits=11)
        info = b.info()
        assert len(info) == count and all(g["compiled"] == 2 and g["qubits"] == n for g in info)
        h = qv.qv_create(n, 0)
        one = []
        for c in range(count):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, circuits[c], tile_bits=11)
            one.append(qv.qv_expect_pauli(h, terms))
        qv.qv_destroy(h)
        for rep in range(2):
            e = b.run()
            for c in (0, 7, count - 1):
                assert e[c] == pytest.approx(orc.energy(n, circuits[c], terms), abs=2e-5), (c, rep)
            assert np.max(np.abs(np.array(e) - np.array(one))) <= 2e-5, rep
        psi = qv.qv_get_state(states[count - 1])
        assert np.linalg.norm(psi.astype(complex) - orc.run(n, circuits[count - 1])) <= 1e-5
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_batch_energy_many_groups(qvlib, orc, cuda):
    """A Hamiltonian of 95 X-mask groups (a pure-Z chain and 94 single-term X
    strings): the groups fill the batched kernel's shared memory, so the pure-Z
    group is summed term by term instead of through chunk tables; energies
    equal the oracle's."""
    qv = qvlib
    n = 12
    rng = W.SplitMix64(4242)
    masks = sorted(set(int(m) for m in rng.integers(1, (1 << n) - 1, 200)))[:94]
    terms = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)] + \
            [(0.01 * (k + 1), m, 0) for k, m in enumerate(masks)]
    circuits = [W.random_circuit(n, 4, seed=4300 + c) for c in range(3)]
    states = [qv.qv_create(n, 0) for _ in circuits]
    try:
        b = qv.Batch(list(zip(states, circuits)), terms)
        e = b.run()
        for c, g in enumerate(circuits):
            assert e[c] == pytest.approx(orc.energy(n, g, terms), abs=2e-5 * sum(abs(t[0]) for t in terms)), c
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)
