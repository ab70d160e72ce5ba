"""Closed-form QFT check on the GPU, the 33-qubit (64 GiB) QFT, and full-size
checks of the bench, batch and gradient workloads."""
import math

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [10, 13])
def test_verify_qft_matches_numpy_distance(qvlib, cuda, dtype, n):
    """The GPU distance equals the distance numpy computes from the fetched state."""
    qv = qvlib
    N = 1 << n
    h = qv.qv_create(n, dtype)
    for j in (0, 5, N - 1):
        qv.qv_set_basis(h, j)
        qv.qv_apply_circuit(h, W.qft_circuit(n))
        psi = qv.qv_get_state(h).astype(complex)
        k = np.arange(N)
        ref = np.exp(2j * np.pi * ((j * k) % N) / N) / math.sqrt(N)
        want = float(np.linalg.norm(psi - ref))
        got = qv.qv_verify_qft(h, j)
        assert got == pytest.approx(want, abs=1e-9)
        assert got <= (1e-5 if dtype == 0 else 1e-12)
        # a wrong j is far away
        assert qv.qv_verify_qft(h, (j + 1) % N) > 0.5
    qv.qv_destroy(h)


def test_qft_33_qubits_closed_form(qvlib, cuda):
    """33-qubit complex64 QFT of a random basis state (64 GiB), fused passes."""
    qv = qvlib
    torch = cuda
    free, _ = torch.cuda.mem_get_info()
    n = 33
    if free < (8 << n) + (4 << 30):
        pytest.skip("needs 68 GiB of free device memory")
    j = int(W.SplitMix64(W.config_seed(4, 99)).integers(0, (1 << n) - 1, 1)[0])
    h = qv.qv_create(n, 0)
    qv.qv_set_basis(h, j)
    qv.qv_apply_circuit(h, W.qft_circuit(n))
    d = qv.qv_verify_qft(h, j)
    nrm = qv.qv_norm2(h)
    qv.qv_destroy(h)
    assert d <= 1e-5
    # complex64 rounds 1/sqrt(2) down by ~1.6e-8 relative; 33 Hadamards per
    # amplitude leave ||psi||^2 about 1e-6 low, within the 1e-5 state bound
    assert nrm == pytest.approx(1.0, abs=1e-5)


def test_distance_mixed_precision(qvlib, orc, cuda):
    qv = qvlib
    n = 14
    g = W.random_circuit(n, 5, seed=8)
    a = qv.qv_create(n, 0)
    b = qv.qv_create(n, 1)
    qv.qv_apply_circuit(a, g)
    qv.qv_apply_circuit(b, g)
    pa, pb = qv.qv_get_state(a).astype(complex), qv.qv_get_state(b)
    assert qv.qv_distance(a, b) == pytest.approx(float(np.linalg.norm(pa - pb)), rel=1e-6, abs=1e-12)
    assert qv.qv_distance(b, b) == 0.0
    qv.qv_set_basis(b, 1)
    assert qv.qv_distance(a, b) == pytest.approx(float(np.linalg.norm(pa - np.eye(1 << n)[1])), rel=1e-9)
    qv.qv_destroy(a)
    qv.qv_destroy(b)


def _inverse_random_circuit(gates):
    """U3(t, p, l)^-1 = U3(-t, -l, -p); CNOT is its own inverse; reversed order."""
    out = []
    for g in reversed(gates):
        if g.kind == "u3":
            t, p, l = g.theta
            out.append(g._replace(theta=(-t, -l, -p)))
        else:
            out.append(g)
    return out


def test_bench_circuit_30_qubits_properties(qvlib, cuda):
    """The 30-qubit, 1,780-gate circuit the bench times, at full size, in the
    bench's launch configuration: the fused passes agree with the per-gate
    kernels (an independent kernel family), keep the norm, and the inverse
    circuit brings the state back to |0...0>."""
    qv = qvlib
    n, layers = 30, 40
    gates = W.random_circuit(n, layers, W.config_seed(1))
    assert len(gates) == 1780
    hf = qv.qv_create(n, 0)
    hp = qv.qv_create(n, 0)
    try:
        qv.qv_apply_circuit(hf, gates, mode=qv.QV_MODE_FUSED)
        qv.qv_apply_circuit(hp, gates, mode=qv.QV_MODE_PLAIN)
        assert qv.qv_distance(hf, hp) <= 1e-5
        assert abs(qv.qv_norm2(hf) - 1.0) <= 1e-5
        qv.qv_apply_circuit(hf, _inverse_random_circuit(gates), mode=qv.QV_MODE_FUSED)
        qv.qv_set_basis(hp, 0)
        assert qv.qv_distance(hf, hp) <= 2e-5
    finally:
        qv.qv_destroy(hf)
        qv.qv_destroy(hp)


def test_batch_256_ansatz_20_qubits_full_size(qvlib, orc, cuda):
    """The batched workload at full size (256 parameter sets of the 20-qubit,
    12-layer ansatz, <H> each, one graph), as the bench runs it: four sampled
    members against the oracle's energy, every member within the spectral
    bound ||H||_1 and against the one-by-one GPU path."""
    qv = qvlib
    n, layers, count = 20, 12, 256
    terms = W.ansatz_hamiltonian(n)
    circuits = [W.ansatz_circuit(n, layers, W.config_seed(2, c))[0] for c in range(count)]
    states = [qv.qv_create(n, 0) for _ in range(count)]
    try:
        b = qv.Batch(list(zip(states, circuits)), terms)
        e = b.run()
        l1 = sum(abs(c) for c, _, _ in terms)
        assert np.all(np.abs(e) <= l1 + 1e-9)
        for c in (0, 77, 128, 255):
            assert e[c] == pytest.approx(orc.energy(n, circuits[c], terms), abs=1e-4), c
        h = qv.qv_create(n, 0)
        for c in range(0, count, 37):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, circuits[c])
            assert e[c] == pytest.approx(qv.qv_expect_pauli(h, terms), abs=1e-5), c
        qv.qv_destroy(h)
        b.close()
    finally:
        for h in states:
            qv.qv_destroy(h)


def test_adjoint_26_qubits_full_size(qvlib, cuda):
    """The gradient workload at full size (26-qubit ansatz, 16 layers, 832
    parameters): the compiled sweep against the per-gate sweep (an independent
    kernel family) on every parameter, and three sampled parameters against
    central differences of GPU energies (h = 1e-3, O(h^2))."""
    qv = qvlib
    n, layers = 26, 16
    gates, npar = W.ansatz_circuit(n, layers, W.config_seed(3))
    terms = W.ansatz_hamiltonian(n)
    h = qv.qv_create(n, 0)
    try:
        g3, e3 = qv.qv_adjoint_grad(h, gates, terms, npar, sweep_mode=qv.QV_SWEEP_COMPILED)
        qv.qv_set_basis(h, 0)
        g1, e1 = qv.qv_adjoint_grad(h, gates, terms, npar, sweep_mode=qv.QV_SWEEP_PER_GATE)
        assert np.max(np.abs(g3 - g1)) <= 1e-5
        assert e3 == pytest.approx(e1, abs=1e-6)
        params = np.zeros(npar)
        for g in gates:
            for a, p in enumerate(g.param):
                if p >= 0:
                    params[p] = g.theta[a]

        def energy(pv):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, W.with_params(gates, pv))
            return qv.qv_expect_pauli(h, terms)
        hstep = 1e-3
        for p in (0, 417, npar - 1):
            up, dn = params.copy(), params.copy()
            up[p] += hstep
            dn[p] -= hstep
            fd = (energy(up) - energy(dn)) / (2 * hstep)
            assert g3[p] == pytest.approx(fd, abs=1e-2), p  # FP32 energies, divided by 2h
    finally:
        qv.qv_destroy(h)
