"""Parity of the per-gate CUDA kernels (Eq. 5 pair update, controlled and
diagonal forms, swaps) and of the reductions against the CPU oracle, on the
same seeded inputs, through the C ABI."""
import math

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from paper_2508_15545_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

# ||psi_gpu - psi_ref||_2 bounds: one gate moves a C64 amplitude by at most a
# few ulp of float (2^-24 ~ 6e-8) relative, so a unit vector picks up <~ 1e-6;
# complex128 stays near 1e-15 per gate.
TOL1 = {0: 2e-6, 1: 1e-13}
TOL_CIRCUIT = {0: 1e-5, 1: 1e-12}


def dist(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b))


def new_state(qv, n, dtype, psi=None):
    h = qv.qv_create(n, dtype)
    if psi is not None:
        qv.qv_set_state(h, psi)
    return h


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 12])
def test_apply_1q_every_target(qvlib, orc, cuda, dtype, n):
    qv = qvlib
    for t in range(n):
        U = W.random_matrix_2x2(100 * n + t)
        psi = W.random_state(n, 7 * n + t)
        h = new_state(qv, n, dtype, psi)
        qv.qv_apply_1q(h, t, U)
        got = qv.qv_get_state(h)
        qv.qv_destroy(h)
        want = orc.apply_1q(psi.copy(), t, U)
        assert dist(got, want) <= TOL1[dtype], (n, t)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [2, 3, 5, 9])
def test_apply_controlled_every_pair(qvlib, orc, cuda, dtype, n):
    qv = qvlib
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = W.random_matrix_2x2(1000 * n + 10 * c + t)
            psi = W.random_state(n, 3 * c + 5 * t + n)
            h = new_state(qv, n, dtype, psi)
            qv.qv_apply_controlled(h, c, t, U)
            got = qv.qv_get_state(h)
            qv.qv_destroy(h)
            want = orc.apply_controlled(psi.copy(), c, t, U)
            assert dist(got, want) <= TOL1[dtype], (n, c, t)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_gate_kinds_plain_mode(qvlib, orc, cuda, dtype, n):
    """Every gate kind (diagonal fast paths included), random controls and swaps."""
    qv = qvlib
    gates = W.random_gate_list(n, 150, seed=77 + n)
    psi = W.random_state(n, 99 + n)
    h = new_state(qv, n, dtype, psi)
    qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_PLAIN)
    got = qv.qv_get_state(h)
    qv.qv_destroy(h)
    want = orc.run(n, gates, psi.copy())
    assert dist(got, want) <= TOL_CIRCUIT[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_random_circuit_16q_plain(qvlib, orc, cuda, dtype):
    """16 qubits, 20 layers of U3 + brickwork CNOT (470 gates) from |0...0>."""
    qv = qvlib
    n = 16
    gates = W.random_circuit(n, 20, W.config_seed(0))
    h = qv.qv_create(n, dtype)
    qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_PLAIN)
    got = qv.qv_get_state(h)
    ez, tot = qv.qv_expect_z(h)
    qv.qv_destroy(h)
    want = orc.run(n, gates)
    assert dist(got, want) <= TOL_CIRCUIT[dtype]
    ez_ref = orc.expect_z(want)
    assert np.max(np.abs(ez - ez_ref)) <= (2e-5 if dtype == 0 else 1e-12)
    assert tot == pytest.approx(ez_ref.sum(), abs=1e-4 if dtype == 0 else 1e-11)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [1, 3, 9, 13, 14, 15, 17])
def test_reductions(qvlib, orc, cuda, dtype, n):
    qv = qvlib
    psi = W.random_state(n, 500 + n)
    h = new_state(qv, n, dtype, psi)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == 0 else psi
    tol = 1e-7 if dtype == 0 else 1e-13
    assert qv.qv_norm2(h) == pytest.approx(orc.norm2(ref), abs=tol)
    w = np.linspace(-1, 2, n)
    ez, tot = qv.qv_expect_z(h, w)
    ez_ref = orc.expect_z(ref)
    assert np.max(np.abs(ez - ez_ref)) <= tol
    assert tot == pytest.approx(float(np.dot(w, ez_ref)), abs=10 * tol)
    terms = W.ansatz_hamiltonian(n) if n >= 2 else [(0.5, 1, 0), (0.25, 0, 1)]
    terms = terms + [(0.3, (1 << n) - 1, 0), (-0.7, 0, (1 << n) - 1), (0.2, 1, 1)]
    got = qv.qv_expect_pauli(h, terms)
    want = orc.expect_terms(ref, terms)
    assert got == pytest.approx(want, abs=tol * 10 * len(terms))
    qv.qv_destroy(h)


@pytest.mark.parametrize("n", [14, 17])
def test_norm_and_z_sums_exact_squares(qvlib, orc, cuda, n):
    """complex64 norm and Z sums on a state whose magnitudes span six decades
    (not normalised): the squares are formed exactly (rounded product plus its
    FMA error term) and merged in two-float arithmetic, so they agree with the
    oracle on the stored amplitudes to about 1e-13 relative, where rounded FP32
    squares would leave errors near 1e-8."""
    qv = qvlib
    psi = W.random_state(n, 900 + n, normalize=False)
    scale = 10.0 ** (3.0 * W.SplitMix64(n + 1).uniform(1 << n) - 1.5)
    psi = (psi * scale).astype(np.complex64)
    h = new_state(qv, n, 0, psi)
    ref = qv.qv_get_state(h).astype(np.complex128)
    want = orc.norm2(ref)
    assert abs(qv.qv_norm2(h) - want) <= 1e-12 * want
    ez, _ = qv.qv_expect_z(h)
    assert np.max(np.abs(ez - orc.expect_z(ref))) <= 1e-12 * want
    qv.qv_destroy(h)


@pytest.mark.parametrize("n", [2, 5, 10])
def test_permute_qubits(qvlib, orc, cuda, n):
    qv = qvlib
    rng = W.SplitMix64(n)
    psi = W.random_state(n, 42)
    for _ in range(3):
        perm = [int(x) for x in np.argsort(rng.uniform(n))]
        h = new_state(qv, n, 1, psi)
        qv.qv_permute_qubits(h, perm)
        got = qv.qv_get_state(h)
        qv.qv_destroy(h)
        assert dist(got, orc.permute(psi, perm)) <= 1e-14


def test_basis_and_closed_forms(qvlib, orc, cuda):
    qv = qvlib
    n = 12
    h = qv.qv_create(n, 0)
    qv.qv_apply_circuit(h, [Gate("h", q) for q in range(n)], mode=qv.QV_MODE_PLAIN)
    assert np.allclose(qv.qv_get_state(h), 2 ** (-n / 2), atol=1e-7)
    qv.qv_set_basis(h, 0)
    qv.qv_apply_circuit(h, W.ghz_circuit(n), mode=qv.QV_MODE_PLAIN)
    g = qv.qv_get_state(h)
    assert abs(g[0] - 1 / math.sqrt(2)) < 1e-7 and abs(g[-1] - 1 / math.sqrt(2)) < 1e-7
    assert np.sum(np.abs(g[1:-1])) == 0
    j = 0b101101001011
    qv.qv_set_basis(h, j)
    qv.qv_apply_circuit(h, W.qft_circuit(n), mode=qv.QV_MODE_PLAIN)
    k = np.arange(1 << n)
    want = np.exp(2j * np.pi * ((j * k) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    assert dist(qv.qv_get_state(h), want) <= 1e-5
    qv.qv_destroy(h)


def test_errors_leave_handle_usable(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(5, 0)
    for bad in ([Gate("h", 5)], [Gate("x", 1, ctrl=1)], [Gate("swap", 2, target2=2)],
                [Gate("rx", 0, theta=(float("nan"), 0, 0))]):
        with pytest.raises(qv.QvError) as e:
            qv.qv_apply_circuit(h, bad)
        assert e.value.status == qv.QV_ERR_ARG
    with pytest.raises(qv.QvError):
        qv.qv_apply_1q(h, 0, [[float("inf"), 0], [0, 1]])
    with pytest.raises(qv.QvError):
        qv.qv_set_basis(h, 32)
    with pytest.raises(qv.QvError):
        qv.qv_permute_qubits(h, [0, 0, 1, 2, 3])
    qv.qv_apply_circuit(h, [Gate("x", 0)])
    assert abs(qv.qv_get_state(h)[1] - 1) < 1e-7
    qv.qv_destroy(h)


def test_oom_is_reported(qvlib, cuda):
    qv = qvlib
    with pytest.raises(qv.QvError) as e:
        qv.qv_create(38, 0)     # 2 TiB: refused before any allocation
    assert e.value.status == qv.QV_ERR_OOM


def test_torch_owned_state(qvlib, orc, cuda):
    qv = qvlib
    torch = cuda
    n = 10
    gates = W.random_circuit(n, 4, seed=5)
    s = qv.StateVector(n, qv.QV_C64, stream=torch.cuda.current_stream())
    s.apply(gates, mode=qv.QV_MODE_PLAIN)
    torch.cuda.synchronize()
    got = s.tensor.cpu().numpy()
    assert dist(got, orc.run(n, gates)) <= 1e-5
    s.close()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("nterms", [40, 160])
def test_expect_pauli_one_pass_and_many_groups(qvlib, orc, cuda, dtype, nterms):
    """<psi|H|psi> for random Pauli strings (X, Y, Z mixes): with few X-mask
    groups every group runs in one pass over the state; with more groups than
    shared memory holds (160 distinct masks), one pass per group."""
    qv = qvlib
    n = 11
    rng = W.SplitMix64(1234 + nterms)
    u = rng.integers(0, (1 << n) - 1, 2 * nterms)
    c = rng.uniform(nterms) * 2.0 - 1.0
    terms = [(float(c[k]), int(u[2 * k]), int(u[2 * k + 1])) for k in range(nterms)]
    psi = W.random_state(n, 77 + nterms)
    h = qv.qv_create(n, dtype)
    qv.qv_set_state(h, psi)
    got = qv.qv_expect_pauli(h, terms)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == 0 else psi
    want = orc.expect_terms(ref, terms)
    assert abs(got - want) <= (2e-5 if dtype == 0 else 1e-11) * sum(abs(t[0]) for t in terms)
    qv.qv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [3, 13, 18])
def test_sample_matches_oracle(qvlib, orc, cuda, dtype, n):
    """Inverse-CDF samples equal the oracle's on the same uniforms and the same
    stored amplitudes (bit-exact indices; a target within rounding of a
    cumulative boundary may take either neighbour, checked for validity)."""
    qv = qvlib
    psi = W.random_state(n, 500 + n)
    if n == 13:
        psi[: 1 << 10] = 0          # a run of zero-probability outcomes
        psi /= np.linalg.norm(psi)
    h = qv.qv_create(n, dtype)
    qv.qv_set_state(h, psi)
    stored = qv.qv_get_state(h).astype(np.complex128)
    u = np.concatenate([W.SplitMix64(n).uniform(3000), [0.0, np.nextafter(1.0, 0.0)]])
    got = qv.qv_sample(h, u)
    want = orc.sample(stored, u)
    p = stored.real ** 2 + stored.imag ** 2
    cdf = np.cumsum(p)
    for k in np.nonzero(got != want)[0]:
        i, t = int(got[k]), u[k] * cdf[-1]
        assert p[i] > 0 and cdf[i] >= t - 1e-12 * cdf[-1] and (i == 0 or cdf[i - 1] <= t + 1e-12 * cdf[-1])
    assert np.count_nonzero(got != want) <= 1
    idx = np.array([0, (1 << n) - 1, 5 % (1 << n), 7 % (1 << n)], dtype=np.uint64)
    amps = qv.qv_get_amplitudes(h, idx)
    assert np.array_equal(amps, qv.qv_get_state(h)[idx.astype(np.int64)])
    with pytest.raises(qv.QvError):
        qv.qv_sample(h, [1.0])
    with pytest.raises(qv.QvError):
        qv.qv_get_amplitudes(h, [1 << n])
    qv.qv_destroy(h)


def test_sample_basis_and_ghz(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(20, 0)
    qv.qv_set_basis(h, 123457)
    assert np.all(qv.qv_sample(h, np.linspace(0, 0.999, 50)) == 123457)
    qv.qv_set_basis(h, 0)
    qv.qv_apply_circuit(h, W.ghz_circuit(20))
    s = qv.qv_sample(h, np.linspace(0, 0.999, 200))
    assert set(int(x) for x in s) == {0, (1 << 20) - 1}
    qv.qv_destroy(h)


def _z_heavy_terms(n, seed):
    """Z strings of every shape the pure-Z tables handle: inside one 8-bit chunk
    of the index, spanning two chunks, on the top qubits, the identity, plus a
    few X and Y terms."""
    rng = W.SplitMix64(seed)
    terms = [(0.75, 0, 0)]                                        # identity
    for i in range(n - 1):
        terms.append((1.0 - 0.01 * i, 0, (1 << i) | (1 << (i + 1))))  # ZZ chain: within and across chunks
    for i in range(0, n, 3):
        terms.append((0.3, 0, 1 << i))                            # single Z
    u = rng.integers(1, (1 << n) - 1, 6)
    for k in range(6):
        terms.append((0.2 * (k + 1), 0, int(u[k])))               # wide Z strings (residual terms)
    terms += [(0.5, 1 << (n - 1), 0), (0.25, 0b101, 0b100), (-0.4, 1 << 3, 1 << 7)]
    return terms


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [12, 20, 27])
def test_pauli_z_tables(qvlib, orc, cuda, dtype, n):
    """<psi|H|psi> and H|psi> with a pure-Z group large enough for the chunk
    tables (terms inside 8-bit chunks tabled, the rest summed term by term),
    against the oracle on a random state."""
    qv = qvlib
    terms = _z_heavy_terms(n, 900 + n)
    psi = W.random_state(n, 31 + n)
    h = qv.qv_create(n, dtype)
    out = qv.qv_create(n, dtype)
    try:
        qv.qv_set_state(h, psi)
        got = qv.qv_expect_pauli(h, terms)
        ref = psi.astype(np.complex64).astype(np.complex128) if dtype == 0 else psi
        scale = sum(abs(t[0]) for t in terms)
        assert abs(got - orc.expect_terms(ref, terms)) <= (2e-5 if dtype == 0 else 1e-11) * scale
        qv.qv_apply_pauli(h, terms, out)
        want = orc.apply_pauli_sum(ref.copy(), terms)
        err = np.linalg.norm(qv.qv_get_state(out).astype(np.complex128) - want) / np.linalg.norm(want)
        assert err <= (5e-6 if dtype == 0 else 1e-13)
    finally:
        qv.qv_destroy(h)
        qv.qv_destroy(out)
