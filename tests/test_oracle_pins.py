"""Pins for the CPU oracle: each test checks it against something other than
itself -- dense Kronecker matrices (Sec. II, Eq. 3-4), textbook closed forms,
invariants and hand-written textbook values under tests/golden/."""
import json
import math
import os

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from paper_2508_15545_gb300.workloads import Gate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# textbook Pauli matrices, written out here (not taken from the oracle)
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def kron_all(factors_high_to_low):
    out = np.array([[1.0 + 0j]])
    for f in factors_high_to_low:
        out = np.kron(out, f)
    return out


def dense_1q(n, t, U):
    """I_{2^(n-1-t)} (x) U (x) I_{2^t}: Eq. 3's Kronecker extension of U."""
    return np.kron(np.kron(np.eye(1 << (n - 1 - t)), U), np.eye(1 << t))


def dense_controlled(n, c, t, U):
    """|0><0|_c (x) I + |1><1|_c (x) U_t as a 2^n x 2^n matrix."""
    f0 = [I2] * n
    f1 = [I2] * n
    f0[n - 1 - c] = P0
    f1[n - 1 - c] = P1
    f1[n - 1 - t] = U
    return kron_all(f0) + kron_all(f1)


def dense_pauli(n, xmask, zmask):
    f = []
    for q in range(n - 1, -1, -1):
        x, z = (xmask >> q) & 1, (zmask >> q) & 1
        f.append(PY if (x and z) else PX if x else PZ if z else I2)
    return kron_all(f)


ALL_KINDS_1Q = ["h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "p", "u3", "matrix"]


def _gate(kind, t, seed, ctrl=-1):
    rng = W.SplitMix64(seed)
    th = tuple(float(a) for a in rng.uniform(3) * 4 * math.pi - 2 * math.pi)
    mat = tuple(W.random_unitary(rng).reshape(-1)) if kind == "matrix" else None
    return Gate(kind, t, ctrl=ctrl, theta=th, matrix=mat)


# ----------------------------------------------------------------------------
# gate matrices
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ALL_KINDS_1Q)
def test_gate_matrices_unitary(orc, kind):
    for s in range(5):
        U = orc.gate_matrix(_gate(kind, 0, 77 + s))
        assert np.allclose(U @ U.conj().T, I2, atol=1e-14)


def test_gate_matrix_textbook_values(orc):
    """Fixed points of the gate definitions (OpenQASM / Nielsen-Chuang)."""
    r = 1 / math.sqrt(2)
    M = lambda kind, *th: orc.gate_matrix(Gate(kind, 0, theta=tuple(th) + (0.0,) * (3 - len(th))))
    assert np.allclose(M("h"), [[r, r], [r, -r]])
    assert np.allclose(M("x"), PX) and np.allclose(M("y"), PY) and np.allclose(M("z"), PZ)
    assert np.allclose(M("s"), [[1, 0], [0, 1j]]) and np.allclose(M("sdg"), [[1, 0], [0, -1j]])
    assert np.allclose(M("t"), [[1, 0], [0, (1 + 1j) * r]])
    assert np.allclose(M("tdg"), [[1, 0], [0, (1 - 1j) * r]])
    # rotations at a quarter turn: R_a(pi/2) = (I - i sigma_a)/sqrt(2)
    for kind, P in (("rx", PX), ("ry", PY), ("rz", PZ)):
        assert np.allclose(M(kind, math.pi / 2), (I2 - 1j * P) * r)
        assert np.allclose(M(kind, math.pi), -1j * P)
    for th in np.linspace(-3, 3, 7):
        # U3 special cases
        assert np.allclose(M("u3", th, 0, 0), M("ry", th))
        assert np.allclose(M("u3", 0, 0, th), M("p", th))
        assert np.allclose(M("u3", th, -math.pi / 2, math.pi / 2), M("rx", th))
        # RZ equals P up to the global phase exp(-i th/2)
        assert np.allclose(M("rz", th), np.exp(-0.5j * th) * M("p", th))
        # U3 = exp(i(phi+lambda)/2) RZ(phi) RY(theta) RZ(lambda)
        ph, la = 0.3 * th + 0.1, -0.7 * th + 0.4
        assert np.allclose(M("u3", th, ph, la),
                           np.exp(0.5j * (ph + la)) * M("rz", ph) @ M("ry", th) @ M("rz", la))
    assert np.allclose(M("u3", math.pi / 2, 0, math.pi), M("h"))
    assert np.allclose(M("p", math.pi / 2), M("s")) and np.allclose(M("p", math.pi / 4), M("t"))
    # HXH = Z, Y = iXZ
    assert np.allclose(M("h") @ PX @ M("h"), PZ)
    assert np.allclose(1j * PX @ PZ, PY)


# ----------------------------------------------------------------------------
# Eq. 5 against the dense Kronecker matrix (Eq. 3-4)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_apply_1q_equals_kronecker(orc, n):
    for t in range(n):
        for s, kind in enumerate(["matrix", "u3", "h", "rx"]):
            U = orc.gate_matrix(_gate(kind, t, 1000 * n + 10 * t + s))
            psi = W.random_state(n, 5 + t + 31 * s)
            want = dense_1q(n, t, U) @ psi
            got = orc.apply_1q(psi.copy(), t, U)
            assert np.allclose(got, want, atol=1e-13, rtol=0)


def test_apply_1q_non_unitary_matrix(orc):
    """Eq. 5 is linear for any 2x2 matrix, not only unitaries."""
    U = np.array([[1.5, -0.25j], [2.0 + 1j, 0.0]])
    for n in (3, 5):
        for t in range(n):
            psi = W.random_state(n, 3 * t + n)
            assert np.allclose(orc.apply_1q(psi.copy(), t, U), dense_1q(n, t, U) @ psi, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_controlled_equals_dense(orc, n):
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            U = orc.gate_matrix(_gate("matrix", t, 7 * n + 3 * c + t))
            psi = W.random_state(n, 100 + 10 * c + t)
            want = dense_controlled(n, c, t, U) @ psi
            got = orc.apply_controlled(psi.copy(), c, t, U)
            assert np.allclose(got, want, atol=1e-13, rtol=0)


def test_run_matches_dense_product(orc):
    """A random gate list of every kind, checked gate by gate against dense matrices."""
    n = 5
    gates = W.random_gate_list(n, 120, seed=4242)
    psi = W.random_state(n, 9)
    want = psi.copy()
    for g in gates:
        if g.kind == "swap":
            Mx = np.zeros((1 << n, 1 << n))
            for i in range(1 << n):
                a, b = (i >> g.target) & 1, (i >> g.target2) & 1
                j = i & ~((1 << g.target) | (1 << g.target2)) | (b << g.target) | (a << g.target2)
                Mx[j, i] = 1
            want = Mx @ want
            continue
        U = orc.gate_matrix(g)
        want = (dense_controlled(n, g.ctrl, g.target, U) if g.ctrl >= 0 else dense_1q(n, g.target, U)) @ want
    got = orc.run(n, gates, psi.copy())
    assert np.allclose(got, want, atol=1e-12)


def test_swap_and_permute_equal_axis_transpose(orc):
    n = 5
    psi = W.random_state(n, 11)
    # numpy reshape of a little-endian vector: axis a holds qubit n-1-a
    tens = psi.reshape([2] * n)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            axes = list(range(n))
            axes[n - 1 - a], axes[n - 1 - b] = axes[n - 1 - b], axes[n - 1 - a]
            want = np.transpose(tens, axes).reshape(-1)
            assert np.allclose(orc.apply_swap(psi.copy(), a, b), want)
    rng = W.SplitMix64(5)
    for _ in range(6):
        perm = list(np.argsort(rng.uniform(n)))
        out = orc.permute(psi, perm)
        # out qubit perm[q] = in qubit q  ->  out axis (n-1-perm[q]) = in axis (n-1-q)
        axes = [0] * n
        for q in range(n):
            axes[n - 1 - perm[q]] = n - 1 - q
        want = np.transpose(tens, axes).reshape(-1)
        assert np.allclose(out, want)
        inv = [0] * n
        for q in range(n):
            inv[perm[q]] = q
        assert np.allclose(orc.permute(out, inv), psi)


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------
def test_hadamard_wall_is_uniform(orc):
    n = 10
    psi = orc.run(n, [Gate("h", q) for q in range(n)])
    assert np.allclose(psi, 2 ** (-n / 2), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_ghz(orc, n):
    psi = orc.run(n, W.ghz_circuit(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-15)
    if n >= 2:
        assert orc.expect_pauli(psi, 0, 0b11) == pytest.approx(1.0)
        assert orc.expect_pauli(psi, (1 << n) - 1, 0) == pytest.approx(1.0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_qft_closed_form(orc, n):
    """QFT|j> = sum_k exp(2 pi i j k / 2^n) |k> / 2^(n/2); phase from (j k mod 2^n)."""
    N = 1 << n
    gates = W.qft_circuit(n)
    for j in sorted({0, 1, N - 1, (5 * N) // 7, N // 2}):
        psi = orc.run(n, gates, orc.basis(n, j))
        k = np.arange(N)
        want = np.exp(2j * np.pi * ((j * k) % N) / N) / math.sqrt(N)
        assert np.allclose(psi, want, atol=1e-12)


def test_golden_textbook_two_qubit(orc):
    with open(os.path.join(GOLDEN, "textbook_two_qubit.json")) as f:
        data = json.load(f)
    for case in data["cases"]:
        if case.get("circuit") == "qft":
            gates = W.qft_circuit(2)
        else:
            gates = [Gate(k, t, ctrl=c) for k, t, c in case["gates"]]
        psi = orc.run(2, gates, orc.basis(2, case["input_basis"]))
        want = np.array([complex(re, im) for re, im in case["amplitudes"]])
        assert np.allclose(psi, want, atol=1e-15), case["name"]


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------
def test_norm_preserved_and_inverse_returns_input(orc):
    n = 8
    gates = W.random_circuit(n, 6, seed=17) + W.random_gate_list(n, 60, seed=18)
    psi0 = W.random_state(n, 19)
    psi = orc.run(n, gates, psi0.copy())
    assert orc.norm2(psi) == pytest.approx(1.0, abs=1e-12)
    inv = []
    for g in reversed(gates):
        if g.kind == "swap":
            inv.append(g)
        else:
            Ud = orc.gate_matrix(g).conj().T
            inv.append(Gate("matrix", g.target, ctrl=g.ctrl, matrix=tuple(Ud.reshape(-1))))
    back = orc.run(n, inv, psi)
    assert np.allclose(back, psi0, atol=1e-12)


def test_gates_on_different_qubits_commute(orc):
    n = 6
    a = _gate("u3", 1, 3)
    b = Gate("matrix", 4, ctrl=2, matrix=_gate("matrix", 4, 9).matrix)
    psi = W.random_state(n, 2)
    assert np.allclose(orc.run(n, [a, b], psi.copy()), orc.run(n, [b, a], psi.copy()), atol=1e-14)


# ----------------------------------------------------------------------------
# reductions
# ----------------------------------------------------------------------------
def test_expect_z_product_state_closed_form(orc):
    """U3(theta, phi, lambda)|0> has <Z> = cos(theta), <X> = sin(theta) cos(phi)."""
    n = 7
    rng = W.SplitMix64(8)
    th = rng.uniform(3 * n) * 2 * math.pi
    gates = [Gate("u3", q, theta=(th[3 * q], th[3 * q + 1], th[3 * q + 2])) for q in range(n)]
    psi = orc.run(n, gates)
    assert np.allclose(orc.expect_z(psi), np.cos(th[0::3]), atol=1e-13)
    for q in range(n):
        assert orc.expect_pauli(psi, 1 << q, 0) == pytest.approx(math.sin(th[3 * q]) * math.cos(th[3 * q + 1]), abs=1e-13)
        assert orc.expect_pauli(psi, 0, 1 << q) == pytest.approx(math.cos(th[3 * q]), abs=1e-13)
    # product state: <Z_a Z_b> = <Z_a><Z_b>
    assert orc.expect_pauli(psi, 0, 0b101) == pytest.approx(math.cos(th[0]) * math.cos(th[6]), abs=1e-13)
    assert orc.norm2(psi) == pytest.approx(1.0, abs=1e-14)


def test_expect_pauli_equals_dense(orc):
    n = 5
    psi = W.random_state(n, 23)
    rng = W.SplitMix64(24)
    for _ in range(25):
        x, z = (int(v) for v in rng.integers(0, (1 << n) - 1, 2))
        want = np.vdot(psi, dense_pauli(n, x, z) @ psi)
        assert abs(want.imag) < 1e-12
        assert orc.expect_pauli(psi, x, z) == pytest.approx(want.real, abs=1e-13)
    ez = orc.expect_z(psi)
    for q in range(n):
        assert ez[q] == pytest.approx(np.vdot(psi, dense_pauli(n, 0, 1 << q) @ psi).real, abs=1e-13)


def test_apply_pauli_sum_equals_dense(orc):
    n = 5
    terms = W.ansatz_hamiltonian(n) + [(0.7, 0b00110, 0b00100), (-0.3, 0b10001, 0b11000)]
    Hd = sum(c * dense_pauli(n, x, z) for c, x, z in terms)
    psi = W.random_state(n, 31)
    assert np.allclose(orc.apply_pauli_sum(psi, terms), Hd @ psi, atol=1e-13)
    assert orc.expect_terms(psi, terms) == pytest.approx(np.vdot(psi, Hd @ psi).real, abs=1e-12)


# ----------------------------------------------------------------------------
# gradients
# ----------------------------------------------------------------------------
def test_gradient_closed_form_product_ry(orc):
    """E = sum_q <Z_q> after RY(theta_q)|0> is sum_q cos(theta_q): dE/dtheta_q = -sin(theta_q)."""
    n = 4
    th = [0.3, -1.1, 2.0, 0.77]
    gates = [Gate("ry", q, theta=(th[q], 0, 0), param=(q, -1, -1)) for q in range(n)]
    terms = [(1.0, 0, 1 << q) for q in range(n)]
    ps = orc.param_shift_grad(n, gates, terms, n)
    fd = orc.finite_diff_grad(n, gates, terms, n)
    assert np.allclose(ps, -np.sin(th), atol=1e-12)
    assert np.allclose(fd, -np.sin(th), atol=1e-6)


def test_gradient_u3_and_shared_parameter(orc):
    n = 3
    gates = [Gate("u3", 0, theta=(0.4, 0.9, -0.3), param=(0, 1, 2)),
             Gate("x", 1, ctrl=0),
             Gate("rx", 2, theta=(0.6, 0, 0), param=(3, -1, -1)),
             Gate("rx", 1, theta=(0.6, 0, 0), param=(3, -1, -1)),
             Gate("p", 2, ctrl=1, theta=(1.3, 0, 0), param=(4, -1, -1)),
             Gate("rz", 0, theta=(0.2, 0, 0), param=(5, -1, -1)),
             Gate("h", 0)]
    terms = W.ansatz_hamiltonian(n) + [(0.4, 0b011, 0b010)]
    ps = orc.param_shift_grad(n, gates, terms, 6)
    fd = orc.finite_diff_grad(n, gates, terms, 6)
    assert np.allclose(ps, fd, atol=1e-6)


def test_gradient_controlled_rotations_ps_vs_fd(orc):
    """Controlled rotations (generator eigenvalues -1/2, 0, 1/2) need the
    four-term shift rule; controlled phases and U3's phi / lambda do not."""
    n = 4
    gates = [Gate("h", 0), Gate("h", 2),
             Gate("ry", 1, ctrl=0, theta=(0.7, 0, 0), param=(0, -1, -1)),
             Gate("rx", 3, ctrl=2, theta=(-1.2, 0, 0), param=(1, -1, -1)),
             Gate("rz", 2, ctrl=1, theta=(0.4, 0, 0), param=(2, -1, -1)),
             Gate("u3", 0, ctrl=3, theta=(1.1, -0.2, 0.7), param=(3, 4, 5)),
             Gate("p", 3, ctrl=0, theta=(0.9, 0, 0), param=(6, -1, -1)),
             Gate("h", 1)]
    terms = W.ansatz_hamiltonian(n) + [(0.5, 0b0101, 0b0011)]
    ps = orc.param_shift_grad(n, gates, terms, 7)
    fd = orc.finite_diff_grad(n, gates, terms, 7, h=1e-4)
    assert np.max(np.abs(ps - fd)) <= 1e-7
    assert np.max(np.abs(ps)) > 1e-2


def test_gradient_ansatz_ps_vs_fd(orc):
    n, layers = 4, 2
    gates, npar = W.ansatz_circuit(n, layers, seed=W.config_seed(3, 1))
    terms = W.ansatz_hamiltonian(n)
    ps = orc.param_shift_grad(n, gates, terms, npar)
    fd = orc.finite_diff_grad(n, gates, terms, npar)
    l1 = sum(abs(c) for c, _, _ in terms)
    assert np.max(np.abs(ps - fd)) <= 1e-6 * l1
    assert np.max(np.abs(ps)) > 1e-3


# ----------------------------------------------------------------------------
# workloads (input recipes)
# ----------------------------------------------------------------------------
def test_splitmix64_known_answer():
    """First outputs of SplitMix64 seeded with 0 (Vigna's reference code)."""
    got = [int(v) for v in W.SplitMix64(0).next_block(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_workload_sizes():
    assert len(W.random_circuit(16, 20, W.config_seed(0))) == 470
    assert len(W.random_circuit(30, 40, W.config_seed(1))) == 1780 == W.layer_count_gates(30, 40)
    g, npar = W.ansatz_circuit(26, 16, W.config_seed(3))
    assert npar == 832 and len(g) == 16 * 3 * 26
    g, npar = W.ansatz_circuit(12, 16, W.config_seed(3, 1))
    assert npar == 384
    assert len(W.qft_circuit(33)) == 33 + 528 + 16
    b = W.uneven_batch(64, W.config_seed(4))
    assert len(b) == 64 and all(16 <= n <= 28 and 10 <= d <= 60 for n, d, _ in b)
    assert len(W.ansatz_hamiltonian(20)) == 19 + 20


def test_u3_inverse_identity(orc):
    """U3(t, p, l)^-1 = U3(-t, -l, -p), used to undo the bench circuit on the GPU."""
    from paper_2508_15545_gb300.workloads import Gate
    for t, p, l in [(0.3, 1.1, -0.7), (2.9, -2.0, 0.4), (0.0, 0.5, 0.5)]:
        U = orc.gate_matrix(Gate("u3", 0, theta=(t, p, l)))
        V = orc.gate_matrix(Gate("u3", 0, theta=(-t, -l, -p)))
        assert np.allclose(V @ U, np.eye(2), atol=1e-14)


def test_sample_pins(orc):
    """Inverse-CDF sampling: a basis state always gives its index; a known
    distribution gives the outcomes its cumulative sums fix, skipping
    zero-probability outcomes; brute force on a random small state."""
    psi = orc.basis(5, 19)
    assert np.all(orc.sample(psi, [0.0, 0.3, 0.999999]) == 19)
    amp = np.array([0.5, 0, 0.5j, 0, -0.5, 0.5, 0, 0], dtype=np.complex128)   # p = 1/4 at 0, 2, 4, 5 (exact)
    got = orc.sample(amp, [0.0, 0.1, 0.25, 0.5, 0.7499, 0.75, 0.99, np.nextafter(1.0, 0.0)])
    assert [int(x) for x in got] == [0, 0, 2, 4, 4, 5, 5, 5]
    amp0 = np.array([0.6, 0.8, 0.0, 0.0], dtype=np.complex128)   # last outcomes have p = 0
    assert orc.sample(amp0, [np.nextafter(1.0, 0.0)])[0] == 1
    rng = np.random.default_rng(3)
    psi = W.random_state(6, 44)
    u = rng.random(300)
    p = np.abs(psi) ** 2
    for uk, ik in zip(u, orc.sample(psi, u)):
        acc, want = 0.0, None
        for i, pi in enumerate(p):          # first index whose running sum exceeds u * total
            acc += pi
            if acc > uk * p.sum():
                want = i
                break
        assert int(ik) == want
