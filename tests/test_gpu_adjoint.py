"""Adjoint gradient and H|psi> against the oracle: gradients by the exact
parameter-shift rule and central differences (re-simulation only), H|psi> by
the oracle's Pauli-sum apply."""
import math

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from paper_2508_15545_gb300.workloads import Gate

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [3, 8, 13])
def test_apply_pauli_sum(qvlib, orc, cuda, dtype, n):
    qv = qvlib
    terms = W.ansatz_hamiltonian(n) + [(0.3, (1 << n) - 1, 0), (-0.7, 0b101, 0b110), (0.25, 0, (1 << n) - 1)]
    psi = W.random_state(n, 11 + n)
    a = qv.qv_create(n, dtype)
    b = qv.qv_create(n, dtype)
    qv.qv_set_state(a, psi)
    qv.qv_apply_pauli(a, terms, b)
    got = qv.qv_get_state(b)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == 0 else psi
    want = orc.apply_pauli_sum(ref, terms)
    tol = 2e-5 if dtype == 0 else 1e-12
    assert np.max(np.abs(got - want)) <= tol * len(terms)
    qv.qv_destroy(a)
    qv.qv_destroy(b)


def _adjoint(qv, n, dtype, gates, terms, npar, psi0=None, sweep=0):
    h = qv.qv_create(n, dtype)
    if psi0 is not None:
        qv.qv_set_state(h, psi0)
    before = qv.qv_get_state(h)
    g, e = qv.qv_adjoint_grad(h, gates, terms, npar, sweep_mode=sweep)
    after = qv.qv_get_state(h)
    qv.qv_destroy(h)
    return g, e, before, after


@pytest.mark.parametrize("dtype", [0, 1])
def test_adjoint_mixed_gates(qvlib, orc, cuda, dtype):
    """U3 (three trainable angles), RX/RY/RZ/P, controlled parametrised gates,
    a shared parameter, a SWAP and fixed gates."""
    qv = qvlib
    n = 6
    gates = [Gate("h", 0), Gate("u3", 1, theta=(0.4, 0.9, -0.3), param=(0, 1, 2)),
             Gate("x", 2, ctrl=1), Gate("rx", 3, theta=(0.6, 0, 0), param=(3, -1, -1)),
             Gate("rx", 4, theta=(0.6, 0, 0), param=(3, -1, -1)), Gate("swap", 0, target2=5),
             Gate("p", 2, ctrl=4, theta=(1.3, 0, 0), param=(4, -1, -1)),
             Gate("ry", 5, ctrl=0, theta=(-0.8, 0, 0), param=(5, -1, -1)),
             Gate("rz", 0, theta=(0.2, 0, 0), param=(6, -1, -1)), Gate("z", 3, ctrl=2),
             Gate("u3", 4, ctrl=3, theta=(1.1, -0.2, 0.7), param=(7, 8, -1))]
    terms = W.ansatz_hamiltonian(n) + [(0.4, 0b011, 0b010), (-0.3, 0, 0b110001)]
    psi0 = W.random_state(n, 3)
    g, e, before, after = _adjoint(qv, n, dtype, gates, terms, 9, psi0)
    want_e = orc.energy(n, gates, terms, psi0)
    ref = orc.param_shift_grad(n, gates, terms, 9, psi0)
    tol = 1e-4 if dtype == 0 else 1e-10
    assert e == pytest.approx(want_e, abs=tol)
    assert np.max(np.abs(g - ref)) <= tol, (g, ref)
    # the handle holds psi0 again
    assert np.linalg.norm(after.astype(complex) - before.astype(complex)) <= (1e-5 if dtype == 0 else 1e-12)


# sweep: 1 = one pass per gate, 2 = shared-memory tiles, 3 = compiled passes (complex64)
@pytest.mark.parametrize("sweep", [1, 2, 3])
@pytest.mark.parametrize("dtype", [0, 1])
def test_adjoint_ansatz_12q_vs_param_shift_and_fd(qvlib, orc, cuda, dtype, sweep):
    """12-qubit copy of the 26-qubit gradient workload: 16 layers of RY, RZ and
    a CZ ring (384 parameters), H = sum Z_i Z_i+1 + 0.5 sum X_i."""
    qv = qvlib
    n, layers = 12, 16
    gates, npar = W.ansatz_circuit(n, layers, W.config_seed(3, 1))
    terms = W.ansatz_hamiltonian(n)
    g, e, _, _ = _adjoint(qv, n, dtype, gates, terms, npar, sweep=sweep)
    ps = orc.param_shift_grad(n, gates, terms, npar)
    fd = orc.finite_diff_grad(n, gates, terms, npar, h=1e-3)
    l1 = sum(abs(c) for c, _, _ in terms)
    assert np.max(np.abs(ps - fd)) <= 1e-6 * l1
    tol = 1e-4 if dtype == 0 else 1e-9
    assert np.max(np.abs(g - ps)) <= tol
    assert e == pytest.approx(orc.energy(n, gates, terms), abs=tol)


def test_autograd_function(qvlib, orc, cuda):
    torch = cuda
    from paper_2508_15545_gb300.autograd import Expectation, expectation
    n, layers = 10, 3
    gates, npar = W.ansatz_circuit(n, layers, W.config_seed(3, 2))
    terms = W.ansatz_hamiltonian(n)
    model = Expectation(n, gates, terms, npar)
    p0 = np.array([g.theta[0] for g in gates if g.param[0] >= 0])
    order = [g.param[0] for g in gates if g.param[0] >= 0]
    params = torch.zeros(npar, dtype=torch.float64)
    params[order] = torch.tensor(p0)
    params.requires_grad_(True)
    e = expectation(params, model)
    e.backward()
    ps = orc.param_shift_grad(n, gates, terms, npar)
    assert float(e.detach()) == pytest.approx(orc.energy(n, gates, terms), abs=1e-5)
    assert np.max(np.abs(params.grad.numpy() - ps)) <= 1e-4
    model.close()


def test_adjoint_rejects_bad_params(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(4, 0)
    with pytest.raises(qv.QvError):
        qv.qv_adjoint_grad(h, [Gate("h", 0, param=(0, -1, -1))], [(1.0, 0, 1)], 1)
    with pytest.raises(qv.QvError):
        qv.qv_adjoint_grad(h, [Gate("ry", 0, param=(3, -1, -1))], [(1.0, 0, 1)], 2)
    qv.qv_destroy(h)


def _mixed_trainable(n, count, seed):
    """Random trainable gates on every qubit, controls near and far (outside
    a tile), diagonal gates on qubits outside a tile, SWAPs, fixed gates."""
    rng = W.SplitMix64(seed)
    gates, p = [], 0
    for k in range(count):
        u = rng.uniform(6)
        t = int(u[0] * n) % n
        c = int(u[1] * n) % n
        kind = ("u3", "rx", "ry", "rz", "p", "h", "swap", "cz", "cx")[int(u[2] * 9) % 9]
        th = (float(u[3]) * 6.0 - 3.0, float(u[4]) * 6.0 - 3.0, float(u[5]) * 6.0 - 3.0)
        ctrl = c if (c != t and u[5] < 0.35) else -1
        if kind == "swap":
            if c != t:
                gates.append(Gate("swap", t, target2=c))
            continue
        if kind in ("cz", "cx"):
            if c != t:
                gates.append(Gate("z" if kind == "cz" else "x", t, ctrl=c))
            continue
        if kind == "h":
            gates.append(Gate("h", t))
            continue
        na = 3 if kind == "u3" else 1
        par = tuple(p + a if a < na else -1 for a in range(3))
        p += na
        gates.append(Gate(kind, t, ctrl=ctrl, theta=th if kind == "u3" else (th[0], 0.0, 0.0), param=par))
    return gates, p


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [13, 15])
def test_adjoint_tiled_sweep_mixed(qvlib, orc, cuda, dtype, n):
    """Tiled reverse sweep on states of several tiles: controls and diagonal
    targets outside the tile, SWAPs, every trainable kind; against the
    oracle's parameter-shift gradient and against the per-gate sweep."""
    qv = qvlib
    gates, npar = _mixed_trainable(n, 70, seed=400 + n)
    terms = W.ansatz_hamiltonian(n) + [(0.35, 0b1010, 0b0110), (-0.2, 0, (1 << n) - 1)]
    psi0 = W.random_state(n, 9 + n)
    g1, e1, _, _ = _adjoint(qv, n, dtype, gates, terms, npar, psi0, sweep=1)
    ref = orc.param_shift_grad(n, gates, terms, npar, psi0)
    tol = 1e-4 if dtype == 0 else 1e-10
    for sweep in (2, 3):
        g2, e2, before, after = _adjoint(qv, n, dtype, gates, terms, npar, psi0, sweep=sweep)
        assert e2 == pytest.approx(orc.energy(n, gates, terms, psi0), abs=tol)
        assert np.max(np.abs(g2 - ref)) <= tol, sweep
        assert np.max(np.abs(g2 - g1)) <= tol, sweep
        assert np.linalg.norm(after.astype(complex) - before.astype(complex)) <= (2e-5 if dtype == 0 else 1e-12)


@pytest.mark.parametrize("dtype", [0, 1])
def test_adjoint_tiled_zero_angles(qvlib, orc, cuda, dtype):
    """Trainable gates at angle 0 are diagonal (RX(0) = I, U3(0, p, l) =
    diag(1, e^{i(p+l)})) while their derivatives are not: the tiled sweep must
    still bring their targets into the tile."""
    qv = qvlib
    n = 14
    gates = [Gate("h", q) for q in range(n)]
    gates += [Gate("rx", 13, theta=(0.0, 0, 0), param=(0, -1, -1)),
              Gate("ry", 12, theta=(0.0, 0, 0), param=(1, -1, -1)),
              Gate("u3", 11, theta=(0.0, 0.4, -0.9), param=(2, 3, 4)),
              Gate("x", 13, ctrl=2), Gate("rx", 10, ctrl=13, theta=(0.0, 0, 0), param=(5, -1, -1)),
              Gate("rz", 9, theta=(0.0, 0, 0), param=(6, -1, -1)),
              Gate("u3", 13, theta=(0.7, 0.1, 0.2), param=(7, -1, 8))]
    terms = [(1.0, 1 << 13, 0), (0.5, 1 << 12, 1 << 11), (0.25, 0, (1 << 10) | (1 << 9)), (0.3, 1 << 11, 0)]
    psi0 = W.random_state(n, 123)
    ref = orc.param_shift_grad(n, gates, terms, 9, psi0)
    tol = 1e-4 if dtype == 0 else 1e-10
    for sweep in (2, 3):
        g, e, _, _ = _adjoint(qv, n, dtype, gates, terms, 9, psi0, sweep=sweep)
        assert np.max(np.abs(g - ref)) <= tol, (sweep, g, ref)


def test_adjoint_cache_follows_the_angles(qvlib, orc, cuda):
    """The compiled sweep is kept per handle for the last gate list; new
    angles (same structure) must give the new gradient."""
    qv = qvlib
    n, layers = 12, 3
    gates, npar = W.ansatz_circuit(n, layers, W.config_seed(3, 7))
    terms = W.ansatz_hamiltonian(n)
    rng = W.SplitMix64(99)
    h = qv.qv_create(n, 0)
    try:
        for rep in range(3):
            params = rng.uniform(npar) * 2 * math.pi if rep else None
            gl = gates if params is None else W.with_params(gates, params)
            for _ in range(2):   # the second call reuses the compiled sweep
                qv.qv_set_basis(h, 0)
                g, e = qv.qv_adjoint_grad(h, gl, terms, npar)
                ref = orc.param_shift_grad(n, gl, terms, npar)
                assert np.max(np.abs(g - ref)) <= 1e-4, rep
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
def test_apply_pauli_many_groups(qvlib, orc, cuda, dtype):
    """H|psi> with so many X-mask groups (a pure-Z chain and 189 single-term X
    strings for complex64, 119 for complex128) that the groups fill the
    kernel's shared memory: the pure-Z group is then summed term by term
    instead of through chunk tables, and the result equals the oracle's."""
    qv = qvlib
    n = 12
    rng = W.SplitMix64(4343)
    masks = sorted(set(int(m) for m in rng.integers(1, (1 << n) - 1, 400)))[:189 if dtype == 0 else 119]
    terms = [(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)] + \
            [(0.01 * (k + 1), m, 0) for k, m in enumerate(masks)]
    psi = W.random_state(n, 4344)
    a = qv.qv_create(n, dtype)
    b = qv.qv_create(n, dtype)
    try:
        qv.qv_set_state(a, psi)
        qv.qv_apply_pauli(a, terms, b)
        ref = psi.astype(np.complex64).astype(np.complex128) if dtype == 0 else psi
        want = orc.apply_pauli_sum(ref, terms)
        tol = 2e-5 if dtype == 0 else 1e-12
        assert np.max(np.abs(qv.qv_get_state(b) - want)) <= tol * sum(abs(t[0]) for t in terms)
    finally:
        qv.qv_destroy(a)
        qv.qv_destroy(b)
