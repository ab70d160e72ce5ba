"""Parity of the fused tiled passes (planner + on-chip kernel) against the CPU
oracle and against the per-gate kernels, through the C ABI."""
import math

import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from paper_2508_15545_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def dist(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b))


def run_gpu(qv, n, dtype, gates, psi=None, mode=2, tile_bits=0, basis=0, flags=0):
    h = qv.qv_create(n, dtype)
    try:
        if psi is not None:
            qv.qv_set_state(h, psi)
        else:
            qv.qv_set_basis(h, basis)
        qv.qv_apply_circuit(h, gates, mode=mode, tile_bits=tile_bits, flags=flags)
        return qv.qv_get_state(h)
    finally:
        qv.qv_destroy(h)


# flags: 0 = compiled passes with gate fusion (and 4x4 pair ops for complex64),
# 1 = no fusion, 2 = interpreting kernel, 4 = fusion without 4x4 pair ops
@pytest.mark.parametrize("flags", [0, 1, 2, 4])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,k", [(10, 10), (11, 10), (11, 11), (12, 12), (13, 10), (13, 12), (16, 11), (17, 12)])
def test_random_gate_kinds_fused(qvlib, orc, cuda, dtype, n, k, flags):
    """Every gate kind, random controls (inside and outside the tile), swaps."""
    qv = qvlib
    gates = W.random_gate_list(n, 200, seed=1000 * n + k, ctrl_prob=0.4)
    psi = W.random_state(n, 31 * n + k)
    got = run_gpu(qv, n, dtype, gates, psi=psi, tile_bits=k, flags=flags)
    want = orc.run(n, gates, psi.copy())
    assert dist(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_random_circuit_16q_fused(qvlib, orc, cuda, dtype):
    qv = qvlib
    n = 16
    gates = W.random_circuit(n, 20, W.config_seed(0))
    want = orc.run(n, gates)
    for k in (10, 11, 12):
        for flags in (0, 2):
            got = run_gpu(qv, n, dtype, gates, tile_bits=k, flags=flags)
            assert dist(got, want) <= TOL[dtype], (k, flags)


@pytest.mark.parametrize("n", [10, 12, 15])
def test_qft_closed_form_fused(qvlib, cuda, n):
    qv = qvlib
    N = 1 << n
    gates = W.qft_circuit(n)
    for j in (1, N - 1, (3 * N) // 7):
        k = np.arange(N)
        want = np.exp(2j * np.pi * ((j * k) % N) / N) / math.sqrt(N)
        for dtype in (0, 1):
            got = run_gpu(qv, n, dtype, gates, basis=j)
            assert dist(got, want) <= (1e-5 if dtype == 0 else 1e-12)


def test_ansatz_fused(qvlib, orc, cuda):
    qv = qvlib
    n = 14
    gates, _ = W.ansatz_circuit(n, 6, W.config_seed(2, 3))
    want = orc.run(n, gates)
    got = run_gpu(qv, n, 0, gates)
    assert dist(got, want) <= 1e-5


def test_ghz_fused(qvlib, cuda):
    qv = qvlib
    n = 20
    got = run_gpu(qv, n, 0, W.ghz_circuit(n))
    assert abs(got[0] - 1 / math.sqrt(2)) < 1e-6 and abs(got[-1] - 1 / math.sqrt(2)) < 1e-6
    assert np.sum(np.abs(got[1:-1])) == 0


@pytest.mark.parametrize("n", [10, 13, 18])
def test_permute_qubits_fused(qvlib, orc, cuda, n):
    qv = qvlib
    rng = W.SplitMix64(n + 1)
    psi = W.random_state(n, 4)
    for _ in range(3):
        perm = [int(x) for x in np.argsort(rng.uniform(n))]
        h = qv.qv_create(n, 1)
        qv.qv_set_state(h, psi)
        qv.qv_permute_qubits(h, perm)
        got = qv.qv_get_state(h)
        qv.qv_destroy(h)
        assert dist(got, orc.permute(psi, perm)) <= 1e-14


def test_fused_equals_plain_22q(qvlib, orc, cuda):
    """Same seeded circuit through both GPU paths and the oracle at 22 qubits."""
    qv = qvlib
    n = 22
    gates = W.random_circuit(n, 8, seed=77)
    fused = run_gpu(qv, n, 0, gates, mode=qv.QV_MODE_FUSED)
    plain = run_gpu(qv, n, 0, gates, mode=qv.QV_MODE_PLAIN)
    want = orc.run(n, gates)
    assert dist(fused, want) <= 1e-5
    assert dist(plain, want) <= 1e-5
    assert dist(fused, plain.astype(np.complex128)) <= 1e-5


def test_fused_reports_bad_tile_bits(qvlib, cuda):
    qv = qvlib
    h = qv.qv_create(11, 0)
    with pytest.raises(qv.QvError):
        qv.qv_apply_circuit(h, [Gate("h", 0)], mode=qv.QV_MODE_FUSED, tile_bits=13)
    with pytest.raises(qv.QvError):
        qv.qv_apply_circuit(h, [Gate("h", 0)], mode=qv.QV_MODE_FUSED, tile_bits=12)   # > n
    qv.qv_destroy(h)


def pair_heavy_circuit(n, pairs, reps, seed):
    """Dense runs of gates on two qubits (U3 on each, CNOT both ways, CZ, RZ,
    controlled U3), the shape the 4x4 pair ops absorb, with a few gates on
    other qubits between the runs."""
    rng = W.SplitMix64(seed)
    gates = []
    for r in range(reps):
        for a, b in pairs:
            th = rng.uniform(9) * 2 * math.pi
            gates += [Gate("u3", a, theta=tuple(th[0:3])), Gate("u3", b, theta=tuple(th[3:6])),
                      Gate("x", b, ctrl=a), Gate("rz", a, theta=(th[6], 0, 0)), Gate("z", a, ctrl=b),
                      Gate("u3", b, ctrl=a, theta=tuple(th[6:9])), Gate("x", a, ctrl=b),
                      Gate("u3", a, theta=tuple(th[1:4])), Gate("h", b)]
        gates.append(Gate("h", (r * 5) % n))
    return gates


@pytest.mark.parametrize("n,k,pairs", [(12, 10, [(6, 7)]), (14, 12, [(1, 2), (9, 13)]),
                                       (16, 11, [(5, 15), (3, 4)]), (13, 12, [(0, 1), (7, 12)])])
def test_pair_ops_fused(qvlib, orc, cuda, n, k, pairs):
    """4x4 pair ops (complex64 compiled passes) against the oracle and against
    the same plan without them; the planner must actually form pair ops."""
    qv = qvlib
    gates = pair_heavy_circuit(n, pairs, 6, seed=77 + n)
    with_pairs = qv.qv_plan_cost(n, 0, gates, tile_bits=k)["flops"]
    without = qv.qv_plan_cost(n, 0, gates, tile_bits=k, flags=qv.QV_PLAN_NO_PAIRS)["flops"]
    assert with_pairs < without
    psi = W.random_state(n, 5 * n + k)
    want = orc.run(n, gates, psi.copy())
    got = run_gpu(qv, n, 0, gates, psi=psi, tile_bits=k)
    got_np = run_gpu(qv, n, 0, gates, psi=psi, tile_bits=k, flags=qv.QV_PLAN_NO_PAIRS)
    assert dist(got, want) <= TOL[0]
    assert dist(got_np, want) <= TOL[0]


def test_plan_cache_follows_the_gate_list(qvlib, orc, cuda):
    """The handle keeps the last plan and compiled program; a changed angle,
    gate list, tile size or flag must re-plan, the same list must reuse."""
    qv = qvlib
    n = 14
    g1 = W.random_circuit(n, 6, W.config_seed(0, 11))
    g2 = W.random_circuit(n, 6, W.config_seed(0, 12))          # same structure, other angles
    g3 = W.random_gate_list(n, 80, seed=5, ctrl_prob=0.3)      # other structure
    g1b = list(g1)
    g1b[7] = g1b[7]._replace(theta=(g1b[7].theta[0] + 1e-3, g1b[7].theta[1], g1b[7].theta[2]))  # one angle moved
    h = qv.qv_create(n, 0)
    try:
        for gates, tb, flags in [(g1, 0, 0), (g1, 0, 0), (g2, 0, 0), (g1, 0, 0), (g1b, 0, 0), (g3, 0, 0),
                                 (g3, 10, 0), (g3, 10, qv.QV_PLAN_NO_PAIRS), (g1, 11, 0), (g1, 0, 0)]:
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, gates, mode=2, tile_bits=tb, flags=flags)
            assert dist(qv.qv_get_state(h), orc.run(n, gates)) <= TOL[0], (tb, flags)
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
def test_host_memory_state(qvlib, orc, cuda, dtype):
    """A state kept in mapped host memory (the slower tier behind NVLink-C2C)
    goes through the same kernels: fused and per-gate circuits, reductions,
    the adjoint gradient, and distance to a device-memory copy."""
    qv = qvlib
    n = 17
    gates = W.random_gate_list(n, 150, seed=31, ctrl_prob=0.3)
    psi = W.random_state(n, 8)
    want = orc.run(n, gates, psi.copy())
    hd = qv.qv_create(n, dtype)
    for mode in (qv.QV_MODE_FUSED, qv.QV_MODE_PLAIN):
        hh = qv.qv_create(n, dtype, flags=qv.QV_ALLOC_HOST)
        qv.qv_set_state(hh, psi)
        qv.qv_apply_circuit(hh, gates, mode=mode)
        got = qv.qv_get_state(hh)
        assert dist(got, want) <= TOL[dtype], mode
        z, _ = qv.qv_expect_z(hh)
        ref = got.astype(np.complex128)
        assert np.max(np.abs(np.asarray(z) - orc.expect_z(ref))) <= (1e-6 if dtype == 0 else 1e-12)
        qv.qv_set_state(hd, psi)
        qv.qv_apply_circuit(hd, gates, mode=mode)
        assert qv.qv_distance(hh, hd) <= 2 * TOL[dtype]
        qv.qv_destroy(hh)
    # adjoint with psi in host memory (lambda stays on the device)
    ag, npar = W.ansatz_circuit(12, 2, W.config_seed(3, 9))
    terms = W.ansatz_hamiltonian(12)
    hh = qv.qv_create(12, dtype, flags=qv.QV_ALLOC_HOST)
    g, e = qv.qv_adjoint_grad(hh, ag, terms, npar)
    ref = orc.param_shift_grad(12, ag, terms, npar)
    assert np.max(np.abs(g - ref)) <= (1e-4 if dtype == 0 else 1e-10)
    qv.qv_destroy(hh)
    qv.qv_destroy(hd)


@pytest.mark.parametrize("n", [24, 28])
@pytest.mark.parametrize("k", [10, 11, 12])
def test_qft_with_swaps_large(qvlib, cuda, n, k):
    """QFT with its final qubit-reversal SWAPs on states of many tiles. The
    SWAPs become relabels that can leave a pass with a single stage; its
    warps must not store into positions other warps still have to load
    (this caught such a race)."""
    qv = qvlib
    j = int(W.SplitMix64(W.config_seed(4, 98)).integers(0, (1 << n) - 1, 1)[0])
    h = qv.qv_create(n, 0)
    try:
        qv.qv_set_basis(h, j)
        qv.qv_apply_circuit(h, W.qft_circuit(n), mode=qv.QV_MODE_FUSED, tile_bits=k)
        assert qv.qv_verify_qft(h, j) <= 1e-5
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("k", [10, 12])
def test_permutation_passes_24q(qvlib, orc, cuda, k):
    """Pure relabel passes (random qubit permutations) on a 24-qubit state,
    against the oracle's index permutation."""
    qv = qvlib
    n = 24
    psi = W.random_state(n, 91)
    rng = W.SplitMix64(17)
    h = qv.qv_create(n, 0)
    try:
        qv.qv_set_state(h, psi)
        want = psi.astype(np.complex64).astype(np.complex128)
        for rep in range(3):
            perm = [int(x) for x in np.argsort(rng.uniform(n))]
            qv.qv_permute_qubits(h, perm)
            want = orc.permute(want, perm)
        assert dist(qv.qv_get_state(h), want) <= 1e-6
    finally:
        qv.qv_destroy(h)


@pytest.mark.parametrize("n,k", [(11, 10), (14, 11), (20, 12)])
def test_sign_flip_ops(qvlib, orc, cuda, n, k):
    """Diagonal ops of +1 / -1 entries (Z, CZ) run as sign-bit flips: Z and CZ
    on every kind of target and control position (register bits, the packed
    lane qubit 0, thread bits, qubits outside the tile), between layers of
    random rotations, on a random state; the result equals the oracle's."""
    qv = qvlib
    rot = W.random_gate_list(n, 2 * n, seed=300 + n, kinds=("u3", "ry", "h"), ctrl_prob=0.0)
    signs = []
    for q in range(n):
        signs.append(Gate("z", q))
        for c in (0, (q + 1) % n, (q + n // 2) % n, n - 1):
            if c != q:
                signs.append(Gate("z", q, ctrl=c))
    gates = rot + signs + rot[::-1] + signs[::3] + W.random_gate_list(n, n, seed=700 + n, kinds=("u3",))
    psi = W.random_state(n, 50 + n)
    got = run_gpu(qv, n, 0, gates, psi=psi, tile_bits=k)
    want = orc.run(n, gates, psi.copy())
    assert dist(got, want) <= TOL[0]
    # the same circuit through the per-gate kernels
    plain = run_gpu(qv, n, 0, gates, psi=psi, mode=1)
    assert dist(got, plain) <= TOL[0]
