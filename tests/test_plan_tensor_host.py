"""Host-side checks of the tensor-core plans (QV_PLAN_TENSOR), no GPU.

The planner's output -- per pass the tile's physical qubits, per stage the
register and thread layouts and one 16x16 matrix (two where a qubit outside the
tile selects one) -- is replayed here in numpy on a small state, exactly as the
tensor-core kernel would move and multiply the data, and compared with the
oracle (Eq. 3 gate by gate, Eq. 5). A wrong matrix product, embedding, layout or
SWAP relabel shows up as a distance far above rounding."""
import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W
from paper_2508_15545_gb300.workloads import Gate


@pytest.fixture(scope="module")
def qv(qvlib):
    return qvlib


def deposit(v, positions):
    """Integer whose bit positions[b] is bit b of v (v may be an array)."""
    out = np.zeros_like(v)
    for b, p in enumerate(positions):
        out |= ((v >> b) & 1) << p
    return out


def replay(qv, n, gates, tile_bits, psi):
    """Applies the tensor-core plan of `gates` to psi (complex128) in numpy."""
    arr = (qv.gates_to_c(gates), len(gates))
    flags = qv.QV_PLAN_TENSOR
    npass = qv.qv_plan_info(n, 0, arr, tile_bits, flags)["passes"]
    psi = psi.copy()
    for p in range(npass):
        first = qv.qv_plan_tc_stage(n, arr, p, 0, tile_bits)
        k = first["k"]
        tq = np.array(first["tile_qubit"], dtype=np.int64)
        outside = [q for q in range(n) if q not in set(tq.tolist())]
        B, T = 1 << (n - k), 1 << (k - 4)
        b = np.arange(B, dtype=np.int64)
        base = deposit(b, outside)                               # (B,)
        t = np.arange(T, dtype=np.int64)
        r = np.arange(16, dtype=np.int64)

        def phys(tile_pos):                                      # tile positions -> physical index bits
            return deposit(tile_pos, tq)

        for s in range(first["nstages"]):
            st = qv.qv_plan_tc_stage(n, arr, p, s, tile_bits)
            lin = deposit(t, st["in_thr"])[:, None] | deposit(r, st["in_reg"])[None, :]     # (T, 16)
            lout = deposit(t, st["out_thr"])[:, None] | deposit(r, st["out_reg"])[None, :]
            iin = base[:, None, None] | phys(lin)[None]
            iout = base[:, None, None] | phys(lout)[None]
            x = psi[iin]                                                                   # (B, T, 16)
            if st["has_matrix"]:
                v = ((base >> st["ext"]) & 1) if st["ext"] >= 0 else np.zeros(B, dtype=np.int64)
                M = st["m"][v]                                                             # (B, 16, 16)
                x = np.einsum("bij,btj->bti", M, x)
            new = np.empty_like(psi)
            new[iout] = x
            psi = new
    return psi


CASES = [
    ("random circuit", 13, lambda n: W.random_circuit(n, 8, W.config_seed(0, 3))),
    ("random circuit", 12, lambda n: W.random_circuit(n, 10, W.config_seed(0, 4))),
    ("every gate kind", 13, lambda n: W.random_gate_list(n, 150, seed=77)),
    ("every gate kind", 12, lambda n: W.random_gate_list(n, 200, seed=78, ctrl_prob=0.5)),
    ("qft with swaps", 13, lambda n: W.qft_circuit(n)),
    ("ansatz", 12, lambda n: W.ansatz_circuit(n, 4, W.config_seed(2, 1))[0]),
]


@pytest.mark.parametrize("tile_bits", [11, 12])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tensor_plan_replays_to_the_oracle(qv, orc, case, tile_bits):
    name, n, make = CASES[case]
    gates = make(n)
    psi0 = W.random_state(n, 100 + case)
    want = orc.run(n, gates, psi0.copy())
    got = replay(qv, n, gates, tile_bits, psi0)
    assert np.linalg.norm(got - want) <= 1e-12, name


def test_tensor_plan_stage_structure(qv):
    """Load and store layouts put lanes on tile positions 0..4 and registers
    above them; every matrix is unitary for a unitary circuit; the slot cap
    holds."""
    n = 16
    gates = W.random_circuit(n, 12, W.config_seed(0, 5))
    arr = (qv.gates_to_c(gates), len(gates))
    for k in (11, 12):
        info = qv.qv_plan_info(n, 0, arr, k, qv.QV_PLAN_TENSOR)
        assert info["passes"] >= 1 and info["ops"] >= 1
        for p in range(info["passes"]):
            s0 = qv.qv_plan_tc_stage(n, arr, p, 0, k)
            last = qv.qv_plan_tc_stage(n, arr, p, s0["nstages"] - 1, k)
            for st, lay in ((s0, "in"), (last, "out")):
                assert st[lay + "_thr"][:5] == [0, 1, 2, 3, 4]
                assert min(st[lay + "_reg"]) >= 5
            slots = 0
            for s in range(s0["nstages"]):
                st = qv.qv_plan_tc_stage(n, arr, p, s, k)
                if st["has_matrix"]:
                    slots += 2 if st["ext"] >= 0 else 1
                    for v in range(2 if st["ext"] >= 0 else 1):
                        M = st["m"][v]
                        assert np.allclose(M.conj().T @ M, np.eye(16), atol=1e-12)
            assert slots <= (10 if k == 12 else 7)


def test_tensor_plan_rejects_small_tiles_and_complex128(qv):
    gates = [Gate("h", 0)]
    with pytest.raises(qv.QvError):
        qv.qv_plan_info(12, 0, gates, 10, qv.QV_PLAN_TENSOR)
    with pytest.raises(qv.QvError):
        qv.qv_plan_info(12, 1, gates, 11, qv.QV_PLAN_TENSOR)


def test_tensor_plan_30_qubit_stage_count(qv):
    """The bench circuit: fewer stages than the FP32 plan, since a stage takes
    every gate inside its four register qubits (controls included)."""
    n = 30
    gates = W.random_circuit(n, 40, W.config_seed(1))
    arr = (qv.gates_to_c(gates), len(gates))
    for k in (11, 12):
        tc = qv.qv_plan_info(n, 0, arr, k, qv.QV_PLAN_TENSOR)
        fp = qv.qv_plan_info(n, 0, arr, k)
        assert tc["stages"] < fp["stages"], (k, tc, fp)
