"""The state split of Sec. III-D (Eq. 9) on gloo ranks on the CPU.

Each rank holds its contiguous range of a random state; the library's schedule
(qv_dist_plan) says which gates run on the shard and when a global qubit is
exchanged with local qubit L - 1; ``dist.exchange_half`` trades the half shards
between ranks over gloo (host buffers). The local steps run in the oracle (an
L-qubit state per rank: test infrastructure standing in for the GPU here). The
shards, gathered and put back in logical qubit order, must equal the oracle's
run of the whole circuit on the whole state: every pair sees the same
arithmetic, so the two agree to the last bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _circuit(n, seed):
    from paper_2508_15545_gb300 import workloads as W
    return W.random_gate_list(n, 160, seed=seed, ctrl_prob=0.4) + W.random_circuit(n, 3, W.config_seed(0, seed)) + \
        W.qft_circuit(n)


def _to_gates(arr_ng):
    """qv_gate records of a local step -> workload gate records (for the oracle)."""
    from paper_2508_15545_gb300 import qv, workloads as W
    arr, ng = arr_ng
    names = {v: k for k, v in qv.KIND.items()}
    out = []
    for k in range(ng):
        x = arr[k]
        kind = names[int(x.kind)]
        mat = tuple(complex(x.u[e].re, x.u[e].im) for e in range(4)) if kind == "matrix" else None
        out.append(W.Gate(kind, int(x.target), target2=int(x.target2), ctrl=int(x.ctrl),
                          theta=(float(x.theta[0]), float(x.theta[1]), float(x.theta[2])), matrix=mat))
    return out


def _rank(rank, world, port, n, seed, restore, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2508_15545_gb300 import dist as D, workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = n - D.global_bits(world)
        psi0 = W.random_state(n, seed)
        shard = np.ascontiguousarray(psi0[rank << L:(rank + 1) << L])
        t = torch.from_numpy(shard.view(np.float64))        # the exchange moves raw amplitude bytes
        gates = _circuit(n, seed)

        def local(arr_ng):
            O.run(L, _to_gates(arr_ng), shard)

        perm = D.run_schedule(n, rank, world, gates, t, local, restore=restore)
        parts = [torch.empty_like(t) for _ in range(world)] if rank == 0 else None
        dist.gather(t, parts, dst=0)
        if rank == 0:
            phys = np.concatenate([p.numpy().view(np.complex128) for p in parts])
            q.put(("ok", phys, perm))
        else:
            q.put(("ok", None, perm))
    except Exception as e:  # noqa: BLE001
        q.put(("error", repr(e), None))
    finally:
        dist.destroy_process_group()


def _logical(phys, perm):
    """State in logical qubit order: bit q of the logical index is bit perm[q] of the physical one."""
    n = len(perm)
    i = np.arange(1 << n, dtype=np.int64)
    src = np.zeros_like(i)
    for q, p in enumerate(perm):
        src |= ((i >> q) & 1) << p
    return phys[src]


@pytest.mark.parametrize("restore", [False, True])
@pytest.mark.parametrize("world,n", [(2, 9), (4, 10)])
def test_split_state_matches_oracle(orc, world, n, restore):
    seed = 40 + world
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, seed, restore, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    errs = [r for r in res if r[0] != "ok"]
    assert not errs, errs
    perms = [r[2] for r in res]
    assert all(p == perms[0] for p in perms)                # every rank ends in the same qubit order
    if restore:
        assert perms[0] == list(range(n))                    # back in the natural order
    phys = next(r[1] for r in res if r[1] is not None)
    from paper_2508_15545_gb300 import workloads as W
    want = orc.run(n, _circuit(n, seed), W.random_state(n, seed))
    got = _logical(phys, perms[0])
    assert np.array_equal(got, want) or np.linalg.norm(got - want) <= 1e-13


@pytest.mark.parametrize("g", [1, 2, 3])
def test_schedule_pairs_ranks_consistently(qvlib, g):
    """For every rank of 2^g: the same step kinds in the same order; at an
    exchange, partners name each other, trade opposite halves, and differ
    exactly in the exchanged global bit. Controls and diagonal gates on global
    qubits never need an exchange."""
    qv = qvlib
    from paper_2508_15545_gb300 import workloads as W
    n = 12
    gates = _circuit(n, 7)
    plans = [qv.qv_dist_plan(n, g, r, gates) for r in range(1 << g)]
    kinds = [[s["kind"] for s in p[0]] for p in plans]
    assert all(k == kinds[0] for k in kinds)
    for r, (steps, _, perm) in enumerate(plans):
        assert sorted(perm) == list(range(n))
        for k, s in enumerate(steps):
            if s["kind"] != "exchange":
                continue
            peer = s["peer"]
            ps = plans[peer][0][k]
            assert peer == r ^ (1 << s["global_bit"]) and ps["peer"] == r
            assert ps["global_bit"] == s["global_bit"] and ps["send_upper"] != s["send_upper"]
            assert s["send_upper"] == (((r >> s["global_bit"]) & 1) == 0)
    # a circuit of diagonal gates and controls on the global qubits: no exchange at all
    top = list(range(n - g, n))
    diag = [W.Gate("rz", t, theta=(0.3 * t, 0, 0)) for t in top] + \
           [W.Gate("x", 0, ctrl=t) for t in top] + [W.Gate("p", top[0], ctrl=1, theta=(0.7, 0, 0))]
    for r in range(1 << g):
        steps, _, _ = qv.qv_dist_plan(n, g, r, diag)
        assert all(s["kind"] == "local" for s in steps)
    # a segment whose gates are all controlled by a global qubit is empty on the
    # ranks where that qubit is 0, but still a step there
    gated = [W.Gate("u3", 2, ctrl=n - 1, theta=(0.4, 0.1, 0.2)), W.Gate("x", 1, ctrl=n - 1), W.Gate("h", n - 1),
             W.Gate("u3", 3, ctrl=n - 2, theta=(0.3, 0.2, 0.1))]
    seqs = [qv.qv_dist_plan(n, g, r, gated)[0] for r in range(1 << g)]
    assert all([s["kind"] for s in q] == [s["kind"] for s in seqs[0]] for q in seqs)
    size = [q[0]["end"] - q[0]["begin"] for q in seqs]
    assert size[0] < size[-1]            # the controlled gates fell away on rank 0, the step did not


def test_schedule_rejects_bad_arguments(qvlib):
    qv = qvlib
    from paper_2508_15545_gb300 import workloads as W
    gates = W.random_circuit(8, 2, 1)
    for g, r in ((0, 0), (8, 0), (2, 4), (1, -1)):
        with pytest.raises(qv.QvError):
            qv.qv_dist_plan(8, g, r, gates)
