"""A state split over the ranks of a process group (Sec. III-D, Eq. 9).

Rank r of C = 2^g ranks holds the contiguous amplitudes [r 2^n / C,
(r + 1) 2^n / C - 1]. The schedule (which gates run locally, where a global
qubit is exchanged with local qubit L - 1, the final qubit order) comes from the
library (``qv_dist_plan``); this module moves the half shards between ranks
with ``torch.distributed`` and runs the local steps through the C ABI on the
rank's own GPU. There is no CPU fallback: a local step always runs in the
library's kernels. ``run_schedule`` takes the local executor as an argument so
that the exchange protocol is the same whatever executes the local steps.
"""
from __future__ import annotations

import math
from typing import Callable, List

from . import qv


def global_bits(world: int) -> int:
    g = int(round(math.log2(world)))
    if (1 << g) != world or world < 2:
        raise ValueError("the split needs a power-of-two number of ranks >= 2, got %d" % world)
    return g


def exchange_half(shard, peer: int, send_upper: bool, group=None):
    """Trades one half of ``shard`` (a 1-D tensor of the rank's amplitudes, any
    element type) with rank ``peer``: this rank's upper half when send_upper,
    else its lower half, replaced by the partner's half of the same size. The
    received half lands in a buffer of this rank's own memory first."""
    import torch
    import torch.distributed as dist
    h = shard.numel() // 2
    mine = shard[h:] if send_upper else shard[:h]
    recv = torch.empty_like(mine)
    ops = [dist.P2POp(dist.isend, mine.contiguous(), peer, group), dist.P2POp(dist.irecv, recv, peer, group)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    mine.copy_(recv)


def run_schedule(n: int, rank: int, world: int, gates, shard, apply_local: Callable, group=None,
                 restore: bool = False) -> List[int]:
    """Runs ``gates`` on this rank's ``shard``: local steps through
    ``apply_local((gate array, count))``, exchanges with ``exchange_half``.
    Returns final_perm (logical qubit q sits at physical qubit final_perm[q];
    the identity with ``restore``)."""
    g = global_bits(world)
    steps, (lg, _), perm = qv.qv_dist_plan(n, g, rank, gates, restore)
    import ctypes
    base = ctypes.addressof(lg)
    size = ctypes.sizeof(qv.qv_gate)
    for st in steps:
        if st["kind"] == "local":
            b, e = st["begin"], st["end"]
            arr = (qv.qv_gate * (e - b)).from_address(base + b * size)
            apply_local((arr, e - b))
        else:
            exchange_half(shard, st["peer"], st["send_upper"], group)
    return perm


class DistState:
    """An n-qubit complex64 state split over the ranks of the default process
    group, one shard per rank on its current CUDA device (a torch tensor of
    2^(n - g) complex64 wrapped with qv_wrap). ``apply`` runs a circuit with
    exchanges over NCCL; ``perm`` tracks where each logical qubit sits."""

    def __init__(self, n: int, group=None):
        import torch
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.g = global_bits(self.world)
        if n - self.g < 1:
            raise ValueError("n too small for %d ranks" % self.world)
        self.n, self.L = n, n - self.g
        self.shard = torch.zeros(1 << self.L, dtype=torch.complex64, device="cuda")
        if self.rank == 0:
            self.shard[0] = 1.0
        self.h = qv.qv_wrap(self.shard.data_ptr(), self.L, qv.QV_C64, torch.cuda.current_stream())
        self.perm = list(range(n))

    def apply(self, gates, mode: int = qv.QV_MODE_AUTO, restore: bool = True):
        """Applies ``gates`` (logical qubits) from the natural qubit order; with
        ``restore`` (the default) the state ends in the natural order again,
        else ``perm`` says where each logical qubit sits and the next apply()
        refuses to start."""
        if self.perm != list(range(self.n)):
            raise RuntimeError("apply() starts from the natural qubit order")
        flat = self.shard.view(-1)
        self.perm = run_schedule(self.n, self.rank, self.world, gates, flat,
                                 lambda arr: qv.qv_apply_circuit(self.h, arr, mode), self.group, restore)

    def close(self):
        if self.h:
            qv.qv_destroy(self.h)
            self.h = None
