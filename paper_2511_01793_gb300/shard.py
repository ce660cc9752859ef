"""A minibatch split across ranks (one process per GPU), host side.

Every rank holds the whole object, probe and data of one reconstruction in its
own context.  For each minibatch the slots 0..b-1 are cut into contiguous
shares of ceil(b / world) slots; rank r steps its share (emg_shard_step), the
ranks all-gather the per-slot results z~_k, Q~_k and max|z_k|^2, and every rank
combines all b slots in slot order (emg_shard_apply).  The combine therefore
sees exactly what it sees on one GPU, in the same order, and every rank ends
each minibatch with bitwise the state that emg_step_minibatch gives.

The exchange is the only collective on the data path: per minibatch it moves
b m^2 16 + 4 b bytes (the patches of all slots).  This module holds only the
partition and the exchange; every step of the method runs in the library.
"""
from __future__ import annotations

import math
from typing import List, Optional, Tuple

import numpy as np

from . import emg_shard_apply, emg_shard_step


def slot_ranges(b: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous shares of the slots 0..b-1: rank r gets [r c, min(b, (r + 1) c)), c = ceil(b / world)."""
    if b < 0 or world < 1:
        raise ValueError("need b >= 0 and world >= 1")
    c = max(1, math.ceil(b / world))
    return [(min(b, r * c), min(b, (r + 1) * c)) for r in range(world)]


def padded_slots(b: int, world: int) -> int:
    """Slots a buffer needs so that each rank's share is one equal-sized piece (world ceil(b / world))."""
    return world * max(1, math.ceil(b / world))


def exchange_slots(buffers, b: int, world: int, rank: int, group=None) -> None:
    """All-gathers each rank's share of every buffer (leading dimension = slots) in place.

    After the call every rank's buffers hold the shares of all ranks.  Works
    with any torch.distributed backend (NCCL on GPUs, gloo on CPU tensors).
    """
    if world == 1:
        return
    import torch
    import torch.distributed as dist

    c = max(1, math.ceil(b / world))
    for t in buffers:
        if t.is_complex():
            t = torch.view_as_real(t)
        pieces = list(t[:world * c].split(c))
        mine = t[rank * c:(rank + 1) * c].clone()
        dist.all_gather(pieces, mine, group=group)


class ShardedReconstruction:
    """One rank's side of a reconstruction whose minibatches are split across ranks.

    ``ctx`` is this rank's ``Context`` (same data, parameters and initial state
    on every rank).  ``step(idx)`` runs one minibatch; ``run_epoch(order)`` runs
    the consecutive minibatches of one permutation.  The slot buffers are torch
    tensors on the context's device; the collectives are issued on the
    context's stream.
    """

    def __init__(self, ctx, world: int, rank: int, group=None):
        import torch

        self.ctx, self.world, self.rank, self.group = ctx, world, rank, group
        B = ctx.params.minibatch
        slots = padded_slots(B, world)
        m = ctx.m
        dev = ctx.obj.device
        self.zt = torch.zeros((slots, m, m), dtype=torch.complex64, device=dev)
        self.qt = torch.zeros((slots, m, m), dtype=torch.complex64, device=dev)
        self.mu = torch.zeros((slots,), dtype=torch.float32, device=dev)

    def step(self, idx) -> None:
        import torch

        idx = np.ascontiguousarray(idx, dtype=np.int32)
        b = len(idx)
        s0, s1 = slot_ranges(b, self.world)[self.rank]
        ptrs = (self.zt.data_ptr(), self.qt.data_ptr(), self.mu.data_ptr())
        emg_shard_step(self.ctx.ctx, idx, s0, s1, *ptrs)
        with torch.cuda.stream(self.ctx.stream):
            exchange_slots((self.zt, self.qt, self.mu), b, self.world, self.rank, self.group)
        emg_shard_apply(self.ctx.ctx, idx, *ptrs)

    def run_epoch(self, order, minibatch: Optional[int] = None) -> None:
        B = minibatch or self.ctx.params.minibatch
        order = np.asarray(order, dtype=np.int32)
        for b0 in range(0, len(order), B):
            self.step(order[b0:b0 + B])
