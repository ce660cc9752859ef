"""The host side of a minibatch split across ranks, on CPU with gloo ranks.

paper_2511_01793_gb300.shard cuts a minibatch's slots into contiguous shares,
one per rank, and all-gathers the per-slot results in place.  These tests run
2 and 3 gloo ranks as processes: each rank fills only its own share of the
slot buffers (z~_k, Q~_k, mu_k stand-ins), the exchange runs, and every rank
must then hold exactly the buffers of a single rank that computed every slot,
so the combine that follows sees the same inputs in the same order on every
rank and for every rank count.
"""
import os
import socket

import numpy as np
import pytest

from paper_2511_01793_gb300.shard import padded_slots, slot_ranges


def test_slot_ranges_partition_the_minibatch():
    for b in (1, 2, 4, 7, 63, 64, 256):
        for world in (1, 2, 3, 4, 8):
            r = slot_ranges(b, world)
            assert len(r) == world
            covered = [k for s0, s1 in r for k in range(s0, s1)]
            assert covered == list(range(b))                     # contiguous, in order, disjoint
            sizes = [s1 - s0 for s0, s1 in r]
            assert max(sizes) - min(s for s in sizes if s > 0) <= max(1, -(-b // world))
            assert padded_slots(b, world) >= b and padded_slots(b, world) % world == 0


def _slot_data(b, m, seed):
    """Deterministic stand-ins of one minibatch's per-slot results."""
    rng = np.random.default_rng(seed)
    zt = (rng.standard_normal((b, m, m)) + 1j * rng.standard_normal((b, m, m))).astype(np.complex64)
    qt = (rng.standard_normal((b, m, m)) + 1j * rng.standard_normal((b, m, m))).astype(np.complex64)
    mu = rng.uniform(0.5, 2.0, b).astype(np.float32)
    mu[::5] = 0.0                                             # empty patches drop out of the probe mean
    return zt, qt, mu


def _combine(zt, qt, mu):
    """A fixed-order combine of the slots (slot order), as the library's combine sums them."""
    num = np.zeros(zt.shape[1:], dtype=np.complex64)
    qs = np.zeros(qt.shape[1:], dtype=np.complex64)
    n = 0
    for k in range(len(zt)):
        num = num + zt[k]
        if mu[k] > 0:
            qs = qs + qt[k]
            n += 1
    return num, qs, n


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2511_01793_gb300.shard import exchange_slots

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = 8
    try:
        for b in (64, 7, 4, 1):
            zt_all, qt_all, mu_all = _slot_data(b, m, seed=b)
            slots = padded_slots(64, world)
            zt = torch.full((slots, m, m), complex(np.nan, np.nan), dtype=torch.complex64)
            qt = torch.full((slots, m, m), complex(np.nan, np.nan), dtype=torch.complex64)
            mu = torch.full((slots,), np.nan, dtype=torch.float32)
            s0, s1 = slot_ranges(b, world)[rank]
            zt[s0:s1] = torch.from_numpy(zt_all[s0:s1])            # this rank's share only
            qt[s0:s1] = torch.from_numpy(qt_all[s0:s1])
            mu[s0:s1] = torch.from_numpy(mu_all[s0:s1])
            exchange_slots((zt, qt, mu), b, world, rank)
            got = (zt[:b].numpy(), qt[:b].numpy(), mu[:b].numpy())
            ok = all(np.array_equal(g, e) for g, e in zip(got, (zt_all, qt_all, mu_all)))
            c_got, c_ref = _combine(*got), _combine(zt_all, qt_all, mu_all)
            ok = ok and np.array_equal(c_got[0], c_ref[0]) and np.array_equal(c_got[1], c_ref[1]) \
                and c_got[2] == c_ref[2]
            with open(os.path.join(out_dir, f"r{rank}_b{b}"), "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_gives_every_rank_the_single_rank_buffers(tmp_path, world):
    import torch.multiprocessing as mp

    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        for b in (64, 7, 4, 1):
            assert (tmp_path / f"r{rank}_b{b}").read_text() == "ok", (rank, b)
