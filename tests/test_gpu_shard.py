"""A minibatch split across ranks, the ranks emulated one after another on one GPU.

Each emulated rank has its own context on the same data and initial state.
Rank r steps its share of the minibatch's slots (emg_shard_step) into one set
of slot buffers that all ranks write, which leaves those buffers exactly as the
all-gather of the multi-GPU path would (tests/test_shard_cpu.py checks that
exchange on gloo ranks).  Every rank then combines from them
(emg_shard_apply).  No kernel waits on another rank: the ranks run in turn.
Every rank must end each minibatch with bitwise the state of
emg_step_minibatch on one context, for 2, 3 and 4 ranks, shares that are empty
(b < ranks) included, over several minibatches and a whole epoch.
"""
import numpy as np
import pytest

from emg_cases import Case, make_context, oracle_params, state

pytestmark = pytest.mark.gpu


def _run_split(lib, ctxs, idx, buffers):
    from paper_2511_01793_gb300.shard import slot_ranges

    world = len(ctxs)
    zt, qt, mu = buffers
    for r, c in enumerate(ctxs):
        s0, s1 = slot_ranges(len(idx), world)[r]
        lib.emg_shard_step(c.ctx, idx, s0, s1, zt.data_ptr(), qt.data_ptr(), mu.data_ptr())
    for c in ctxs:
        lib.emg_shard_apply(c.ctx, idx, zt.data_ptr(), qt.data_ptr(), mu.data_ptr())


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("m,levels,prolong,B", [(64, 3, "bilinear", 10), (128, 3, "bilinear", 9), (32, 1, "const", 7)])
def test_split_minibatches_equal_the_one_gpu_step_bitwise(lib, world, m, levels, prolong, B):
    import torch

    from paper_2511_01793_gb300.shard import padded_slots

    case = Case(n=2 * m + 40, m=m, side=5, noise_peak=1e4, seed=400 + m + world)
    p = oracle_params(minibatch=B, levels=levels, prolong=prolong)
    ref = make_context(lib, case, p, seed=9)
    ranks = [make_context(lib, case, p, seed=9) for _ in range(world)]
    slots = padded_slots(B, world)
    buffers = (torch.zeros((slots, m, m), dtype=torch.complex64, device="cuda"),
               torch.zeros((slots, m, m), dtype=torch.complex64, device="cuda"),
               torch.zeros((slots,), dtype=torch.float32, device="cuda"))
    rng = np.random.default_rng(world)
    order = rng.permutation(case.n_pos).astype(np.int32)
    # minibatches of B, then a short one with fewer positions than ranks (empty shares)
    batches = [order[:B], order[B:2 * B], order[2 * B:2 * B + 1]]
    for idx in batches:
        lib.emg_step_minibatch(ref.ctx, idx)
        _run_split(lib, ranks, idx, buffers)
        z_r, q_r = state(ref)
        for c in ranks:
            z, q = state(c)
            assert np.array_equal(z, z_r) and np.array_equal(q, q_r)
    for c in [ref] + ranks:
        c.close()


def test_split_epoch_equals_run_epochs_bitwise(lib):
    import torch

    from paper_2511_01793_gb300.shard import padded_slots

    m, B, world = 64, 8, 3
    case = Case(n=2 * m + 40, m=m, side=6, noise_peak=1e4, seed=450)
    p = oracle_params(minibatch=B, levels=2, prolong="bilinear")
    ref = make_context(lib, case, p, seed=11)
    ranks = [make_context(lib, case, p, seed=11) for _ in range(world)]
    order = np.random.default_rng(2).permutation(case.n_pos).astype(np.int32)
    lib.emg_run_epochs(ref.ctx, 1, order[None, :])
    slots = padded_slots(B, world)
    buffers = (torch.zeros((slots, m, m), dtype=torch.complex64, device="cuda"),
               torch.zeros((slots, m, m), dtype=torch.complex64, device="cuda"),
               torch.zeros((slots,), dtype=torch.float32, device="cuda"))
    for b0 in range(0, len(order), B):
        _run_split(lib, ranks, order[b0:b0 + B], buffers)
    z_r, q_r = state(ref)
    for c in ranks:
        z, q = state(c)
        assert np.array_equal(z, z_r) and np.array_equal(q, q_r)
    for c in [ref] + ranks:
        c.close()


def test_split_minibatch_rejects_the_atomic_scatter_and_bad_ranges(lib):
    import torch

    case = Case(n=104, m=32, side=4, seed=460)
    p = oracle_params(minibatch=6)
    c = make_context(lib, case, p, scatter=lib.EMG_SCATTER_ATOMIC)
    buf = torch.zeros((6, 32, 32), dtype=torch.complex64, device="cuda")
    mu = torch.zeros(6, dtype=torch.float32, device="cuda")
    idx = np.arange(6, dtype=np.int32)
    with pytest.raises(lib.EmgError):
        lib.emg_shard_step(c.ctx, idx, 0, 3, buf.data_ptr(), buf.data_ptr(), mu.data_ptr())
    c.close()
    c = make_context(lib, case, p)
    for s0, s1 in ((-1, 2), (3, 2), (0, 7)):
        with pytest.raises(lib.EmgError):
            lib.emg_shard_step(c.ctx, idx, s0, s1, buf.data_ptr(), buf.data_ptr(), mu.data_ptr())
    c.close()
