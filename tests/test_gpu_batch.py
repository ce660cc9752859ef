"""Batches of uneven reconstructions in one graph launch per epoch, the FFT
tiling (CTAs per position) and its autotuner."""
import numpy as np
import pytest

from emg_cases import Case, make_context, oracle_params, rel_err, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    assert t.cuda.is_available()
    return t


@pytest.mark.parametrize("m,levels,prolong,a,b", [(64, 3, "bilinear", 2, 4), (128, 2, "const", 2, 4),
                                                   (128, 3, "bilinear", 2, 4), (128, 3, "bilinear", 4, 8),
                                                   (128, 5, "const", 2, 8)])
def test_fft_tiling_does_not_change_results(lib, torch, m, levels, prolong, a, b):
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=60 + m)
    p = oracle_params(minibatch=6, levels=levels, prolong=prolong)
    c1 = make_context(lib, case, p, seed=4)
    lib.emg_set_cluster(c1.ctx, a)
    lib.emg_run_epochs(c1.ctx, 2)
    c2 = make_context(lib, case, p, seed=4)
    lib.emg_set_cluster(c2.ctx, b)
    lib.emg_run_epochs(c2.ctx, 2)
    z1, q1 = state(c1)
    z2, q2 = state(c2)
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
    c1.close()
    c2.close()


def test_single_cta_and_cluster_tilings_agree_for_small_probes(lib, torch):
    case = Case(n=104, m=32, side=4, seed=61)
    p = oracle_params(minibatch=6, levels=2)
    c1 = make_context(lib, case, p, seed=4)
    lib.emg_set_cluster(c1.ctx, 1)
    lib.emg_run_epochs(c1.ctx, 2)
    c2 = make_context(lib, case, p, seed=4)
    lib.emg_set_cluster(c2.ctx, 2)
    lib.emg_run_epochs(c2.ctx, 2)
    z1, q1 = state(c1)
    z2, q2 = state(c2)
    assert rel_err(z2, z1) <= 1e-5 and rel_err(q2, q1) <= 1e-5
    c1.close()
    c2.close()


def test_invalid_tilings_are_rejected(lib, torch):
    case = Case(n=104, m=32, side=4, seed=62)
    c = make_context(lib, case, oracle_params(minibatch=4))
    for bad in (3, 4, 8, 16):
        with pytest.raises(lib.EmgError):
            lib.emg_set_cluster(c.ctx, bad)
    c.close()


@pytest.mark.parametrize("m", [32, 128])
def test_autotune_keeps_the_state_and_the_results(lib, torch, m):
    case = Case(n=2 * m + 40, m=m, side=4, seed=63 + m)
    p = oracle_params(minibatch=6, levels=2)
    c1 = make_context(lib, case, p, seed=5)
    z0, q0 = state(c1)
    chosen, ms = lib.emg_autotune(c1.ctx)
    z_after, q_after = state(c1)
    assert np.array_equal(z0, z_after) and np.array_equal(q0, q_after)
    assert chosen in ((1, 2) if m <= 32 else (2, 4, 8)) and ms > 0
    lib.emg_run_epochs(c1.ctx, 1)
    c2 = make_context(lib, case, p, seed=5)
    lib.emg_run_epochs(c2.ctx, 1)
    z1, q1 = state(c1)
    z2, q2 = state(c2)
    assert rel_err(z1, z2) <= 1e-5 and rel_err(q1, q2) <= 1e-5
    c1.close()
    c2.close()


def test_batch_of_uneven_problems_equals_individual_runs(lib, torch):
    specs = [  # m, n, side, levels, prolong, minibatch
        (32, 112, 5, 1, "const", 7),
        (64, 200, 4, 3, "bilinear", 5),
        (128, 300, 3, 2, "const", 4),
        (64, 180, 5, 2, "bilinear", 9),
    ]
    cases, params = [], []
    for i, (m, n, side, levels, prolong, B) in enumerate(specs):
        cases.append(Case(n=n, m=m, side=side, noise_peak=1e4, seed=70 + i))
        params.append(oracle_params(minibatch=B, levels=levels, prolong=prolong))
    batch_ctx = [make_context(lib, c, p, seed=100 + i) for i, (c, p) in enumerate(zip(cases, params))]
    solo_ctx = [make_context(lib, c, p, seed=100 + i) for i, (c, p) in enumerate(zip(cases, params))]
    b = lib.emg_batch_create([c.ctx for c in batch_ctx])
    lib.emg_batch_run_epochs(b, 3)
    for c in solo_ctx:
        lib.emg_run_epochs(c.ctx, 3)
    for cb, cs in zip(batch_ctx, solo_ctx):
        zb, qb = state(cb)
        zs, qs = state(cs)
        assert np.array_equal(zb, zs) and np.array_equal(qb, qs)
    lib.emg_batch_destroy(b)
    for c in batch_ctx + solo_ctx:
        c.close()


def test_batch_with_tensor_core_dft_contexts_equals_individual_runs(lib, torch):
    """Contexts on the tensor-core DFT path (two-CTA cluster kernels, TMA,
    bounded waits) inside one batch graph, beside an FP32 one."""
    specs = [  # m, n, side, levels, prolong, minibatch, dft
        (128, 300, 3, 2, "bilinear", 4, 1),
        (256, 560, 2, 3, "bilinear", 3, 1),
        (128, 280, 3, 3, "bilinear", 5, 0),
    ]
    cases, params, dfts = [], [], []
    for i, (m, n, side, levels, prolong, B, dft) in enumerate(specs):
        cases.append(Case(n=n, m=m, side=side, noise_peak=1e4, seed=90 + i))
        params.append(oracle_params(minibatch=B, levels=levels, prolong=prolong))
        dfts.append(dft)
    batch_ctx = [make_context(lib, c, p, seed=200 + i, dft=d) for i, (c, p, d) in enumerate(zip(cases, params, dfts))]
    solo_ctx = [make_context(lib, c, p, seed=200 + i, dft=d) for i, (c, p, d) in enumerate(zip(cases, params, dfts))]
    b = lib.emg_batch_create([c.ctx for c in batch_ctx])
    lib.emg_batch_run_epochs(b, 2)
    for c in solo_ctx:
        lib.emg_run_epochs(c.ctx, 2)
    for cb, cs in zip(batch_ctx, solo_ctx):
        zb, qb = state(cb)
        zs, qs = state(cs)
        assert np.array_equal(zb, zs) and np.array_equal(qb, qs)
    lib.emg_batch_destroy(b)
    for c in batch_ctx + solo_ctx:
        c.close()


def test_autotune_on_the_tensor_core_path_keeps_results(lib, torch):
    """The tiling autotuner on a tensor-core DFT context (m = 128: 2, 4 or 8 CTAs
    per position in the step kernel that follows the transforms)."""
    case = Case(n=300, m=128, side=3, noise_peak=1e4, seed=97)
    p = oracle_params(minibatch=4, levels=3, prolong="bilinear")
    tuned = make_context(lib, case, p, dft=1)
    plain = make_context(lib, case, p, dft=1)
    chosen, ms = lib.emg_autotune(tuned.ctx)
    assert chosen in (2, 4, 8) and ms > 0
    z0, q0 = state(tuned)
    assert np.array_equal(z0, case.z0.astype(np.complex128))      # the bound state is left alone
    lib.emg_run_epochs(tuned.ctx, 2)
    lib.emg_run_epochs(plain.ctx, 2)
    zt, qt = state(tuned)
    zp, qp = state(plain)
    assert np.array_equal(zt, zp) and np.array_equal(qt, qp)      # tilings agree bitwise for m >= 64
    tuned.close()
    plain.close()
