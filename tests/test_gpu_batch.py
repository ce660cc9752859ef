"""Batches of uneven reconstructions in one graph launch per epoch, the FFT
tiling (CTAs per position) and its autotuner."""
import numpy as np
import pytest

import oracle as O
from emg_cases import Case, make_context, oracle_inputs, oracle_params, rel_err, state

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


def test_batch_of_uneven_problems_matches_the_oracle(lib, torch):
    """Four uneven problems in one batch graph, two epochs, each problem against
    the FP64 oracle on the same inputs and the same default schedules
    (SplitMix64 + Fisher-Yates from the problem's seed).  From perturbed-truth
    states the iteration is well conditioned, so the per-step bound carries over
    to whole epochs: relative L2 error <= 1e-5 per epoch run, on the object and
    the probe, after each epoch."""
    specs = [  # m, n, side, levels, prolong, minibatch
        (32, 112, 5, 1, "const", 7),
        (64, 200, 4, 3, "bilinear", 5),
        (128, 300, 3, 2, "bilinear", 4),
        (64, 180, 5, 2, "const", 9),
    ]
    cases, params, ctxs = [], [], []
    for i, (m, n, side, levels, prolong, B) in enumerate(specs):
        case = Case(n=n, m=m, side=side, noise_peak=1e4, seed=170 + i)
        p = oracle_params(minibatch=B, levels=levels, prolong=prolong)
        cases.append(case)
        params.append(p)
        ctxs.append(make_context(lib, case, p, seed=300 + i))
    b = lib.emg_batch_create([c.ctx for c in ctxs])
    orc = [(c.z0.astype(np.complex128), c.q0.astype(np.complex128)) for c in cases]
    worst = 0.0
    for epoch in range(2):
        lib.emg_batch_run_epochs(b, 1)
        for i, (case, p, ctx) in enumerate(zip(cases, params, ctxs)):
            _, _, pos, a, po = oracle_inputs(case, p)
            order = np.array(O.schedule_permutation(300 + i, epoch, case.n_pos), dtype=np.int32)
            z_o, q_o, _ = O.run_epochs(orc[i][0], orc[i][1], pos, a, order[None, :], po, eval_misfit=False)
            orc[i] = (z_o, q_o)
            z_g, q_g = state(ctx)
            ez, eq = rel_err(z_g, z_o), rel_err(q_g, q_o)
            worst = max(worst, ez, eq)
            assert ez <= 1e-5 * (epoch + 1), (i, epoch, ez)
            assert eq <= 1e-5 * (epoch + 1), (i, epoch, eq)
    print(f"\nbatch vs oracle, worst relative error after 2 epochs: {worst:.2e}")
    lib.emg_batch_destroy(b)
    for c in ctxs:
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


def _epoch_by_hand(lib, ctx, order, b):
    """One epoch as explicit minibatches of b positions (the last one shorter)."""
    for i in range(0, len(order), b):
        lib.emg_step_minibatch(ctx.ctx, order[i:i + b])


@pytest.mark.parametrize("m,dft", [(32, 0), (128, 0), (128, 1)])
def test_minibatch_can_change_after_creation(lib, torch, m, dft):
    """An epoch at B = 4, then B grows to 7 (new buffers, a new captured epoch)
    and shrinks to 3: equal bitwise to the same minibatches stepped by hand on
    a context created with the largest B."""
    case = Case(n=2 * m + 40, m=m, side=5, noise_peak=1e4, seed=80 + m + dft)
    p = oracle_params(minibatch=4, levels=2, prolong="bilinear")
    orders = np.stack([O.schedule_permutation(9, e, case.n_pos) for e in range(3)]).astype(np.int32)
    c1 = make_context(lib, case, p, seed=9, dft=dft)
    lib.emg_run_epochs(c1.ctx, 1, orders[0:1])
    lib.emg_set_minibatch(c1.ctx, 7)
    lib.emg_run_epochs(c1.ctx, 1, orders[1:2])
    lib.emg_set_minibatch(c1.ctx, 3)
    lib.emg_run_epochs(c1.ctx, 1, orders[2:3])
    p7 = oracle_params(minibatch=7, levels=2, prolong="bilinear")
    c2 = make_context(lib, case, p7, seed=9, dft=dft)
    for order, b in zip(orders, (4, 7, 3)):
        _epoch_by_hand(lib, c2, order, b)
    z1, q1 = state(c1)
    z2, q2 = state(c2)
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
    with pytest.raises(lib.EmgError):
        lib.emg_set_minibatch(c1.ctx, 0)
    with pytest.raises(lib.EmgError):
        lib.emg_set_minibatch(c1.ctx, case.n_pos + 1)
    c1.close()
    c2.close()


def test_scatter_mode_can_change_after_creation(lib, torch):
    """Deterministic -> atomic equals an atomic context up to rounding; back to
    deterministic equals a deterministic context bitwise."""
    m = 64
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=91)
    p = oracle_params(minibatch=5, levels=2, prolong="bilinear")
    det = make_context(lib, case, p, seed=4)
    lib.emg_run_epochs(det.ctx, 2)
    ato = make_context(lib, case, p, seed=4, scatter=1)
    lib.emg_run_epochs(ato.ctx, 2)
    c = make_context(lib, case, p, seed=4)
    lib.emg_run_epochs(c.ctx, 1)                      # captures a deterministic epoch first
    lib.emg_set_scatter(c.ctx, lib.EMG_SCATTER_ATOMIC)
    lib.emg_run_epochs(c.ctx, 1)
    z, q = state(c)
    c1 = make_context(lib, case, p, seed=4)
    lib.emg_run_epochs(c1.ctx, 1)
    lib.emg_set_scatter(c1.ctx, lib.EMG_SCATTER_ATOMIC)
    lib.emg_set_scatter(c1.ctx, lib.EMG_SCATTER_DETERMINISTIC)
    lib.emg_run_epochs(c1.ctx, 1)
    zd, qd = state(det)
    za, qa = state(ato)
    z1, q1 = state(c1)
    assert rel_err(z, zd) <= 1e-5 and rel_err(q, qd) <= 1e-5 and rel_err(z, za) <= 1e-5
    assert np.array_equal(z1, zd) and np.array_equal(q1, qd)
    with pytest.raises(lib.EmgError):
        lib.emg_set_scatter(c1.ctx, 2)
    for x in (det, ato, c, c1):
        x.close()


def test_autotune_search_chooses_b_tiling_and_scatter(lib, torch):
    """The search leaves the bound state and the epoch counter alone, returns a
    candidate B with a positive misfit rate, and the context then runs exactly
    as one created with the chosen settings."""
    m = 64
    case = Case(n=2 * m + 72, m=m, side=6, noise_peak=1e5, seed=93)
    p = oracle_params(minibatch=8, levels=2, prolong="bilinear")
    c = make_context(lib, case, p, seed=6)
    z0, q0 = state(c)
    res = lib.emg_autotune_search(c.ctx, minibatch=(4, 12, 36), trial_epochs=2, tune_tiling=True,
                                  allow_atomic=False)
    z_after, q_after = state(c)
    assert np.array_equal(z0, z_after) and np.array_equal(q0, q_after)
    assert res["minibatch"] in (4, 12, 36) and res["cluster"] in (2, 4) and res["scatter"] == 0
    assert res["misfit_rate"] > 0 and res["ms_per_epoch"] > 0
    lib.emg_run_epochs(c.ctx, 2)
    pb = oracle_params(minibatch=res["minibatch"], levels=2, prolong="bilinear")
    ref = make_context(lib, case, pb, seed=6)
    lib.emg_set_cluster(ref.ctx, res["cluster"])
    lib.emg_run_epochs(ref.ctx, 2)
    z1, q1 = state(c)
    z2, q2 = state(ref)
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
    res2 = lib.emg_autotune_search(c.ctx, minibatch=(), trial_epochs=1, tune_tiling=False, allow_atomic=True)
    assert res2["minibatch"] == res["minibatch"] and res2["scatter"] in (0, 1)
    with pytest.raises(lib.EmgError):
        lib.emg_autotune_search(c.ctx, minibatch=(0,))
    with pytest.raises(lib.EmgError):
        lib.emg_autotune_search(c.ctx, minibatch=(4,), trial_epochs=0)
    c.close()
    ref.close()


@pytest.mark.parametrize("m,levels,prolong,cl", [(64, 3, "bilinear", 2), (128, 3, "bilinear", 4),
                                                  (128, 2, "const", 8), (128, 7, "const", 2)])
def test_fused_probe_prep_equals_the_separate_kernel(lib, torch, m, levels, prolong, cl):
    """The probe prep inside the step launch (ticket-ordered prep clusters) gives
    bitwise the results of the prep as its own kernel, over graph-replayed epochs
    and single minibatches."""
    case = Case(n=2 * m + 40, m=m, side=5, noise_peak=1e4, seed=95 + m + levels)
    p = oracle_params(minibatch=7, levels=levels, prolong=prolong)
    out = []
    for fuse in (1, 0):
        c = make_context(lib, case, p, seed=3)
        lib.emg_set_cluster(c.ctx, cl)
        lib.emg_set_prep_fusion(c.ctx, fuse)
        lib.emg_run_epochs(c.ctx, 2)
        lib.emg_step_minibatch(c.ctx, [0, 3, 5])
        out.append(state(c))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_host_buffer_call_reports_a_wait_that_gave_up_and_recovers(lib, torch):
    """The host-buffer entry point queues its downloads and waits once; a bounded
    wait that gave up in the step kernel (made to run out) still makes it return
    EMG_ETIMEOUT, and the next call runs normally with the same result as a
    fresh context."""
    m = 128
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=97)
    p = oracle_params(minibatch=10, levels=3, prolong="bilinear")
    c = make_context(lib, case, p, seed=2)
    d = np.ascontiguousarray(case.d, dtype=np.float32)
    z = case.z0.astype(np.complex64).copy()
    q = case.q0.astype(np.complex64).copy()
    lib.emg_debug_prep_wait_extra(c.ctx, 1000)
    with pytest.raises(lib.EmgError) as err:
        lib.emg_reconstruct_host(c.ctx, d, z, q, 1, running=True)
    assert err.value.status == lib.EMG_ETIMEOUT
    lib.emg_debug_prep_wait_extra(c.ctx, 0)
    z1, q1 = case.z0.astype(np.complex64).copy(), case.q0.astype(np.complex64).copy()
    lib.emg_set_epoch(c.ctx, 0)
    r1, _ = lib.emg_reconstruct_host(c.ctx, d, z1, q1, 2, running=True)
    ref = make_context(lib, case, p, seed=2)
    z2, q2 = case.z0.astype(np.complex64).copy(), case.q0.astype(np.complex64).copy()
    r2, _ = lib.emg_reconstruct_host(ref.ctx, d, z2, q2, 2, running=True)
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2) and np.array_equal(r1, r2)
    assert np.all(np.isfinite(r1)) and r1[0] > 0
    c.close()
    ref.close()


def test_fused_prep_wait_gives_up_reports_and_recovers(lib, torch):
    """The step kernel's bounded wait for the fused prep, made to run out (it waits
    for prep tiles that never come): the call reports EMG_ETIMEOUT after about
    1 s, and the context then runs exactly as a fresh one."""
    import time

    m = 128
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=99)
    p = oracle_params(minibatch=6, levels=3, prolong="bilinear")
    c = make_context(lib, case, p, seed=2)
    lib.emg_debug_prep_wait_extra(c.ctx, 1000)
    t0 = time.perf_counter()
    with pytest.raises(lib.EmgError) as err:
        lib.emg_step_minibatch(c.ctx, [0, 1, 2], want_misfit=True)
    assert err.value.status == lib.EMG_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.9
    lib.emg_debug_prep_wait_extra(c.ctx, 0)
    # recovery: rebind the initial state and compare with a fresh context
    c.obj.copy_(torch.from_numpy(case.z0.astype(np.complex64)))
    c.probe.copy_(torch.from_numpy(case.q0.astype(np.complex64)))
    torch.cuda.synchronize()
    lib.emg_set_epoch(c.ctx, 0)
    lib.emg_run_epochs(c.ctx, 2)
    ref = make_context(lib, case, p, seed=2)
    lib.emg_run_epochs(ref.ctx, 2)
    z1, q1 = state(c)
    z2, q2 = state(ref)
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
    c.close()
    ref.close()
