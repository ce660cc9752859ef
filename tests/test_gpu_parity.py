"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: the per-step bound is a relative L2 error of 1e-5 on the object
pixels a minibatch covers and on the probe (FP32 arithmetic, FP64 oracle).
States are "perturbed truth" so that no Fourier coefficient carrying data is
below FP32 resolution; the ill-conditioned first step from the flat initial
object is covered separately with its own derived bound.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from emg_cases import (Case, c64, covered_mask, epoch_deviations, gpu_params, make_context, oracle_ensemble_states,
                       oracle_inputs, oracle_params, rel_err, state)

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t

    assert t.cuda.is_available()
    return t


# ----------------------------------------------------------------- FFT

@pytest.mark.parametrize("m", [16, 32, 64, 128, 256])
def test_fft2_forward_inverse_match_the_dft(lib, torch, m):
    rng = np.random.default_rng(m)
    x = (rng.standard_normal((3, m, m)) + 1j * rng.standard_normal((3, m, m))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    lib.emg_fft2(xd.data_ptr(), yd.data_ptr(), m, 3, False)
    torch.cuda.synchronize()
    ref = O.dft2(x.astype(np.complex128))
    assert rel_err(yd.cpu().numpy(), ref) < 2e-6
    lib.emg_fft2(yd.data_ptr(), yd.data_ptr(), m, 3, True)   # in place
    torch.cuda.synchronize()
    assert rel_err(yd.cpu().numpy(), x.astype(np.complex128)) < 2e-6
    # inverse against the oracle on an independent input
    lib.emg_fft2(xd.data_ptr(), yd.data_ptr(), m, 3, True)
    torch.cuda.synchronize()
    assert rel_err(yd.cpu().numpy(), O.idft2(x.astype(np.complex128))) < 2e-6


@pytest.mark.parametrize("m", [16, 32, 64, 128, 256])
def test_simulated_intensities_match_the_forward_model(lib, torch, m):
    case = Case(n=2 * m + 24, m=m, side=3)
    out = torch.empty((case.n_pos, m, m), dtype=torch.float32, device="cuda")
    zd = torch.from_numpy(case.z_true).cuda()
    qd = torch.from_numpy(case.q_true).cuda()
    pd = torch.from_numpy(case.pos).cuda()
    lib.emg_simulate_intensity(zd.data_ptr(), case.n, case.n, qd.data_ptr(), m, pd.data_ptr(),
                               case.n_pos, out.data_ptr())
    torch.cuda.synchronize()
    ref = O.forward_intensity(case.q_true.astype(np.complex128), case.z_true.astype(np.complex128), case.pos)
    got = out.cpu().numpy()
    for k in range(case.n_pos):
        assert rel_err(got[k], ref[k]) < 1e-5, k


@pytest.mark.parametrize("m", [32, 128, 256])
def test_misfit_matches_the_oracle(lib, torch, m):
    case = Case(n=2 * m + 16, m=m, side=4, noise_peak=1e4)
    p = oracle_params()
    ctx = make_context(lib, case, p)
    got = lib.emg_misfit(ctx.ctx)
    zo, qo, pos, a, _ = oracle_inputs(case, p)
    ref = O.misfit(qo, zo, pos, a)
    assert abs(got - ref) <= 1e-5 * ref
    ctx.close()


def test_normalize_probe_matches_dp_avg(lib, torch):
    case = Case(n=80, m=32, side=4)
    p = oracle_params()
    ctx = make_context(lib, case, p)
    lib.emg_normalize_probe(ctx.ctx)
    _, q = state(ctx)
    ref = O.dp_avg_scale(case.q0.astype(np.complex128), case.d.astype(np.float64))
    assert rel_err(q, ref) < 1e-6
    ctx.close()


# ------------------------------------------------------ one minibatch step

STEP_CASES = [
    # m, levels, prolong, joint, combine, n_batch
    (16, 1, "const", True, "wavg", 7),
    (32, 1, "const", True, "wavg", 12),
    (32, 1, "const", False, "wavg", 9),
    (32, 2, "const", True, "wavg", 12),
    (32, 3, "bilinear", True, "wavg", 12),
    (32, 2, "const", True, "sum", 5),
    (64, 1, "const", True, "wavg", 10),
    (64, 3, "const", True, "wavg", 10),
    (64, 4, "bilinear", True, "wavg", 10),
    (128, 1, "const", True, "wavg", 6),
    (128, 3, "bilinear", True, "wavg", 6),
    (128, 7, "const", True, "wavg", 3),
    (256, 1, "const", True, "wavg", 4),
    (256, 3, "bilinear", True, "wavg", 4),
]


@pytest.mark.parametrize("m,levels,prolong,joint,combine,nb", STEP_CASES)
def test_one_minibatch_matches_the_oracle(lib, torch, m, levels, prolong, joint, combine, nb):
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5 if m >= 64 else None, seed=m + levels)
    p = oracle_params(alpha=0.05, levels=levels, minibatch=nb, prolong=prolong, joint=joint,
                      combine=combine)
    rng = np.random.default_rng(m * 10 + levels)
    idx = list(rng.permutation(case.n_pos - 4)[: nb - 2]) + [case.n_pos - 4, case.n_pos - 3]
    ctx = make_context(lib, case, p)
    lib.emg_set_verify(ctx.ctx, True)
    sampled = lib.emg_step_minibatch(ctx.ctx, idx, want_misfit=True)
    z_g, q_g = state(ctx)
    stats = lib.emg_position_stats(ctx.ctx, nb)
    zo, qo, pos, a, po = oracle_inputs(case, p)
    info = {}
    z_o, q_o = O.minibatch_step(zo, qo, pos, a, idx, po, out=info)
    mask = covered_mask(case, idx)
    assert rel_err(z_g, z_o, mask) <= STEP_TOL
    assert rel_err(q_g, q_o) <= STEP_TOL
    assert np.array_equal(z_g[~mask], case.z0.astype(np.complex128)[~mask])
    for i, st in enumerate(info["positions"]):
        assert abs(stats[i, 0] - st["surrogate_before"]) <= 1e-5 * st["surrogate_before"]
        assert abs(stats[i, 2] - st["mu"]) <= 1e-6 * st["mu"]
        assert abs(stats[i, 1] - st["surrogate_after"]) <= 1e-5 * st["surrogate_before"]
    assert abs(sampled - info["sampled_misfit"]) <= 1e-5 * info["sampled_misfit"]
    ctx.close()


def test_patch_outside_the_object_leaves_probe_and_object_alone(lib, torch):
    case = Case(n=80, m=32, side=3)
    p = oracle_params(minibatch=1)
    ctx = make_context(lib, case, p)
    outside = case.n_pos - 1            # top-left (-m-3, 5): entirely above the object
    lib.emg_step_minibatch(ctx.ctx, [outside])
    z_g, q_g = state(ctx)
    assert np.array_equal(z_g, case.z0.astype(np.complex128))
    assert np.array_equal(q_g, case.q0.astype(np.complex128))
    assert lib.emg_position_stats(ctx.ctx, 1)[0, 2] == 0.0
    ctx.close()


def test_batch_one_epoch_matches_the_papers_sequential_sweep(lib, torch):
    case = Case(n=72, m=16, side=4, edge=False)
    p = oracle_params(minibatch=1, levels=2)
    ctx = make_context(lib, case, p)
    order = np.random.default_rng(3).permutation(case.n_pos).astype(np.int32)
    lib.emg_run_epochs(ctx.ctx, 1, order[None, :])
    z_g, q_g = state(ctx)
    zo, qo, pos, a, po = oracle_inputs(case, p)
    z_s, q_s = O.sequential_sweep(zo, qo, pos, a, order, po)
    assert rel_err(z_g, z_s) <= 1e-5
    assert rel_err(q_g, q_s) <= 1e-5
    ctx.close()


# ------------------------------------------------------------- epochs

ENSEMBLE = 12     # oracle runs from inputs jiggled by one FP32 rounding


def _gpu_epoch_states(lib, pos, d, n, p, z0, q0, orders):
    """The library's epochs one at a time: per epoch (Phi, running Phi, z, Q)."""
    import paper_2511_01793_gb300 as emg
    import torch as t

    ctx = emg.Context(pos, d, n, n, gpu_params(emg, p), obj=t.from_numpy(z0), probe=t.from_numpy(q0))
    out = []
    for order in orders:
        run, mis = lib.emg_run_epochs(ctx.ctx, 1, order[None, :], running=True, misfit=True)
        z, q = state(ctx)
        out.append((float(mis[0]), float(run[0]), z, q))
    ctx.close()
    return out


def _assert_within_envelope(keys, d_gpu, env, label):
    """Every epoch and quantity: GPU deviation <= max(1e-3, the oracle ensemble's envelope)."""
    bound = np.maximum(1e-3, env)
    ratio = d_gpu / bound
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    print(f"\n{label}: max deviation / bound per quantity: " +
          ", ".join(f"{k} {ratio[:, i].max():.2f}" for i, k in enumerate(keys)) +
          f"; last epoch deviations " + ", ".join(f"{k} {d_gpu[-1, i]:.2e} (env {env[-1, i]:.2e})"
                                                   for i, k in enumerate(keys)))
    assert np.all(d_gpu <= bound), f"epoch {worst[0] + 1}, {keys[worst[1]]}: ratio {ratio[worst]:.2f}"


def test_config_parity_n128_m32_fifty_epochs(lib, torch):
    """The small configuration end to end: 50 epochs, FP32 GPU vs FP64 oracle.

    This nonconvex iteration amplifies rounding: oracle runs whose inputs differ
    by one FP32 rounding spread by several percent in misfit after 50 epochs,
    so a fixed 1e-3 bound cannot hold for any FP32 implementation.  Every epoch,
    the GPU's deviation from the central oracle run (end-of-epoch misfit,
    running misfit, aligned object, probe and RMS phase errors) must stay within
    max(1e-3, the ensemble envelope): the largest deviation so far between any
    two of the central run and ENSEMBLE oracle runs from inputs jiggled by one
    FP32 rounding.  Both runs must also converge.
    """
    w = synth.make_workload("parity_n128_m32")
    pr = w.params
    d = O.forward_intensity(w.q_true, w.z_true, w.pos).astype(np.float32)
    a = np.sqrt(d.astype(np.float64))
    q0 = c64(O.dp_avg_scale(w.q_init_blurred, d.astype(np.float64)))
    z0 = c64(np.ones((pr["n"], pr["n"])))
    orders = synth.epoch_orders(len(w.pos), pr["epochs"], pr["order_seed"])
    p = O.Params(alpha=float(np.float32(pr["alpha"])), levels=pr["levels"], minibatch=pr["minibatch"],
                 prolong=pr["prolong"], w_eps=float(np.float32(1e-6)))
    z64, q64 = z0.astype(np.complex128), q0.astype(np.complex128)
    central, members = oracle_ensemble_states(z64, q64, w.pos, a, orders, p, ENSEMBLE)
    gpu = _gpu_epoch_states(lib, w.pos, d, pr["n"], p, z0, q0, orders)
    region = O.illuminated_region(w.q_true, w.pos, z0.shape)
    keys, d_gpu, env = epoch_deviations(gpu, central, members, region)
    _assert_within_envelope(keys, d_gpu, env, "n128_m32, 50 epochs")
    phi0 = O.misfit(q64, z64, w.pos, a)
    assert central[-1][0] < 1e-2 * phi0 and gpu[-1][0] < 1e-2 * phi0


@pytest.mark.slow
def test_config_parity_mg_n512_m128_epochs(lib, torch):
    """The performance configuration (512^2 object, 128^2 probe, 900 positions,
    Poisson 1e4, three levels with bilinear prolongation, B = 64) over several
    epochs from the flat object and the blurred probe: every epoch the GPU's
    deviation from the central FP64 oracle run stays within max(1e-3, the
    envelope of ENSEMBLE jiggled oracle runs), for the misfit, the running
    misfit and the aligned object, probe and RMS phase errors (the envelope is
    the largest deviation between any two runs of the ensemble)."""
    epochs = 6
    w = synth.make_workload("mg_n512_m128")
    pr = w.params
    d0 = O.forward_intensity(w.q_true, w.z_true, w.pos)
    d = synth.poisson_noise(d0, pr["peak"], np.random.Generator(np.random.PCG64(pr["noise_seed"])))
    d = d.astype(np.float32)
    a = np.sqrt(d.astype(np.float64))
    q0 = c64(O.dp_avg_scale(w.q_init_blurred, d.astype(np.float64)))
    z0 = c64(np.ones((pr["n"], pr["n"])))
    orders = synth.epoch_orders(len(w.pos), epochs, pr["order_seed"])
    p = O.Params(alpha=float(np.float32(pr["alpha"])), levels=pr["levels"], minibatch=pr["minibatch"],
                 prolong=pr["prolong"], w_eps=float(np.float32(1e-6)))
    z64, q64 = z0.astype(np.complex128), q0.astype(np.complex128)
    central, members = oracle_ensemble_states(z64, q64, w.pos, a, orders, p, ENSEMBLE)
    gpu = _gpu_epoch_states(lib, w.pos, d, pr["n"], p, z0, q0, orders)
    region = O.illuminated_region(w.q_true, w.pos, z0.shape)
    keys, d_gpu, env = epoch_deviations(gpu, central, members, region)
    _assert_within_envelope(keys, d_gpu, env, f"mg_n512_m128, {epochs} epochs")
    phi0 = O.misfit(q64, z64, w.pos, a)
    assert gpu[-1][0] < 0.5 * phi0 and central[-1][0] < 0.5 * phi0


def test_full_size_mg_config_minibatch(lib, torch):
    """The 512/128/L=3/bilinear configuration at full size: one B=64 minibatch, all
    outputs compared element by element with the oracle."""
    w = synth.make_workload("mg_n512_m128")
    pr = w.params
    d0 = O.forward_intensity(w.q_true, w.z_true, w.pos)
    d = synth.poisson_noise(d0, pr["peak"], np.random.Generator(np.random.PCG64(pr["noise_seed"])))
    d = d.astype(np.float32)
    rng = np.random.default_rng(5)
    z0 = c64(synth.perturb(w.z_true, 0.3, rng))
    q0 = c64(synth.perturb(w.q_true, 0.3, rng))
    order = synth.epoch_orders(len(w.pos), 1, pr["order_seed"])[0]
    idx = order[: pr["minibatch"]]
    p = O.Params(alpha=float(np.float32(pr["alpha"])), levels=pr["levels"], minibatch=pr["minibatch"],
                 prolong=pr["prolong"], w_eps=float(np.float32(1e-6)))
    import paper_2511_01793_gb300 as emg
    import torch as t

    ctx = emg.Context(w.pos, d, pr["n"], pr["n"], gpu_params(emg, p),
                      obj=t.from_numpy(z0), probe=t.from_numpy(q0))
    lib.emg_step_minibatch(ctx.ctx, idx)
    z_g, q_g = state(ctx)
    a = np.sqrt(d.astype(np.float64))
    z_o, q_o = O.minibatch_step(z0.astype(np.complex128), q0.astype(np.complex128), w.pos, a, idx, p)
    cs = Case.__new__(Case)
    cs.n, cs.m, cs.pos = pr["n"], pr["m"], w.pos
    mask = covered_mask(cs, idx)
    assert rel_err(z_g, z_o, mask) <= STEP_TOL
    assert rel_err(q_g, q_o) <= STEP_TOL
    ctx.close()


# --------------------------------------------------------- determinism

def test_bitwise_repeatable_and_resumable(lib, torch):
    case = Case(n=96, m=32, side=5)
    p = oracle_params(minibatch=6, levels=2)
    c1 = make_context(lib, case, p, seed=99)
    lib.emg_run_epochs(c1.ctx, 4)
    z1, q1 = state(c1)
    c2 = make_context(lib, case, p, seed=99)
    lib.emg_run_epochs(c2.ctx, 2)
    zz, qq = state(c2)
    # resume from a checkpoint of (z, Q, epoch) in a fresh context
    c3 = make_context(lib, case, p, seed=99)
    c3.bind(c64(zz), c64(qq))
    lib.emg_set_epoch(c3.ctx, 2)
    lib.emg_run_epochs(c3.ctx, 2)
    z3, q3 = state(c3)
    assert np.array_equal(z1, z3) and np.array_equal(q1, q3)
    c4 = make_context(lib, case, p, seed=99)
    lib.emg_run_epochs(c4.ctx, 4)
    z4, q4 = state(c4)
    assert np.array_equal(z1, z4) and np.array_equal(q1, q4)
    for c in (c1, c2, c3, c4):
        c.close()


def test_default_schedule_is_the_documented_permutation(lib, torch):
    case = Case(n=80, m=16, side=4)
    p = oracle_params(minibatch=5)
    c1 = make_context(lib, case, p, seed=7)
    lib.emg_run_epochs(c1.ctx, 2)
    orders = np.stack([O.schedule_permutation(7, e, case.n_pos) for e in range(2)]).astype(np.int32)
    c2 = make_context(lib, case, p, seed=123)
    lib.emg_run_epochs(c2.ctx, 2, orders)
    a1, b1 = state(c1)
    a2, b2 = state(c2)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    c1.close()
    c2.close()


def test_host_buffer_entry_point_equals_device_path(lib, torch):
    case = Case(n=96, m=32, side=5)
    p = oracle_params(minibatch=7, levels=2)
    c1 = make_context(lib, case, p, seed=5)
    lib.emg_run_epochs(c1.ctx, 2)
    z1, q1 = state(c1)
    c2 = make_context(lib, case, p, seed=5)
    zh = case.z0.copy()
    qh = case.q0.copy()
    lib.emg_reconstruct_host(c2.ctx, case.d, zh, qh, 2)
    assert np.array_equal(z1, zh.astype(np.complex128)) and np.array_equal(q1, qh.astype(np.complex128))
    c1.close()
    c2.close()


def test_graph_replay_equals_direct_launches(lib, torch):
    """Epochs replayed from the captured CUDA graph equal direct launches bitwise
    (profiling mode runs the direct path)."""
    case = Case(n=2 * 64 + 40, m=64, side=4, noise_peak=1e5)
    p = oracle_params(minibatch=5, levels=3, prolong="bilinear")
    c1 = make_context(lib, case, p, seed=3)
    lib.emg_run_epochs(c1.ctx, 3)
    c2 = make_context(lib, case, p, seed=3)
    lib.emg_set_profiling(c2.ctx, True)
    lib.emg_run_epochs(c2.ctx, 3)
    a1, b1 = state(c1)
    a2, b2 = state(c2)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    c1.close()
    c2.close()


def test_run_until_stops_where_the_rules_say(lib, torch):
    """emg_run_until applies the stopping criterion (Sec. 4.1) and the noise-floor
    rule (Sec. 4.3) to the misfit after each epoch."""
    case = Case(n=96, m=32, side=5, noise_peak=1e3, seed=9)
    p = oracle_params(alpha=0.05, minibatch=4)
    ctx = make_context(lib, case, p)
    hist = lib.emg_run_until(ctx.ctx, 60, window=3, patience=4)
    assert 1 <= len(hist) <= 60
    stop = O.stopping_epoch(list(hist), 3, 4)
    assert (stop == len(hist)) if stop else (len(hist) == 60)
    ctx.close()
    # the noise floor: Phi at the true object and probe on the noisy data
    ctx = make_context(lib, case, p)
    truth = lib.Context(case.pos, case.d, case.n, case.n, lib.emg_default_params(alpha=0.05, minibatch=4),
                        obj=torch.from_numpy(case.z_true), probe=torch.from_numpy(case.q_true))
    floor = lib.emg_misfit(truth.ctx)
    truth.close()
    hist = lib.emg_run_until(ctx.ctx, 200, window=5, patience=10, floor=floor)
    stop = O.stopping_epoch(list(hist), 5, 10, floor)
    assert stop == len(hist) or len(hist) == 200
    assert hist[-1] > 0
    ctx.close()


ATOMIC_CASES = [
    # m, levels, prolong, combine, dft, n_batch
    (32, 2, "const", "wavg", 0, 12),
    (32, 1, "const", "sum", 0, 5),
    (128, 3, "bilinear", "wavg", 0, 6),
    (256, 3, "bilinear", "wavg", 0, 4),
    (128, 3, "bilinear", "wavg", 1, 6),
]


@pytest.mark.parametrize("m,levels,prolong,combine,dft,nb", ATOMIC_CASES)
def test_atomic_scatter_matches_the_oracle_twice_in_a_row(lib, torch, m, levels, prolong, combine, dft, nb):
    """EMG_SCATTER_ATOMIC: patches added into object-sized accumulators with FP32
    atomics (any order), finalised by the combine.  Two minibatches in a row also
    check that the accumulators are left at zero."""
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5 if m >= 64 else None, seed=m + 3 * levels)
    p = oracle_params(alpha=0.05, levels=levels, minibatch=nb, prolong=prolong, combine=combine)
    rng = np.random.default_rng(m + nb)
    perm = rng.permutation(case.n_pos)
    idx1, idx2 = [int(k) for k in perm[:nb]], [int(k) for k in perm[nb:2 * nb]]
    ctx = make_context(lib, case, p, dft=dft, scatter=lib.EMG_SCATTER_ATOMIC)
    det = make_context(lib, case, p, dft=dft)
    zo, qo, pos, a, po = oracle_inputs(case, p)
    tol = 1e-5 if dft == 0 else 4 * 3 * 2.0 ** -16
    for step, idx in enumerate((idx1, idx2)):
        z_before = state(ctx)[0]
        lib.emg_step_minibatch(ctx.ctx, idx)
        lib.emg_step_minibatch(det.ctx, idx)
        z_g, q_g = state(ctx)
        z_d, q_d = state(det)
        zo, qo = O.minibatch_step(zo, qo, pos, a, idx, po)
        mask = covered_mask(case, idx)
        assert rel_err(z_g, zo, mask) <= tol and rel_err(q_g, qo) <= tol
        assert rel_err(z_g, z_d, mask) <= 1e-6        # the two scatters differ by rounding order only
        if step == 0:
            assert np.array_equal(q_g, q_d)           # same probe combine from the same snapshot
        else:
            assert rel_err(q_g, q_d) <= 1e-6
        assert np.array_equal(z_g[~mask], z_before[~mask])
    ctx.close()
    det.close()


@pytest.mark.parametrize("m,levels,prolong,nb", [(32, 2, "bilinear", 7), (128, 3, "bilinear", 5)])
def test_rectangular_object_minibatch_matches_the_oracle(lib, torch, m, levels, prolong, nb):
    """An object of n_rows != n_cols, with patches leaving it on every side (zero-padding of P_k)."""
    import synth
    from emg_cases import c64

    rng = np.random.Generator(np.random.PCG64(m + 17))
    n_rows, n_cols = 2 * m + 24, m + m // 2 + 8
    z_true = c64(synth.make_object(n_rows, n_cols, rng, phi_max=1.2, sigma=3.0))
    q_true = c64(synth.make_probe(m, radius=m / 3.2))
    rows = np.arange(-m // 4, n_rows - m // 2, max(m // 3, 2))
    cols = np.arange(-m // 3, n_cols - m // 3, max(m // 3, 2))
    pos = np.array([(r, c) for r in rows for c in cols], dtype=np.int32)
    d = np.ascontiguousarray(O.forward_intensity(q_true.astype(np.complex128), z_true.astype(np.complex128), pos),
                             dtype=np.float32)
    z0 = c64(synth.perturb(z_true, 0.3, rng))
    q0 = c64(synth.perturb(q_true, 0.3, rng))
    p = oracle_params(alpha=0.05, levels=levels, minibatch=nb, prolong=prolong)
    idx = [int(k) for k in rng.permutation(len(pos))[:nb]]
    ctx = lib.Context(pos, d, n_rows, n_cols, gpu_params(lib, p), obj=torch.from_numpy(z0), probe=torch.from_numpy(q0))
    lib.emg_step_minibatch(ctx.ctx, idx)
    z_g, q_g = state(ctx)
    ctx.close()
    po = O.Params(alpha=float(np.float32(p.alpha)), levels=levels, minibatch=nb, prolong=prolong,
                  w_eps=float(np.float32(p.w_eps)))
    z_o, q_o = O.minibatch_step(z0.astype(np.complex128), q0.astype(np.complex128), pos,
                                np.sqrt(np.maximum(d.astype(np.float64), 0.0)), idx, po)
    mask = np.zeros((n_rows, n_cols), dtype=bool)
    for k in idx:
        r0, c0 = pos[k]
        mask[max(r0, 0):max(min(r0 + m, n_rows), 0), max(c0, 0):max(min(c0 + m, n_cols), 0)] = True
    assert rel_err(z_g, z_o, mask) <= STEP_TOL and rel_err(q_g, q_o) <= STEP_TOL
    assert np.array_equal(z_g[~mask], z0.astype(np.complex128)[~mask])


@pytest.mark.parametrize("m,levels,nb", [(256, 6, 2), (256, 3, 1)])
def test_deepest_hierarchy_and_single_position_at_the_largest_probe(lib, torch, m, levels, nb):
    """m = 256 at its deepest supported multigrid (L = 6: 8 px at the coarsest level,
    one row per CTA of the 8-CTA cluster) and a minibatch of one position."""
    case = Case(n=2 * m + 40, m=m, side=3, noise_peak=1e5, seed=levels + nb)
    p = oracle_params(alpha=0.05, levels=levels, minibatch=nb, prolong="bilinear")
    idx = [0, case.n_pos - 3][:nb]
    ctx = make_context(lib, case, p)
    lib.emg_step_minibatch(ctx.ctx, idx)
    z_g, q_g = state(ctx)
    ctx.close()
    zo, qo, pos, a, po = oracle_inputs(case, p)
    z_o, q_o = O.minibatch_step(zo, qo, pos, a, idx, po)
    mask = covered_mask(case, idx)
    assert rel_err(z_g, z_o, mask) <= STEP_TOL and rel_err(q_g, q_o) <= STEP_TOL


@pytest.mark.parametrize("m,levels", [(16, 1), (64, 2), (128, 3), (256, 3)])
def test_pinned_host_intensity_equals_device_intensity(lib, torch, m, levels):
    """Pinned host data is read in place: all at once by emg_set_intensity, and
    minibatch by minibatch during the first epoch of the host-buffer entry point.
    Both equal the device-data results bitwise, also from a source that is not
    16-byte aligned."""
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=70 + m)
    p = oracle_params(minibatch=6, levels=levels, prolong="bilinear")
    c1 = make_context(lib, case, p, seed=5)
    lib.emg_run_epochs(c1.ctx, 2)
    z1, q1 = state(c1)
    flat = case.d.astype(np.float32).ravel()
    store = torch.empty(flat.size + 1, dtype=torch.float32).pin_memory()
    for off in (0, 1):
        host = store[off:off + flat.size]
        host.copy_(torch.from_numpy(flat))
        c2 = make_context(lib, case, p, seed=5)
        lib.emg_set_intensity(c2.ctx, host.data_ptr())
        lib.emg_run_epochs(c2.ctx, 2)
        z2, q2 = state(c2)
        assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
        c3 = make_context(lib, case, p, seed=5)
        zeros = torch.zeros(flat.size, dtype=torch.float32, device="cuda")
        lib.emg_set_intensity(c3.ctx, zeros.data_ptr())  # the call below must bring the data itself
        zh = torch.from_numpy(case.z0.astype(np.complex64)).pin_memory()
        qh = torch.from_numpy(case.q0.astype(np.complex64)).pin_memory()
        lib.emg_reconstruct_host(c3.ctx, host.numpy().reshape(case.d.shape), zh.numpy(), qh.numpy(), 2)
        assert np.array_equal(z1, zh.numpy().astype(np.complex128))
        assert np.array_equal(q1, qh.numpy().astype(np.complex128))
        # a second call on the same context replays the captured streamed epoch
        zh.copy_(torch.from_numpy(case.z0.astype(np.complex64)))
        qh.copy_(torch.from_numpy(case.q0.astype(np.complex64)))
        orders = np.stack([O.schedule_permutation(5, e, case.n_pos) for e in range(2)]).astype(np.int32)
        lib.emg_reconstruct_host(c3.ctx, host.numpy().reshape(case.d.shape), zh.numpy(), qh.numpy(), 2, orders)
        assert np.array_equal(z1, zh.numpy().astype(np.complex128))
        c2.close()
        c3.close()
    c1.close()


@pytest.mark.parametrize("scatter,dft", [(0, 0), (1, 1)])
def test_create_releases_everything_when_an_allocation_fails(lib, torch, scatter, dft):
    """Host-side fault injection: each device allocation of emg_create fails in
    turn; every attempt returns EMG_ENOMEM and leaves no device memory behind."""
    m = 128
    case = Case(n=2 * m + 40, m=m, side=3, seed=78)
    p = oracle_params(minibatch=4, levels=2)
    make_context(lib, case, p, scatter=scatter, dft=dft).close()   # lazy CUDA state in place
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for after in range(64):
            lib.emg_debug_fail_alloc(after)
            try:
                ctx = make_context(lib, case, p, scatter=scatter, dft=dft)
            except lib.EmgError as e:
                assert e.status == lib.EMG_ENOMEM
                failures += 1
                continue
            ctx.close()      # `after` exceeded the allocations of one create
            break
    finally:
        lib.emg_debug_fail_alloc(-1)
    assert failures >= 10
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
