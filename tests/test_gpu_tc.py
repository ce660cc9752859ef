"""Tensor-core 2-D DFT (BF16 operands split into high and low parts, three
products accumulated in FP32) against the oracle's transform (Sec. 2.1).

Error model of one 1-D pass: every operand x is carried as xh + xl with
|x - xh - xl| <= u^2 |x| (u = 2^-8, the bf16 unit roundoff) and the dropped
product xl yl is at most u^2 |x y|, so each of the 2m real products of an
output carries a relative error below 3 u^2; with FP32 accumulation (2m terms,
u32 = 2^-24, sqrt(2m) u32 < 2e-6) the L2 error of a pass relative to its output
stays below 3 u^2.  Two passes per 2-D transform: TOL = 2 * 3 u^2 = 9.2e-5.

At m = 256 each 1-D transform is by default a radix-16 pass: two 16-point DFT
products with an FP32 twiddle multiply between them (relative error about
2^-23, negligible).  Each product has the error model above, so a 1-D
transform stays below 2 * 3 u^2 and a 2-D one below 4 * 3 u^2.  With
EMG_TC_RADIX16=0 the dense pass (one product) runs instead.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

U = 2.0 ** -8
TOL = 2 * 3 * U * U
RADIX16 = not os.environ.get("EMG_TC_RADIX16", "").startswith("0")


def products(m):
    """DFT products per 1-D transform of size m."""
    return 2 if (m == 256 and RADIX16) else 1


def tol(m):
    return 2 * products(m) * 3 * U * U


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(lib, torch, x, inverse):
    count, m, _ = x.shape
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64)).cuda()
    yd = torch.empty_like(xd)
    lib.emg_dft2_bf16x3(xd.data_ptr(), yd.data_ptr(), m, count, inverse,
                        torch.cuda.current_stream().cuda_stream)
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("m,count,inverse", [(128, 1, 0), (128, 3, 1), (256, 1, 0), (256, 2, 1), (256, 5, 0)])
def test_tc_dft2_matches_the_oracle_on_gaussian_tiles(lib, torch, m, count, inverse):
    rng = np.random.default_rng(7 * m + count)
    x = (rng.standard_normal((count, m, m)) + 1j * rng.standard_normal((count, m, m))).astype(np.complex64)
    got = _run(lib, torch, x, inverse)
    for k in range(count):
        xk = x[k].astype(np.complex128)
        ref = O.idft2(xk) if inverse else O.dft2(xk)
        assert rel(got[k], ref) <= tol(m)


@pytest.mark.parametrize("m", [128, 256])
def test_tc_dft2_on_exit_waves_and_round_trip(lib, torch, m):
    """Exit waves of the synthetic workload (probe disk times a phase object):
    most of the energy sits near DC, the regime of the method's data."""
    from synth import inputs as S
    rng = np.random.default_rng(m)
    q = S.make_probe(m, radius=m / 3.2)
    z = S.make_object(m, m, rng, phi_max=np.pi)
    psi = (q * z)[None].astype(np.complex64)
    Psi = _run(lib, torch, psi, 0)
    ref = O.dft2(psi[0].astype(np.complex128))
    assert rel(Psi[0], ref) <= tol(m)
    back = _run(lib, torch, Psi.astype(np.complex64), 1)
    assert rel(back[0], psi[0].astype(np.complex128)) <= 2 * tol(m)


@pytest.mark.parametrize("m,r0,c0", [(128, 5, 9), (256, 5, 9), (256, 250, 17)])
def test_tc_dft2_of_a_delta_is_flat(lib, torch, m, r0, c0):
    """F delta_(r0,c0) has modulus 1 everywhere and the phase of the shift theorem."""
    x = np.zeros((1, m, m), dtype=np.complex64)
    x[0, r0, c0] = 1.0
    got = _run(lib, torch, x, 0)[0]
    u = np.arange(m)
    ref = np.exp(-2j * np.pi * (r0 * u[:, None] + c0 * u[None, :]) / m)
    assert np.max(np.abs(got - ref)) <= 3 * U * U * 4 * products(m)


_DENSE_256 = """
import sys
sys.path.insert(0, ".")
import numpy as np, torch
import oracle as O
import paper_2511_01793_gb300 as lib
lib.load()
rng = np.random.default_rng(5)
x = (rng.standard_normal((3, 256, 256)) + 1j * rng.standard_normal((3, 256, 256))).astype(np.complex64)
xd = torch.from_numpy(x).cuda()
yd = torch.empty_like(xd)
lib.emg_dft2_bf16x3(xd.data_ptr(), yd.data_ptr(), 256, 3, 0, torch.cuda.current_stream().cuda_stream)
y = yd.cpu().numpy().astype(np.complex128)
print(max(float(np.linalg.norm(y[k] - O.dft2(x[k].astype(np.complex128))) / np.linalg.norm(O.dft2(x[k].astype(np.complex128)))) for k in range(3)))
"""


def test_tc_dft2_dense_pass_at_256_when_radix16_is_off(lib, torch):
    """EMG_TC_RADIX16=0 (read once per process, so in a child process) selects the
    dense pass at m = 256: one product per 1-D transform, error below 2 * 3 u^2."""
    env = dict(os.environ, EMG_TC_RADIX16="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _DENSE_256], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    err = float(r.stdout.strip().splitlines()[-1])
    assert 0 < err <= 2 * 3 * U * U


# ---------------------------------------------------------------------------
# The minibatch step with the tensor-core DFT pair (params.dft = EMG_DFT_BF16X3)

from emg_cases import Case, covered_mask, make_context, oracle_inputs, oracle_params, rel_err, state  # noqa: E402

# A step runs four 1-D passes (forward and inverse 2-D DFTs) whose relative
# error is each below 3 u^2.  Every other operation is the FP32 path's, whose
# error (about 1e-7 on these cases) is negligible beside it.  The modulus
# replacement keeps the error's size (|a Psi/|Psi|| = a), and the gains of the
# object and probe steps are at most 1.  The step's relative error is therefore
# bounded by that of its exit waves: 4 * 3 u^2 = 1.8e-4 (twice that at m = 256
# with the radix-16 pass, whose 1-D transforms take two products each).
TC_STEP_TOL = 4 * 3 * U * U


def step_tol(m):
    return TC_STEP_TOL * products(m)

TC_CASES = [
    # m, levels, prolong, n_batch
    (128, 1, "const", 6),
    (128, 3, "bilinear", 6),
    (256, 2, "const", 3),
    (256, 3, "bilinear", 4),
]


def _step_both(lib, m, levels, prolong, nb):
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5, seed=m + levels)
    p = oracle_params(alpha=0.05, levels=levels, minibatch=nb, prolong=prolong)
    rng = np.random.default_rng(m * 10 + levels)
    idx = list(rng.permutation(case.n_pos - 4)[: nb - 2]) + [case.n_pos - 4, case.n_pos - 3]
    out = {}
    for dft in (0, 1):
        ctx = make_context(lib, case, p, dft=dft)
        lib.emg_set_verify(ctx.ctx, True)
        sampled = lib.emg_step_minibatch(ctx.ctx, idx, want_misfit=True)
        z, q = state(ctx)
        out[dft] = (z, q, sampled, lib.emg_position_stats(ctx.ctx, nb))
        ctx.close()
    zo, qo, pos, a, po = oracle_inputs(case, p)
    info = {}
    z_o, q_o = O.minibatch_step(zo, qo, pos, a, idx, po, out=info)
    return case, idx, out, (z_o, q_o, info)


@pytest.mark.parametrize("m,levels,prolong,nb", TC_CASES)
def test_tc_step_matches_the_oracle(lib, torch, m, levels, prolong, nb):
    case, idx, out, (z_o, q_o, info) = _step_both(lib, m, levels, prolong, nb)
    mask = covered_mask(case, idx)
    z_t, q_t, sampled, stats = out[1]
    z_f, q_f, _, _ = out[0]
    e_tc = (rel_err(z_t, z_o, mask), rel_err(q_t, q_o))
    e_fft = (rel_err(z_f, z_o, mask), rel_err(q_f, q_o))
    print(f"m={m} L={levels}: tc {e_tc[0]:.2e} {e_tc[1]:.2e}  fft {e_fft[0]:.2e} {e_fft[1]:.2e}  "
          f"sampled {abs(sampled - info['sampled_misfit']) / info['sampled_misfit']:.2e}")
    t = step_tol(m)
    assert e_tc[0] <= t and e_tc[1] <= t
    assert np.array_equal(z_t[~mask], case.z0.astype(np.complex128)[~mask])
    assert abs(sampled - info["sampled_misfit"]) <= t * info["sampled_misfit"]
    for i, st in enumerate(info["positions"]):
        assert abs(stats[i, 2] - st["mu"]) <= 1e-6 * st["mu"]
        assert abs(stats[i, 0] - st["surrogate_before"]) <= t * st["surrogate_before"]
        assert abs(stats[i, 1] - st["surrogate_after"]) <= t * st["surrogate_before"]


def test_tc_epochs_are_bitwise_repeatable(lib, torch):
    m = 128
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5, seed=3)
    p = oracle_params(alpha=0.05, levels=3, minibatch=8, prolong="bilinear")
    res = []
    for _ in range(2):
        ctx = make_context(lib, case, p, dft=1)
        mis = lib.emg_run_epochs(ctx.ctx, 2, misfit=True)
        z, q = state(ctx)
        res.append((z, q, mis))
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2][1], res[1][2][1])


def test_tc_step_is_the_same_for_every_fft_tiling(lib, torch):
    """The cluster size of the step kernel that consumes R_k does not change the results."""
    m = 128
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5, seed=7)
    p = oracle_params(alpha=0.05, levels=3, minibatch=8, prolong="bilinear")
    res = []
    for cl in (2, 4, 8):
        ctx = make_context(lib, case, p, dft=1)
        lib.emg_set_cluster(ctx.ctx, cl)
        lib.emg_run_epochs(ctx.ctx, 2)
        res.append(state(ctx))
        ctx.close()
    for z, q in res[1:]:
        assert np.array_equal(z, res[0][0]) and np.array_equal(q, res[0][1])


def test_full_size_precision_minibatch_matches_the_oracle(lib, torch):
    """One minibatch of the precision workload at full size (object 2048^2,
    probe 256^2, B = 256, L = 3 bilinear) in the launch configuration the bench
    times, with both DFT variants, against the oracle on every covered pixel.
    Only the minibatch's positions carry data (the step reads no other)."""
    import synth
    from emg_cases import c64, gpu_params

    w = synth.make_workload("prec_n2048_m256")
    p = w.params
    n, m, B = p["n"], p["m"], p["minibatch"]
    rng = np.random.Generator(np.random.PCG64(77))
    idx = [int(k) for k in synth.epoch_orders(len(w.pos), 1, p["order_seed"])[0][:B]]
    d = np.zeros((len(w.pos), m, m), dtype=np.float32)
    d_mb = O.forward_intensity(w.q_true, w.z_true, w.pos[idx])
    d[idx] = synth.poisson_noise(d_mb, p["peak"], rng).astype(np.float32)
    z0 = c64(synth.perturb(w.z_true, 0.3, rng))
    q0 = c64(synth.perturb(w.q_true, 0.3, rng))
    po = oracle_params(alpha=p["alpha"], levels=p["levels"], minibatch=B, prolong=p["prolong"])
    a64 = np.sqrt(np.maximum(d.astype(np.float64), 0.0))
    oq = O.Params(alpha=float(np.float32(po.alpha)), levels=po.levels, minibatch=B, prolong=po.prolong,
                  combine=po.combine, w_eps=float(np.float32(po.w_eps)), joint=po.joint)
    z_o, q_o = O.minibatch_step(z0.astype(np.complex128), q0.astype(np.complex128), w.pos, a64, idx, oq)
    mask = np.zeros((n, n), dtype=bool)
    for k in idx:
        r0, c0 = w.pos[k]
        mask[max(r0, 0):min(r0 + m, n), max(c0, 0):min(c0 + m, n)] = True
    for dft, tol in ((lib.EMG_DFT_FFT32, 1e-5), (lib.EMG_DFT_BF16X3, step_tol(m))):
        ctx = lib.Context(w.pos, d, n, n, gpu_params(lib, po, dft=dft), obj=torch.from_numpy(z0),
                          probe=torch.from_numpy(q0))
        lib.emg_step_minibatch(ctx.ctx, idx)
        z_g, q_g = state(ctx)
        ctx.close()
        e_z, e_q = rel_err(z_g, z_o, mask), rel_err(q_g, q_o)
        print(f"dft={dft}: object {e_z:.2e} probe {e_q:.2e}")
        assert e_z <= tol and e_q <= tol
        assert np.array_equal(z_g[~mask], z0.astype(np.complex128)[~mask])


def test_bounded_wait_gives_up_reports_and_leaves_the_device_usable(lib, torch):
    """A wait on an mbarrier that nothing arrives on (the tensor-core kernel's wait)
    gives up after its 1 s limit and sets the device flag; the GPU then still
    computes a correct tensor-core transform."""
    import time

    t0 = time.perf_counter()
    gave_up = lib.emg_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert gave_up == 1
    assert 0.9 <= dt < 60.0
    rng = np.random.default_rng(11)
    x = (rng.standard_normal((2, 128, 128)) + 1j * rng.standard_normal((2, 128, 128))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    lib.emg_dft2_bf16x3(xd.data_ptr(), yd.data_ptr(), 128, 2, False)
    torch.cuda.synchronize()
    want = np.stack([O.dft2(t.astype(np.complex128)) for t in x])
    assert rel_err(yd.cpu().numpy().astype(np.complex128), want) <= TOL
