"""Gradient of the exit-wave misfit (Sec. 2.1) on the GPU against the oracle,
central finite differences and autograd; the plain gradient baseline."""
import numpy as np
import pytest

import oracle as O
import synth
from emg_cases import Case, c64, gpu_params, make_context, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    assert t.cuda.is_available()
    return t


def _gpu_gradient(lib, torch, ctx, z, q):
    zd = torch.from_numpy(c64(z)).cuda()
    qd = torch.from_numpy(c64(q)).cuda()
    gz = torch.empty_like(zd)
    gq = torch.empty_like(qd)
    phi = lib.emg_misfit_gradient(ctx.ctx, zd.data_ptr(), qd.data_ptr(), gz.data_ptr(), gq.data_ptr(), True)
    torch.cuda.synchronize()
    return phi, gz.cpu().numpy().astype(np.complex128), gq.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("chunk", [6, 0])
@pytest.mark.parametrize("m", [16, 32, 64, 128, 256])
def test_gradient_matches_the_oracle(lib, torch, m, chunk):
    """16 positions in chunks of 6 (sums over several launches), and in the
    automatic chunk (one launch here)."""
    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e4, seed=40 + m)
    p = oracle_params(minibatch=6)
    ctx = make_context(lib, case, p)
    lib.emg_set_gradient_chunk(ctx.ctx, chunk)
    phi, gz, gq = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    ctx.close()
    phi_o, gz_o, gq_o = O.misfit_gradients(case.q0.astype(np.complex128), case.z0.astype(np.complex128),
                                           case.pos, case.a64)
    assert abs(phi - phi_o) <= 1e-5 * phi_o
    assert rel_err(gz, gz_o) <= 1e-5
    assert rel_err(gq, gq_o) <= 1e-5


def test_chunked_gradient_sums_are_bitwise_repeatable(lib, torch):
    """Several chunks: the sums of one chunk run beside the next chunk's patches on
    two buffer pairs.  Calls in a row, and a call after a misfit-only one, give
    bitwise the same gradients."""
    m = 64
    case = Case(n=2 * m + 40, m=m, side=5, noise_peak=1e4, seed=140)
    ctx = make_context(lib, case, oracle_params(minibatch=6))
    lib.emg_set_gradient_chunk(ctx.ctx, 5)               # 29 positions: 6 chunks
    first = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    second = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    zd = torch.from_numpy(c64(case.z0)).cuda()
    qd = torch.from_numpy(c64(case.q0)).cuda()
    lib.emg_misfit_gradient(ctx.ctx, zd.data_ptr(), qd.data_ptr(), 0, 0, True)
    third = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    ctx.close()
    for other in (second, third):
        assert other[0] == first[0]
        assert np.array_equal(other[1], first[1]) and np.array_equal(other[2], first[2])
    phi_o, gz_o, gq_o = O.misfit_gradients(case.q0.astype(np.complex128), case.z0.astype(np.complex128),
                                           case.pos, case.a64)
    assert rel_err(first[1], gz_o) <= 1e-5 and rel_err(first[2], gq_o) <= 1e-5


def test_gradient_matches_central_differences(lib, torch):
    """Central differences (h = 1e-3) of the FP64 misfit at the same point."""
    case = Case(n=104, m=32, side=4, noise_peak=1e4, seed=9)
    ctx = make_context(lib, case, oracle_params(minibatch=8))
    _, gz, gq = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    ctx.close()
    z = case.z0.astype(np.complex128)
    q = case.q0.astype(np.complex128)
    h = 1e-3
    rng = np.random.default_rng(2)
    for _ in range(4):
        i, j = rng.integers(20, 80, 2)
        for unit in (1.0, 1j):
            zp, zm = z.copy(), z.copy()
            zp[i, j] += h * unit
            zm[i, j] -= h * unit
            fd = (O.misfit(q, zp, case.pos, case.a64) - O.misfit(q, zm, case.pos, case.a64)) / (2 * h)
            got = gz[i, j].real if unit == 1.0 else gz[i, j].imag
            assert abs(got - fd) <= 1e-4 * np.max(np.abs(gz))
        i, j = rng.integers(0, 32, 2)
        for unit in (1.0, 1j):
            qp, qm = q.copy(), q.copy()
            qp[i, j] += h * unit
            qm[i, j] -= h * unit
            fd = (O.misfit(qp, z, case.pos, case.a64) - O.misfit(qm, z, case.pos, case.a64)) / (2 * h)
            got = gq[i, j].real if unit == 1.0 else gq[i, j].imag
            assert abs(got - fd) <= 1e-4 * np.max(np.abs(gq))


def test_autograd_function_uses_the_kernel_gradient(lib, torch):
    from paper_2511_01793_gb300 import autograd as AG

    case = Case(n=104, m=32, side=4, seed=10)
    ctx = make_context(lib, case, oracle_params(minibatch=8))
    _, gz, gq = _gpu_gradient(lib, torch, ctx, case.z0, case.q0)
    o = torch.from_numpy(case.z0).cuda().requires_grad_(True)
    q = torch.from_numpy(case.q0).cuda().requires_grad_(True)
    loss = 3.0 * AG.misfit(o, q, ctx)
    loss.backward()
    assert np.allclose(o.grad.cpu().numpy(), 3.0 * gz, rtol=1e-6, atol=1e-6 * np.abs(gz).max())
    assert np.allclose(q.grad.cpu().numpy(), 3.0 * gq, rtol=1e-6, atol=1e-6 * np.abs(gq).max())
    ctx.close()


def test_gradient_descent_baseline_reduces_the_misfit(lib, torch):
    from paper_2511_01793_gb300 import autograd as AG

    case = Case(n=104, m=32, side=5, step=8, seed=11, edge=False, pert=0.2)
    ctx = make_context(lib, case, oracle_params(minibatch=8))
    o = torch.from_numpy(case.z0).cuda()
    q = torch.from_numpy(case.q0).cuda()
    _, _, hist = AG.gradient_descent(ctx, o, q, 40)
    ctx.close()
    assert hist[-1] < 0.5 * hist[0]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(hist, hist[1:]))


def test_full_size_gradient_workload(lib, torch):
    """Object 1024^2, probe 256^2, 1600 positions, Poisson 1e4: gradient vs the oracle."""
    import paper_2511_01793_gb300 as emg

    w = synth.make_workload("grad_n1024_m256")
    pr = w.params
    d = O.forward_intensity(w.q_true, w.z_true, w.pos)
    d = synth.poisson_noise(d, pr["peak"], np.random.Generator(np.random.PCG64(pr["noise_seed"]))).astype(np.float32)
    rng = np.random.default_rng(12)
    z = c64(synth.perturb(w.z_true, 0.2, rng))
    q = c64(synth.perturb(w.q_true, 0.2, rng))
    params = emg.emg_default_params(alpha=pr["alpha"], minibatch=pr["minibatch"])
    ctx = emg.Context(w.pos, d, pr["n"], pr["n"], params)
    phi, gz, gq = _gpu_gradient(lib, torch, ctx, z, q)
    ctx.close()
    phi_o, gz_o, gq_o = O.misfit_gradients(q.astype(np.complex128), z.astype(np.complex128), w.pos,
                                           np.sqrt(d.astype(np.float64)))
    assert abs(phi - phi_o) <= 1e-5 * phi_o
    assert rel_err(gz, gz_o) <= 1e-5
    assert rel_err(gq, gq_o) <= 1e-5
