"""Tensor-core 2-D DFT (BF16 operands split into high and low parts, three
products accumulated in FP32) against the oracle's transform (Sec. 2.1).

Error model of one 1-D pass: every operand x is carried as xh + xl with
|x - xh - xl| <= u^2 |x| (u = 2^-8, the bf16 unit roundoff) and the dropped
product xl yl is at most u^2 |x y|, so each of the 2m real products of an
output carries a relative error below 3 u^2; with FP32 accumulation (2m terms,
u32 = 2^-24, sqrt(2m) u32 < 2e-6) the L2 error of a pass relative to its output
stays below 3 u^2.  Two passes per 2-D transform: TOL = 2 * 3 u^2 = 9.2e-5.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

U = 2.0 ** -8
TOL = 2 * 3 * U * U


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
        assert rel(got[k], ref) <= TOL


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
    assert rel(Psi[0], ref) <= TOL
    back = _run(lib, torch, Psi.astype(np.complex64), 1)
    assert rel(back[0], psi[0].astype(np.complex128)) <= 2 * TOL


def test_tc_dft2_of_a_delta_is_flat(lib, torch):
    """F delta_(r0,c0) has modulus 1 everywhere and the phase of the shift theorem."""
    m = 128
    x = np.zeros((1, m, m), dtype=np.complex64)
    x[0, 5, 9] = 1.0
    got = _run(lib, torch, x, 0)[0]
    u = np.arange(m)
    ref = np.exp(-2j * np.pi * (5 * u[:, None] + 9 * u[None, :]) / m)
    assert np.max(np.abs(got - ref)) <= 3 * U * U * 4
