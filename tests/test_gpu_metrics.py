"""The FP64 reconstruction-error reductions of the library against the oracle.

emg_illuminated_region and emg_aligned_errors reduce, on the GPU and in FP64,
what the oracle's illuminated_region and aligned_errors compute on the host:
the region the scan illuminates, the best scale c of the (c z, Q / c)
ambiguity of blind ptychography (Sec. 2.1), the aligned object and probe
errors and the RMS phase difference.  Both sides read the same complex64
arrays, so they agree to FP64 rounding.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _problem(n, m, side, step, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    z_true = synth.make_object(n, n, rng, phi_max=np.pi).astype(np.complex64)
    q_true = synth.make_probe(m, radius=m / 3.2).astype(np.complex64)
    pos = synth.make_scan(n, m, side, step, 2, rng)
    # a reconstruction-like state: the truth times a complex scale, perturbed
    c = 0.7 * np.exp(1j * 2.1)
    z = (synth.perturb(z_true.astype(np.complex128), 0.05, rng) * c).astype(np.complex64)
    q = (synth.perturb(q_true.astype(np.complex128), 0.05, rng) / c).astype(np.complex64)
    return z_true, q_true, pos, z, q


def _region_gpu(lib, q_ref, pos, n, frac):
    import torch

    mask = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    qd = torch.from_numpy(q_ref).cuda()
    pd = torch.from_numpy(pos).cuda()
    lib.emg_illuminated_region(qd.data_ptr(), q_ref.shape[0], pd.data_ptr(), len(pos), n, n, frac,
                               mask.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return mask


@pytest.mark.parametrize("n,m,side,step,frac", [(96, 32, 6, 10, 0.1), (512, 128, 30, 12, 0.1), (300, 64, 9, 25, 0.5)])
def test_illuminated_region_matches_the_oracle(lib, n, m, side, step, frac):
    z_true, q_true, pos, _, _ = _problem(n, m, side, step, seed=11 + n)
    mask = _region_gpu(lib, q_true, pos, n, frac).cpu().numpy().astype(bool)
    ref = O.illuminated_region(q_true.astype(np.complex128), pos, (n, n), frac)
    # the two sides may differ only at pixels whose illumination ties the threshold to rounding
    illum = np.zeros((n, n))
    a2 = np.abs(q_true.astype(np.complex128)) ** 2
    for r0, c0 in pos:
        rs, cs = max(r0, 0), max(c0, 0)
        re_, ce = min(r0 + m, n), min(c0 + m, n)
        illum[rs:re_, cs:ce] += a2[rs - r0:re_ - r0, cs - c0:ce - c0]
    tie = np.abs(illum - frac * illum.max()) <= 1e-12 * illum.max()
    assert np.array_equal(mask[~tie], ref[~tie])
    assert 0 < mask.sum() < n * n


@pytest.mark.parametrize("n,m,side,step", [(96, 32, 6, 10), (512, 128, 30, 12)])
@pytest.mark.parametrize("with_region", [True, False])
def test_aligned_errors_match_the_oracle(lib, n, m, side, step, with_region):
    import torch

    z_true, q_true, pos, z, q = _problem(n, m, side, step, seed=5 + n)
    stream = torch.cuda.current_stream().cuda_stream
    zd, zr = torch.from_numpy(z).cuda(), torch.from_numpy(z_true).cuda()
    qd, qr = torch.from_numpy(q).cuda(), torch.from_numpy(q_true).cuda()
    region = _region_gpu(lib, q_true, pos, n, 0.1) if with_region else None
    got = lib.emg_aligned_errors(zd.data_ptr(), zr.data_ptr(), n, n, qd.data_ptr(), qr.data_ptr(), m,
                                 region.data_ptr() if region is not None else 0, stream)
    mask = region.cpu().numpy().astype(bool) if region is not None else np.ones((n, n), dtype=bool)
    ref = O.aligned_errors(z.astype(np.complex128), q.astype(np.complex128), z_true.astype(np.complex128),
                           q_true.astype(np.complex128), mask)
    assert abs(got["c"] - ref["c"]) <= 1e-12 * abs(ref["c"])
    for key in ("object", "probe", "phase_rms"):
        assert abs(got[key] - ref[key]) <= 1e-9 * ref[key], key
    # the scale found undoes the one applied to the state (about 1 / 0.7 e^{-2.1 i})
    assert abs(got["c"] * 0.7 * np.exp(2.1j) - 1) < 0.05
    # bitwise repeatable
    again = lib.emg_aligned_errors(zd.data_ptr(), zr.data_ptr(), n, n, qd.data_ptr(), qr.data_ptr(), m,
                                   region.data_ptr() if region is not None else 0, stream)
    assert again == got


def test_aligned_errors_are_zero_for_a_scaled_truth(lib):
    import torch

    z_true, q_true, pos, _, _ = _problem(128, 32, 8, 12, seed=3)
    c = np.complex64(1.3 - 0.4j)
    zd = torch.from_numpy((z_true * c).astype(np.complex64)).cuda()
    qd = torch.from_numpy((q_true / c).astype(np.complex64)).cuda()
    zr, qr = torch.from_numpy(z_true).cuda(), torch.from_numpy(q_true).cuda()   # kept alive across the call
    got = lib.emg_aligned_errors(zd.data_ptr(), zr.data_ptr(), 128, 128, qd.data_ptr(), qr.data_ptr(), 32, 0,
                                 torch.cuda.current_stream().cuda_stream)
    assert abs(got["c"] * complex(c) - 1) < 1e-6
    assert got["object"] < 1e-6 and got["probe"] < 1e-6 and got["phase_rms"] < 1e-6
