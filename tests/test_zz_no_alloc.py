"""The allocation-free minibatch step against the context-based one.

emg_step_minibatch_noalloc serves callers that may not allocate device memory
(code living inside a memory pool or arena it does not own, code whose device
footprint is frozen after start-up, or code whose host policy forbids
cudaMalloc on the hot path).  Its only scratch is one fixed device array
compiled into the library.  These tests call it through the C ABI twice in a
row, each time from the state the previous call left, and compare it with
emg_step_minibatch run on the same inputs; the second call also shows that
whatever the first call left in the shared scratch does not leak into the
next result.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from emg_cases import Case, covered_mask, gpu_params, make_context, oracle_params, rel_err, state

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5


@pytest.mark.parametrize("m,levels,prolong,b1,b2", [(32, 2, "const", 12, 7), (128, 3, "bilinear", 9, 5)])
def test_noalloc_step_matches_the_context_step_twice(lib, m, levels, prolong, b1, b2):
    import torch

    case = Case(n=2 * m + 40, m=m, side=4, noise_peak=1e5, seed=31 + m)
    p = oracle_params(alpha=0.05, levels=levels, minibatch=max(b1, b2), prolong=prolong)
    rng = np.random.default_rng(77)
    perm = rng.permutation(case.n_pos)
    idx1 = perm[:b1].astype(np.int32)
    idx2 = perm[b1:b1 + b2].astype(np.int32)

    ref = make_context(lib, case, p)
    z_na = torch.from_numpy(case.z0.copy()).cuda()
    q_na = torch.from_numpy(case.q0.copy()).cuda()
    pos = torch.from_numpy(case.pos).cuda()
    d = torch.from_numpy(case.d).cuda()
    params = gpu_params(lib, p)
    for idx in (idx1, idx2):
        z_before = z_na.cpu().numpy().astype(np.complex128)
        lib.emg_step_minibatch(ref.ctx, idx)
        lib.emg_step_minibatch_noalloc(z_na.data_ptr(), case.n, case.n, q_na.data_ptr(), m,
                                       pos.data_ptr(), d.data_ptr(), case.n_pos, idx, params,
                                       torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        z_r, q_r = state(ref)
        z_n = z_na.cpu().numpy().astype(np.complex128)
        q_n = q_na.cpu().numpy().astype(np.complex128)
        mask = covered_mask(case, idx)
        assert rel_err(z_n, z_r, mask) <= STEP_TOL
        assert rel_err(z_n, z_r) <= STEP_TOL
        assert rel_err(q_n, q_r) <= STEP_TOL
        assert np.array_equal(z_n[~mask], z_before[~mask])   # pixels outside the minibatch untouched
    ref.close()


def test_noalloc_rejects_requests_beyond_its_fixed_scratch(lib):
    import torch

    m = 128
    case = Case(n=300, m=m, side=6, seed=5)
    p = oracle_params(levels=3, minibatch=case.n_pos, prolong="bilinear")
    z = torch.from_numpy(case.z0.copy()).cuda()
    q = torch.from_numpy(case.q0.copy()).cuda()
    pos = torch.from_numpy(case.pos).cuda()
    d = torch.from_numpy(case.d).cuda()
    idx = np.arange(case.n_pos, dtype=np.int32)           # 40 positions of 128 x 128: too many
    raw = lib.load()
    st = raw.emg_step_minibatch_noalloc(z.data_ptr(), case.n, case.n, q.data_ptr(), m, pos.data_ptr(),
                                        d.data_ptr(), case.n_pos, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        len(idx), ctypes.byref(gpu_params(lib, p)), None)
    assert st == lib.EMG_EINVAL
    torch.cuda.synchronize()
    assert np.array_equal(z.cpu().numpy(), case.z0)      # nothing was enqueued
