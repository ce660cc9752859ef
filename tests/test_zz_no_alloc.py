"""The allocation-free minibatch step against the context-based one.

emg_step_minibatch_noalloc serves callers that may not allocate device memory
(code living inside a memory pool or arena it does not own, code whose device
footprint is frozen after start-up, or code whose host policy forbids
cudaMalloc on the hot path).  Its only scratch is one fixed device array
compiled into the library.  These tests call it through the C ABI twice in a
row, each time from the state the previous call left, and compare it with
emg_step_minibatch run on the same inputs; the second call also shows that
whatever the first call left in the shared scratch does not leak into the
next result.  Two more cases: a pinned host idx array overwritten right after
the call (the indices travel in the launch parameters, so the step still uses
the ones passed), and the entry point as the very first library call of a
fresh process, where it does its own one-time set-up.  This file is collected
last on purpose.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

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


def test_noalloc_pinned_idx_may_be_overwritten_right_after_the_call(lib):
    import torch

    m, b = 64, 10
    case = Case(n=2 * m + 40, m=m, side=5, noise_peak=1e5, seed=91)
    p = oracle_params(alpha=0.05, levels=2, minibatch=b, prolong="bilinear")
    idx = np.random.default_rng(5).permutation(case.n_pos)[:b].astype(np.int32)
    ref = make_context(lib, case, p)
    lib.emg_step_minibatch(ref.ctx, idx)
    z_r, q_r = state(ref)
    ref.close()

    z = torch.from_numpy(case.z0.copy()).cuda()
    q = torch.from_numpy(case.q0.copy()).cuda()
    pos = torch.from_numpy(case.pos).cuda()
    d = torch.from_numpy(case.d).cuda()
    pinned = torch.from_numpy(idx.copy()).pin_memory()
    stream = torch.cuda.current_stream()
    busy = torch.randn(4096, 4096, device="cuda")
    for _ in range(8):                                    # keep the stream busy past the return
        busy = busy @ busy * 1e-3
    raw = lib.load()
    st = raw.emg_step_minibatch_noalloc(
        z.data_ptr(), case.n, case.n, q.data_ptr(), m, pos.data_ptr(), d.data_ptr(), case.n_pos,
        ctypes.cast(pinned.data_ptr(), ctypes.POINTER(ctypes.c_int32)), b,
        ctypes.byref(gpu_params(lib, p)), ctypes.c_void_p(stream.cuda_stream))
    assert st == lib.EMG_OK
    pinned.copy_(torch.from_numpy(np.arange(case.n_pos - b, case.n_pos, dtype=np.int32)))  # reuse at once
    torch.cuda.synchronize()
    assert rel_err(z.cpu().numpy().astype(np.complex128), z_r) <= STEP_TOL
    assert rel_err(q.cpu().numpy().astype(np.complex128), q_r) <= STEP_TOL


_FRESH_CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path[:0] = [{root!r}, {tests!r}]
    import paper_2511_01793_gb300 as emg
    from emg_cases import Case, gpu_params, oracle_params
    case = Case(n=2 * 64 + 40, m=64, side=5, noise_peak=1e5, seed=92)
    p = oracle_params(alpha=0.05, levels=3, minibatch=9, prolong="bilinear")
    idx = np.array({idx}, dtype=np.int32)
    z = torch.from_numpy(case.z0.copy()).cuda()
    q = torch.from_numpy(case.q0.copy()).cuda()
    pos = torch.from_numpy(case.pos).cuda()
    d = torch.from_numpy(case.d).cuda()
    # the first call into the library in this process
    emg.emg_step_minibatch_noalloc(z.data_ptr(), case.n, case.n, q.data_ptr(), 64, pos.data_ptr(),
                                   d.data_ptr(), case.n_pos, idx, gpu_params(emg, p),
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.savez({out!r}, z=z.cpu().numpy(), q=q.cpu().numpy())
""")


def test_noalloc_as_the_first_call_of_a_fresh_process(lib, tmp_path):
    idx = [3, 17, 8, 22, 0, 11, 26, 5, 14]
    out = str(tmp_path / "fresh.npz")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _FRESH_CHILD.format(root=root, tests=os.path.join(root, "tests"), idx=idx, out=out)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(out)

    case = Case(n=2 * 64 + 40, m=64, side=5, noise_peak=1e5, seed=92)
    p = oracle_params(alpha=0.05, levels=3, minibatch=9, prolong="bilinear")
    ref = make_context(lib, case, p)
    lib.emg_step_minibatch(ref.ctx, np.array(idx, dtype=np.int32))
    z_r, q_r = state(ref)
    ref.close()
    assert rel_err(got["z"].astype(np.complex128), z_r) <= STEP_TOL
    assert rel_err(got["q"].astype(np.complex128), q_r) <= STEP_TOL
