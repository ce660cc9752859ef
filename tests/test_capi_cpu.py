"""The C ABI without a GPU: library builds, loads, exports every declared
symbol, and its host-only logic (schedule, validation) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2511_01793_gb300 as emg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    emg.build()
    return emg.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "emagpie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_surface():
    assert _declared_functions() == sorted(emg.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_defaults(lib):
    assert emg.emg_status_string(emg.EMG_EINVAL) == "EMG_EINVAL"
    p = emg.emg_default_params()
    assert abs(p.alpha - 0.01) < 1e-9 and p.levels == 1 and p.minibatch == 1 and p.joint == 1
    assert p.prolong == emg.EMG_PROLONG_CONST and p.combine == emg.EMG_COMBINE_WAVG


@pytest.mark.parametrize("seed,epoch,n", [(0, 0, 10), (42, 3, 97), (2**63 + 5, 11, 900)])
def test_schedule_matches_the_oracle(lib, seed, epoch, n):
    got = emg.emg_schedule_permutation(seed, epoch, n)
    assert got.tolist() == O.schedule_permutation(seed, epoch, n)


def _problem(m=32, n_pos=4):
    # pointers are never dereferenced: validation fails before any device work
    return emg.EmgProblem(64, 64, m, n_pos, 0x1000, 0x2000)


@pytest.mark.parametrize("field,value,expect", [
    ("alpha", 0.0, emg.EMG_EINVAL),
    ("alpha", float("nan"), emg.EMG_EINVAL),
    ("levels", 0, emg.EMG_EINVAL),
    ("levels", 6, emg.EMG_EINVAL),          # 32 / 2^5 = 1 < 2
    ("minibatch", 0, emg.EMG_EINVAL),
    ("minibatch", 5, emg.EMG_EINVAL),       # > n_pos
    ("prolong", 7, emg.EMG_EINVAL),
    ("combine", 3, emg.EMG_EINVAL),
    ("scatter", 2, emg.EMG_EINVAL),
    ("joint", 2, emg.EMG_EINVAL),
    ("w_eps", -1.0, emg.EMG_EINVAL),
    ("dft", 2, emg.EMG_EINVAL),
    ("dft", emg.EMG_DFT_BF16X3, emg.EMG_ENOTSUP),   # m = 32: the tensor-core DFT needs m = 128 or 256
])
def test_create_rejects_bad_parameters_before_any_launch(lib, field, value, expect):
    p = emg.emg_default_params()
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    st = lib.emg_create(ctypes.byref(ctx), ctypes.byref(_problem()), ctypes.byref(p), None)
    assert st == expect
    assert ctx.value is None


def test_atomic_weighted_mean_scatter_needs_a_weight_floor(lib):
    p = emg.emg_default_params(scatter=emg.EMG_SCATTER_ATOMIC, w_eps=0.0)
    ctx = ctypes.c_void_p()
    assert lib.emg_create(ctypes.byref(ctx), ctypes.byref(_problem()), ctypes.byref(p), None) == emg.EMG_EINVAL


def test_create_rejects_bad_problems(lib):
    p = emg.emg_default_params()
    ctx = ctypes.c_void_p()
    for prob, expect in [
        (emg.EmgProblem(64, 64, 48, 4, 0x1000, 0x2000), emg.EMG_ENOTSUP),
        (emg.EmgProblem(64, 64, 512, 4, 0x1000, 0x2000), emg.EMG_ENOTSUP),
        (emg.EmgProblem(0, 64, 32, 4, 0x1000, 0x2000), emg.EMG_EINVAL),
        (emg.EmgProblem(64, 64, 32, 0, 0x1000, 0x2000), emg.EMG_EINVAL),
        (emg.EmgProblem(64, 64, 32, 4, 0, 0x2000), emg.EMG_EINVAL),
        (emg.EmgProblem(64, 64, 32, 4, 0x1000, 0), emg.EMG_EINVAL),
    ]:
        assert lib.emg_create(ctypes.byref(ctx), ctypes.byref(prob), ctypes.byref(p), None) == expect
    assert lib.emg_create(None, None, None, None) == emg.EMG_EINVAL


def test_context_free_calls_validate_arguments(lib):
    assert lib.emg_fft2(None, None, 32, 1, 0, None) == emg.EMG_EINVAL
    assert lib.emg_fft2(0x10, 0x10, 48, 1, 0, None) == emg.EMG_ENOTSUP
    assert lib.emg_fft2(0x10, 0x10, 32, 1, 2, None) == emg.EMG_EINVAL
    assert lib.emg_simulate_intensity(None, 8, 8, None, 32, None, 1, None, None) == emg.EMG_EINVAL
    assert lib.emg_schedule_permutation(1, -1, 4, None) == emg.EMG_EINVAL
    assert lib.emg_dft2_bf16x3(None, 0x10, 128, 1, 0, None) == emg.EMG_EINVAL
    assert lib.emg_dft2_bf16x3(0x10, 0x10, 128, 1, 0, None) == emg.EMG_EINVAL   # aliasing
    assert lib.emg_dft2_bf16x3(0x10, 0x20, 128, 1, 2, None) == emg.EMG_EINVAL
    assert lib.emg_dft2_bf16x3(0x10, 0x20, 64, 1, 0, None) == emg.EMG_ENOTSUP
    assert lib.emg_dft2_bf16x3(0x10, 0x20, 256, 0, 0, None) == emg.EMG_OK      # empty batch
    assert lib.emg_set_gradient_chunk(None, 0) == emg.EMG_EINVAL
    assert lib.emg_selftest_bounded_wait(None) == emg.EMG_EINVAL
    assert lib.emg_set_minibatch(None, 4) == emg.EMG_EINVAL
    assert lib.emg_set_scatter(None, 0) == emg.EMG_EINVAL
    assert lib.emg_autotune_search(None, None, None) == emg.EMG_EINVAL
    assert lib.emg_set_cluster(None, 2) == emg.EMG_EINVAL
    assert lib.emg_set_prep_fusion(None, 1) == emg.EMG_EINVAL
    assert lib.emg_debug_prep_wait_extra(None, 0) == emg.EMG_EINVAL
    idx = (ctypes.c_int32 * 2)(0, 1)
    assert lib.emg_shard_step(None, idx, 2, 0, 1, 0x10, 0x20, 0x30) == emg.EMG_EINVAL
    assert lib.emg_shard_apply(None, idx, 2, 0x10, 0x20, 0x30) == emg.EMG_EINVAL
    out = (ctypes.c_double * 5)()
    assert lib.emg_aligned_errors(None, 0x10, 8, 8, 0x20, 0x30, 4, None, out, None) == emg.EMG_EINVAL
    assert lib.emg_aligned_errors(0x10, 0x20, 0, 8, 0x30, 0x40, 4, None, out, None) == emg.EMG_EINVAL
    assert lib.emg_aligned_errors(0x10, 0x20, 8, 8, 0x30, 0x40, 4, None, None, None) == emg.EMG_EINVAL
    assert lib.emg_illuminated_region(None, 4, 0x10, 1, 8, 8, 0.1, 0x20, None) == emg.EMG_EINVAL
    assert lib.emg_illuminated_region(0x10, 4, 0x20, 1, 8, 8, float("nan"), 0x30, None) == emg.EMG_EINVAL
    assert lib.emg_illuminated_region(0x10, 4, 0x20, 0, 8, 8, 0.1, 0x30, None) == emg.EMG_EINVAL
    form = ctypes.c_int32(-1)
    assert lib.emg_dft_bf16x3_form(256, None) == emg.EMG_EINVAL
    assert lib.emg_dft_bf16x3_form(64, ctypes.byref(form)) == emg.EMG_ENOTSUP
    assert lib.emg_dft_bf16x3_form(128, ctypes.byref(form)) == emg.EMG_OK and form.value == 0
    assert lib.emg_dft_bf16x3_form(256, ctypes.byref(form)) == emg.EMG_OK
    assert form.value == (0 if os.environ.get("EMG_TC_RADIX16", "").startswith("0") else 1)
    lib.emg_destroy(None)  # no-op


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    monkeypatch.setattr(emg, "_lib", None)
    monkeypatch.setattr(emg._build, "OUT_DIR", str(tmp_path))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        emg.load()


def test_stopping_rule_matches_the_oracle(lib):
    """Host-only stopping criterion (Sec. 4.1) and noise-floor rule (Sec. 4.3)."""
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(0, 60))
        # a decaying residual with noise and plateaus, as a run produces
        r = np.maximum(1.0 + 10.0 * np.exp(-rng.uniform(0.02, 0.5) * np.arange(n))
                       + rng.normal(0, rng.choice([0.0, 0.01, 0.2]), n), 0.1)
        if trial % 3 == 0:
            r = np.round(r, 1)  # exact ties between averages
        w, p = int(rng.integers(1, 8)), int(rng.integers(1, 12))
        floor = float(rng.choice([0.0, 1.0, 1.2, 2.0]))
        assert emg.emg_stopping_epoch(r, w, p, floor) == O.stopping_epoch(list(r), w, p, floor)
    assert lib.emg_stopping_epoch(None, 3, 5, 10, 0.0, ctypes.byref(ctypes.c_int32())) == emg.EMG_EINVAL
    buf = (ctypes.c_double * 3)(1.0, 2.0, 3.0)
    out = ctypes.c_int32()
    assert lib.emg_stopping_epoch(buf, 3, 0, 10, 0.0, ctypes.byref(out)) == emg.EMG_EINVAL
    assert lib.emg_stopping_epoch(buf, 3, 5, 10, -1.0, ctypes.byref(out)) == emg.EMG_EINVAL
    assert lib.emg_stopping_epoch(buf, 0, 5, 10, 0.0, ctypes.byref(out)) == emg.EMG_OK and out.value == 0
