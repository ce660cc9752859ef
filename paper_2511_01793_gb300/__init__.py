"""Python binding of the GB300 eMAGPIE library (C ABI of ``include/emagpie.h``).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libemagpie.so``.  There is no CPU fallback; ``load()`` raises if
the shared library has not been built (``build()``).

Functions keep the C names (``emg_create``, ``emg_run_epochs`` ...).  Device
buffers are passed as integer addresses (e.g. ``tensor.data_ptr()``); host
buffers as numpy arrays.  Complex arrays are complex64.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "EMG_OK", "EMG_EINVAL", "EMG_ENOMEM", "EMG_ECUDA", "EMG_ETIMEOUT", "EMG_ENOTSUP",
    "EMG_PROLONG_CONST", "EMG_PROLONG_BILINEAR", "EMG_COMBINE_WAVG", "EMG_COMBINE_SUM",
    "EMG_SCATTER_DETERMINISTIC", "EMG_SCATTER_ATOMIC", "EMG_DFT_FFT32", "EMG_DFT_BF16X3", "EmgError", "EmgProblem", "EmgParams",
    "build", "load", "lib_path", "exported_symbols", "emg_default_params", "emg_status_string",
    "emg_create", "emg_set_intensity", "emg_bind_state", "emg_normalize_probe",
    "emg_step_minibatch", "emg_position_stats", "emg_set_verify", "emg_run_epochs", "emg_misfit",
    "emg_set_epoch", "emg_schedule_permutation", "emg_stopping_epoch", "emg_run_until", "emg_reconstruct_host",
    "emg_simulate_intensity", "emg_fft2", "emg_dft2_bf16x3", "emg_dft_bf16x3_form", "emg_aligned_errors", "emg_shard_step",
    "emg_shard_apply",
    "emg_illuminated_region", "emg_step_minibatch_noalloc", "emg_misfit_gradient",
    "emg_set_cluster", "emg_set_prep_fusion", "emg_debug_prep_wait_extra", "emg_set_gradient_chunk", "emg_autotune", "emg_set_minibatch", "emg_set_scatter",
    "emg_selftest_bounded_wait", "emg_debug_fail_alloc", "emg_debug_bounds_errors",
    "emg_debug_bounds_selftest",
    "emg_autotune_search", "EmgTuneRequest", "EmgTuneResult", "emg_batch_create", "emg_batch_run_epochs", "emg_batch_destroy",
    "emg_set_profiling",
    "emg_profile_read",
    "emg_last_error", "emg_destroy", "Context",
]

EMG_OK, EMG_EINVAL, EMG_ENOMEM, EMG_ECUDA, EMG_ETIMEOUT, EMG_ENOTSUP = range(6)
EMG_PROLONG_CONST, EMG_PROLONG_BILINEAR = 0, 1
EMG_COMBINE_WAVG, EMG_COMBINE_SUM = 0, 1
EMG_SCATTER_DETERMINISTIC, EMG_SCATTER_ATOMIC = 0, 1
EMG_DFT_FFT32, EMG_DFT_BF16X3 = 0, 1

_STATUS_NAMES = ["EMG_OK", "EMG_EINVAL", "EMG_ENOMEM", "EMG_ECUDA", "EMG_ETIMEOUT", "EMG_ENOTSUP"]


class EmgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}" + (f" ({msg})" if msg else ""))


class EmgProblem(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("m", ctypes.c_int32),
                ("n_pos", ctypes.c_int32), ("pos", ctypes.c_void_p), ("intensity", ctypes.c_void_p)]


class EmgParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("levels", ctypes.c_int32), ("minibatch", ctypes.c_int32),
                ("prolong", ctypes.c_int32), ("combine", ctypes.c_int32), ("scatter", ctypes.c_int32),
                ("joint", ctypes.c_int32), ("w_eps", ctypes.c_float), ("dft", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_lib: Optional[ctypes.CDLL] = None

_I32P = ctypes.POINTER(ctypes.c_int32)
class EmgTuneRequest(ctypes.Structure):
    _fields_ = [("minibatch", ctypes.c_void_p), ("n_minibatch", ctypes.c_int32), ("trial_epochs", ctypes.c_int32),
                ("tune_tiling", ctypes.c_int32), ("allow_atomic", ctypes.c_int32)]


class EmgTuneResult(ctypes.Structure):
    _fields_ = [("minibatch", ctypes.c_int32), ("cluster", ctypes.c_int32), ("scatter", ctypes.c_int32),
                ("ms_per_epoch", ctypes.c_double), ("misfit_rate", ctypes.c_double)]


_F64P = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_SIGS = {
    "emg_default_params": (ctypes.c_int, [ctypes.POINTER(EmgParams)]),
    "emg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "emg_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(EmgProblem),
                                  ctypes.POINTER(EmgParams), _VP]),
    "emg_set_intensity": (ctypes.c_int, [_VP, _VP]),
    "emg_bind_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "emg_normalize_probe": (ctypes.c_int, [_VP]),
    "emg_step_minibatch": (ctypes.c_int, [_VP, _I32P, ctypes.c_int32, _F64P]),
    "emg_position_stats": (ctypes.c_int, [_VP, _F64P, ctypes.c_int32]),
    "emg_set_verify": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_run_epochs": (ctypes.c_int, [_VP, ctypes.c_int32, _I32P, _F64P, _F64P]),
    "emg_misfit": (ctypes.c_int, [_VP, _F64P]),
    "emg_set_epoch": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "emg_schedule_permutation": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, _I32P]),
    "emg_reconstruct_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int32, _I32P, _F64P, _F64P]),
    "emg_simulate_intensity": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_int32,
                                              _VP, ctypes.c_int32, _VP, _VP]),
    "emg_fft2": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP]),
    "emg_shard_step": (ctypes.c_int, [_VP, _I32P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]),
    "emg_shard_apply": (ctypes.c_int, [_VP, _I32P, ctypes.c_int32, _VP, _VP, _VP]),
    "emg_aligned_errors": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, ctypes.c_int32,
                                          _VP, _F64P, _VP]),
    "emg_illuminated_region": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, _VP, _VP]),
    "emg_stopping_epoch": (ctypes.c_int, [_F64P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int32)]),
    "emg_run_until": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int32), _F64P]),
    "emg_dft2_bf16x3": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP]),
    "emg_dft_bf16x3_form": (ctypes.c_int, [ctypes.c_int32, _I32P]),
    "emg_step_minibatch_noalloc": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_int32,
                                                  _VP, _VP, ctypes.c_int32, _I32P, ctypes.c_int32,
                                                  ctypes.POINTER(EmgParams), _VP]),
    "emg_misfit_gradient": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _F64P]),
    "emg_set_cluster": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_set_prep_fusion": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_debug_prep_wait_extra": (ctypes.c_int, [_VP, ctypes.c_uint32]),
    "emg_set_gradient_chunk": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_autotune": (ctypes.c_int, [_VP, _I32P, _F64P]),
    "emg_set_minibatch": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_selftest_bounded_wait": (ctypes.c_int, [_I32P]),
    "emg_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int32]),
    "emg_debug_bounds_errors": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    "emg_debug_bounds_selftest": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    "emg_set_scatter": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_autotune_search": (ctypes.c_int, [_VP, ctypes.POINTER(EmgTuneRequest), ctypes.POINTER(EmgTuneResult)]),
    "emg_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int32]),
    "emg_batch_run_epochs": (ctypes.c_int, [_VP, ctypes.c_int32, _VP]),
    "emg_batch_destroy": (None, [_VP]),
    "emg_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "emg_profile_read": (ctypes.c_int, [_VP, _F64P, ctypes.POINTER(ctypes.c_int64)]),
    "emg_last_error": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_char_p)]),
    "emg_destroy": (None, [_VP]),
}


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles ``libemagpie.so`` for sm_103a (in-tree) and returns its path."""
    return _build.build(force=force, verbose=verbose)


def lib_path() -> str:
    return _build.lib_path()


def load() -> ctypes.CDLL:
    """Loads the shared library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_2511_01793_gb300.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, where: str, ctx=None):
    if status != EMG_OK:
        msg = ""
        if ctx is not None:
            p = ctypes.c_char_p()
            if load().emg_last_error(ctx, ctypes.byref(p)) == EMG_OK and p.value:
                msg = p.value.decode(errors="replace")
        raise EmgError(status, where, msg)


def _i32(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _ptr_i32(a):
    return None if a is None else a.ctypes.data_as(_I32P)


def emg_default_params(**kw) -> EmgParams:
    p = EmgParams()
    _check(load().emg_default_params(ctypes.byref(p)), "emg_default_params")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def emg_status_string(s: int) -> str:
    return load().emg_status_string(s).decode()


def emg_create(problem: EmgProblem, params: EmgParams, stream: int = 0) -> int:
    ctx = _VP()
    _check(load().emg_create(ctypes.byref(ctx), ctypes.byref(problem), ctypes.byref(params),
                             _VP(stream)), "emg_create")
    return ctx.value


def emg_set_intensity(ctx: int, intensity) -> None:
    """intensity: device address (int) or a host float32 numpy array."""
    if isinstance(intensity, np.ndarray):
        arr = np.ascontiguousarray(intensity, dtype=np.float32)
        _check(load().emg_set_intensity(ctx, arr.ctypes.data), "emg_set_intensity", ctx)
    else:
        _check(load().emg_set_intensity(ctx, intensity), "emg_set_intensity", ctx)


def emg_bind_state(ctx: int, object_ptr: int, probe_ptr: int) -> None:
    _check(load().emg_bind_state(ctx, object_ptr, probe_ptr), "emg_bind_state", ctx)


def emg_normalize_probe(ctx: int) -> None:
    _check(load().emg_normalize_probe(ctx), "emg_normalize_probe", ctx)


def emg_step_minibatch(ctx: int, idx, want_misfit: bool = False) -> Optional[float]:
    a = _i32(idx)
    out = ctypes.c_double()
    _check(load().emg_step_minibatch(ctx, _ptr_i32(a), len(a),
                                     ctypes.byref(out) if want_misfit else None),
           "emg_step_minibatch", ctx)
    return out.value if want_misfit else None


def emg_position_stats(ctx: int, b: int) -> np.ndarray:
    out = np.zeros((b, 3), dtype=np.float64)
    _check(load().emg_position_stats(ctx, out.ctypes.data_as(_F64P), b), "emg_position_stats", ctx)
    return out


def emg_set_verify(ctx: int, verify: bool) -> None:
    _check(load().emg_set_verify(ctx, int(bool(verify))), "emg_set_verify", ctx)


def emg_run_epochs(ctx: int, n_epochs: int, order=None, running: bool = False,
                   misfit: bool = False):
    """Returns (running_misfit, misfit) arrays of length n_epochs (None when not asked)."""
    o = _i32(order)
    r = np.zeros(n_epochs) if running else None
    f = np.zeros(n_epochs) if misfit else None
    _check(load().emg_run_epochs(ctx, n_epochs, _ptr_i32(o),
                                 None if r is None else r.ctypes.data_as(_F64P),
                                 None if f is None else f.ctypes.data_as(_F64P)),
           "emg_run_epochs", ctx)
    return r, f


def emg_misfit(ctx: int) -> float:
    out = ctypes.c_double()
    _check(load().emg_misfit(ctx, ctypes.byref(out)), "emg_misfit", ctx)
    return out.value


def emg_set_epoch(ctx: int, epoch: int) -> None:
    _check(load().emg_set_epoch(ctx, epoch), "emg_set_epoch", ctx)


def emg_schedule_permutation(seed: int, epoch: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    _check(load().emg_schedule_permutation(seed, epoch, n, out.ctypes.data_as(_I32P)),
           "emg_schedule_permutation")
    return out


def emg_reconstruct_host(ctx: int, intensity: np.ndarray, obj: np.ndarray, probe: np.ndarray,
                         n_epochs: int, order=None, running: bool = False, misfit: bool = False):
    """Host-buffer end-to-end call; ``obj`` and ``probe`` (complex64, C-contiguous) are updated in place."""
    for name, arr in (("object", obj), ("probe", probe)):
        if arr.dtype != np.complex64 or not arr.flags.c_contiguous:
            raise TypeError(f"{name} must be a C-contiguous complex64 array")
    if intensity.dtype != np.float32 or not intensity.flags.c_contiguous:
        raise TypeError("intensity must be a C-contiguous float32 array")
    o = _i32(order)
    r = np.zeros(n_epochs) if running else None
    f = np.zeros(n_epochs) if misfit else None
    _check(load().emg_reconstruct_host(ctx, intensity.ctypes.data, obj.ctypes.data, probe.ctypes.data,
                                       n_epochs, _ptr_i32(o),
                                       None if r is None else r.ctypes.data_as(_F64P),
                                       None if f is None else f.ctypes.data_as(_F64P)),
           "emg_reconstruct_host", ctx)
    return r, f


def emg_simulate_intensity(object_ptr: int, n_rows: int, n_cols: int, probe_ptr: int, m: int,
                           pos_ptr: int, n_pos: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().emg_simulate_intensity(object_ptr, n_rows, n_cols, probe_ptr, m, pos_ptr, n_pos,
                                         out_ptr, _VP(stream)), "emg_simulate_intensity")


def emg_stopping_epoch(r, window: int = 5, patience: int = 10, floor: float = 0.0) -> int:
    """The outer iteration (1-based) at which the run stops, or 0 (Sec. 4.1, 4.3)."""
    a = np.ascontiguousarray(r, dtype=np.float64)
    out = ctypes.c_int32()
    _check(load().emg_stopping_epoch(a.ctypes.data_as(_F64P), len(a), window, patience, floor, ctypes.byref(out)),
           "emg_stopping_epoch")
    return int(out.value)


def emg_run_until(ctx: int, max_epochs: int, window: int = 5, patience: int = 10, floor: float = 0.0):
    """Runs epochs until the stopping rules fire; returns the residual after each epoch."""
    hist = np.zeros(max(max_epochs, 1), dtype=np.float64)
    n = ctypes.c_int32()
    _check(load().emg_run_until(ctx, max_epochs, window, patience, floor, ctypes.byref(n),
                                hist.ctypes.data_as(_F64P)), "emg_run_until", ctx)
    return hist[:n.value].copy()


def emg_fft2(in_ptr: int, out_ptr: int, m: int, count: int, inverse: bool, stream: int = 0) -> None:
    _check(load().emg_fft2(in_ptr, out_ptr, m, count, int(bool(inverse)), _VP(stream)), "emg_fft2")


def emg_shard_step(ctx: int, idx, slot_begin: int, slot_end: int, zt_ptr: int, qt_ptr: int, mu_ptr: int) -> None:
    """The per-position step for slots [slot_begin, slot_end) of minibatch idx into caller buffers."""
    a = _i32(idx)
    _check(load().emg_shard_step(ctx, _ptr_i32(a), len(a), slot_begin, slot_end, zt_ptr, qt_ptr, mu_ptr),
           "emg_shard_step", ctx)


def emg_shard_apply(ctx: int, idx, zt_ptr: int, qt_ptr: int, mu_ptr: int) -> None:
    """The combine of all slots of minibatch idx from caller buffers (after the exchange)."""
    a = _i32(idx)
    _check(load().emg_shard_apply(ctx, _ptr_i32(a), len(a), zt_ptr, qt_ptr, mu_ptr), "emg_shard_apply", ctx)


def emg_aligned_errors(object_ptr: int, object_ref_ptr: int, n_rows: int, n_cols: int, probe_ptr: int,
                       probe_ref_ptr: int, m: int, region_ptr: int = 0, stream: int = 0) -> dict:
    """FP64 errors after the best scale c (z -> c z, Q -> Q / c); see include/emagpie.h."""
    out = np.zeros(5, dtype=np.float64)
    _check(load().emg_aligned_errors(object_ptr, object_ref_ptr, n_rows, n_cols, probe_ptr, probe_ref_ptr, m,
                                     region_ptr or None, out.ctypes.data_as(_F64P), _VP(stream)),
           "emg_aligned_errors")
    return dict(c=complex(out[0], out[1]), object=float(out[2]), probe=float(out[3]), phase_rms=float(out[4]))


def emg_illuminated_region(probe_ref_ptr: int, m: int, pos_ptr: int, n_pos: int, n_rows: int, n_cols: int,
                           frac: float, region_ptr: int, stream: int = 0) -> None:
    """Writes the uint8 mask of pixels with summed illumination >= frac * max."""
    _check(load().emg_illuminated_region(probe_ref_ptr, m, pos_ptr, n_pos, n_rows, n_cols, float(frac),
                                         region_ptr, _VP(stream)), "emg_illuminated_region")


def emg_dft2_bf16x3(in_ptr: int, out_ptr: int, m: int, count: int, inverse: bool, stream: int = 0) -> None:
    _check(load().emg_dft2_bf16x3(in_ptr, out_ptr, m, count, int(bool(inverse)), _VP(stream)),
           "emg_dft2_bf16x3")


def emg_dft_bf16x3_form(m: int) -> bool:
    """True if the tensor-core DFT of size m runs as radix-16 passes in this process, False if dense."""
    v = ctypes.c_int32(0)
    _check(load().emg_dft_bf16x3_form(m, ctypes.byref(v)), "emg_dft_bf16x3_form")
    return bool(v.value)


def emg_step_minibatch_noalloc(object_ptr: int, n_rows: int, n_cols: int, probe_ptr: int, m: int,
                               pos_ptr: int, intensity_ptr: int, n_pos: int, idx,
                               params: EmgParams, stream: int = 0) -> None:
    """Allocation-free minibatch step (no context); see include/emagpie.h."""
    a = _i32(idx)
    _check(load().emg_step_minibatch_noalloc(object_ptr, n_rows, n_cols, probe_ptr, m, pos_ptr,
                                             intensity_ptr, n_pos, _ptr_i32(a), len(a),
                                             ctypes.byref(params), _VP(stream)),
           "emg_step_minibatch_noalloc")


def emg_misfit_gradient(ctx: int, object_ptr: int, probe_ptr: int, grad_object_ptr: int = 0,
                        grad_probe_ptr: int = 0, want_misfit: bool = True) -> Optional[float]:
    """Misfit and Wirtinger gradients at (object, probe); gradient pointers may be 0."""
    out = ctypes.c_double()
    _check(load().emg_misfit_gradient(ctx, object_ptr, probe_ptr, grad_object_ptr or None,
                                      grad_probe_ptr or None,
                                      ctypes.byref(out) if want_misfit else None),
           "emg_misfit_gradient", ctx)
    return out.value if want_misfit else None


def emg_set_gradient_chunk(ctx: int, positions: int) -> None:
    """Positions per gradient launch (0, the default: a multiple of the resident position clusters)."""
    _check(load().emg_set_gradient_chunk(ctx, positions), "emg_set_gradient_chunk", ctx)


def emg_set_prep_fusion(ctx: int, enable: bool) -> None:
    _check(load().emg_set_prep_fusion(ctx, int(bool(enable))), "emg_set_prep_fusion", ctx)


def emg_debug_prep_wait_extra(ctx: int, extra: int) -> None:
    """Test hook: later step launches wait for `extra` prep tiles that never come (0: off)."""
    _check(load().emg_debug_prep_wait_extra(ctx, extra), "emg_debug_prep_wait_extra", ctx)


def emg_set_cluster(ctx: int, cluster: int) -> None:
    _check(load().emg_set_cluster(ctx, cluster), "emg_set_cluster", ctx)


def emg_debug_fail_alloc(after: int) -> None:
    """Fault injection: the device allocation after `after` successful ones fails once (-1: off)."""
    _check(load().emg_debug_fail_alloc(after), "emg_debug_fail_alloc")


def emg_debug_bounds_errors() -> Optional[int]:
    """The bounds-check build's error word (cleared on read); None in a build without the checks."""
    out = ctypes.c_uint32()
    st = load().emg_debug_bounds_errors(ctypes.byref(out))
    if st == EMG_ENOTSUP:
        return None
    _check(st, "emg_debug_bounds_errors")
    return out.value


def emg_debug_bounds_selftest() -> Optional[int]:
    """The error word after one check that must fail; None in a build without the checks."""
    out = ctypes.c_uint32()
    st = load().emg_debug_bounds_selftest(ctypes.byref(out))
    if st == EMG_ENOTSUP:
        return None
    _check(st, "emg_debug_bounds_selftest")
    return out.value


def emg_selftest_bounded_wait() -> int:
    """1 when a bounded device wait that nothing satisfies gave up and reported it."""
    out = ctypes.c_int32()
    _check(load().emg_selftest_bounded_wait(ctypes.byref(out)), "emg_selftest_bounded_wait")
    return out.value


def emg_set_minibatch(ctx: int, minibatch: int) -> None:
    _check(load().emg_set_minibatch(ctx, minibatch), "emg_set_minibatch", ctx)


def emg_set_scatter(ctx: int, scatter: int) -> None:
    _check(load().emg_set_scatter(ctx, scatter), "emg_set_scatter", ctx)


def emg_autotune_search(ctx: int, minibatch=(), trial_epochs: int = 2, tune_tiling: bool = True,
                        allow_atomic: bool = False) -> dict:
    """Chooses B (largest misfit decrease per second), then the FFT tiling and
    optionally the scatter mode; sets them on the context and returns them."""
    cands = np.ascontiguousarray(list(minibatch), dtype=np.int32)
    req = EmgTuneRequest(cands.ctypes.data if len(cands) else None, len(cands), trial_epochs,
                         int(tune_tiling), int(allow_atomic))
    res = EmgTuneResult()
    _check(load().emg_autotune_search(ctx, ctypes.byref(req), ctypes.byref(res)), "emg_autotune_search", ctx)
    return {"minibatch": res.minibatch, "cluster": res.cluster, "scatter": res.scatter,
            "ms_per_epoch": res.ms_per_epoch, "misfit_rate": res.misfit_rate}


def emg_autotune(ctx: int):
    """Returns (chosen cluster size, ms per minibatch)."""
    c = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load().emg_autotune(ctx, ctypes.byref(c), ctypes.byref(ms)), "emg_autotune", ctx)
    return c.value, ms.value


def emg_batch_create(ctxs) -> int:
    arr = (_VP * len(ctxs))(*ctxs)
    out = _VP()
    _check(load().emg_batch_create(ctypes.byref(out), arr, len(ctxs)), "emg_batch_create")
    return out.value


def emg_batch_run_epochs(batch: int, n_epochs: int, stream: int = 0) -> None:
    _check(load().emg_batch_run_epochs(batch, n_epochs, _VP(stream)), "emg_batch_run_epochs")


def emg_batch_destroy(batch: int) -> None:
    if batch:
        load().emg_batch_destroy(batch)


def emg_set_profiling(ctx: int, enable: bool) -> None:
    _check(load().emg_set_profiling(ctx, int(bool(enable))), "emg_set_profiling", ctx)


PROFILE_KINDS = ("prep", "step", "apply", "other", "dft")


def emg_profile_read(ctx: int):
    """Returns {kind: (milliseconds, launches)} since the last read."""
    ms = np.zeros(len(PROFILE_KINDS), dtype=np.float64)
    n = np.zeros(len(PROFILE_KINDS), dtype=np.int64)
    _check(load().emg_profile_read(ctx, ms.ctypes.data_as(_F64P),
                                   n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "emg_profile_read", ctx)
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROFILE_KINDS)}


def emg_last_error(ctx: int) -> str:
    p = ctypes.c_char_p()
    _check(load().emg_last_error(ctx, ctypes.byref(p)), "emg_last_error")
    return (p.value or b"").decode(errors="replace")


def emg_destroy(ctx: int) -> None:
    if ctx:
        load().emg_destroy(ctx)


class Context:
    """A reconstruction context holding torch device tensors for its state.

    PyTorch supplies device memory and the stream; all arithmetic runs in the
    library's kernels.  ``obj`` and ``probe`` are complex64 CUDA tensors that
    the library updates in place.
    """

    def __init__(self, pos, intensity, n_rows: int, n_cols: int, params: EmgParams,
                 obj=None, probe=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the eMAGPIE library needs a CUDA device")
        dev = torch.device("cuda", torch.cuda.current_device())

        def on_device(x, np_dtype, t_dtype):
            if isinstance(x, torch.Tensor):
                return x.to(device=dev, dtype=t_dtype).contiguous()
            return torch.as_tensor(np.ascontiguousarray(x, dtype=np_dtype)).to(dev)

        self.pos = on_device(pos, np.int32, torch.int32)
        self.intensity = on_device(intensity, np.float32, torch.float32)
        n_pos, m = int(self.intensity.shape[0]), int(self.intensity.shape[-1])
        self.m, self.n_pos = m, n_pos
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prob = EmgProblem(n_rows, n_cols, m, n_pos, self.pos.data_ptr(), self.intensity.data_ptr())
        self.params = params
        self.ctx = emg_create(prob, params, self.stream.cuda_stream)
        if obj is not None and probe is not None:
            self.bind(obj, probe)

    def bind(self, obj, probe):
        import torch

        self.obj = torch.as_tensor(obj).to(torch.complex64).cuda().contiguous()
        self.probe = torch.as_tensor(probe).to(torch.complex64).cuda().contiguous()
        emg_bind_state(self.ctx, self.obj.data_ptr(), self.probe.data_ptr())

    def close(self):
        if getattr(self, "ctx", None):
            emg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
