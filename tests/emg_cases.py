"""Shared helpers of the GPU parity tests: identical seeded inputs for the
CUDA library and the FP64 oracle, and the library run through its C ABI."""
from __future__ import annotations

import math

import numpy as np

import oracle as O
import synth


def c64(x):
    return np.ascontiguousarray(x, dtype=np.complex64)


def rel_err(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    """A small problem with FP32-rounded inputs shared by both implementations."""

    def __init__(self, n=96, m=32, side=5, step=None, jitter=2, seed=7, edge=True,
                 noise_peak=None, state="perturbed", pert=0.3):
        rng = np.random.Generator(np.random.PCG64(seed))
        step = step if step is not None else max(m // 4, 2)
        self.n, self.m = n, m
        self.z_true = c64(synth.make_object(n, n, rng, phi_max=1.2, sigma=3.0))
        self.q_true = c64(synth.make_probe(m, radius=m / 3.2))
        pos = synth.make_scan(n, m, side, step, jitter, rng).astype(np.int64)
        if edge:
            # patches that leave the object (zero-padding of P_k) and one fully outside
            extra = np.array([[-m // 3, n // 3], [n - m + m // 4, -m // 5], [n - m // 2, n - m // 3],
                              [-m - 3, 5]], dtype=np.int64)
            pos = np.concatenate([pos, extra])
        self.pos = pos.astype(np.int32)
        d = O.forward_intensity(self.q_true.astype(np.complex128), self.z_true.astype(np.complex128), self.pos)
        if noise_peak is not None:
            d = synth.poisson_noise(d, noise_peak, rng)
        self.d = np.ascontiguousarray(d, dtype=np.float32)
        self.a64 = np.sqrt(np.maximum(self.d.astype(np.float64), 0.0))
        if state == "perturbed":
            self.z0 = c64(synth.perturb(self.z_true, pert, rng))
            self.q0 = c64(synth.perturb(self.q_true, pert, rng))
        else:
            self.z0 = c64(np.ones((n, n)))
            self.q0 = c64(O.dp_avg_scale(synth.blur_probe(self.q_true.astype(np.complex128), 2.0),
                                         self.d.astype(np.float64)))

    @property
    def n_pos(self):
        return len(self.pos)


def oracle_params(alpha=0.05, levels=1, minibatch=8, prolong="const", combine="wavg", w_eps=1e-6,
                  joint=True):
    return O.Params(alpha=alpha, levels=levels, minibatch=minibatch, prolong=prolong,
                    combine=combine, w_eps=w_eps, joint=joint)


def gpu_params(emg, p: O.Params, seed=0, dft=0, scatter=0):
    return emg.emg_default_params(
        alpha=float(np.float32(p.alpha)), levels=p.levels, minibatch=p.minibatch,
        prolong=emg.EMG_PROLONG_CONST if p.prolong == "const" else emg.EMG_PROLONG_BILINEAR,
        combine=emg.EMG_COMBINE_WAVG if p.combine == "wavg" else emg.EMG_COMBINE_SUM,
        joint=int(p.joint), w_eps=float(np.float32(p.w_eps)), seed=seed, dft=dft, scatter=scatter)


def oracle_inputs(case: Case, p: O.Params):
    """FP64 copies of the exact FP32 inputs; alpha and w_eps as the GPU sees them."""
    q = O.Params(alpha=float(np.float32(p.alpha)), levels=p.levels, minibatch=p.minibatch,
                 prolong=p.prolong, combine=p.combine, w_eps=float(np.float32(p.w_eps)),
                 joint=p.joint)
    return (case.z0.astype(np.complex128), case.q0.astype(np.complex128), case.pos, case.a64, q)


def make_context(emg, case: Case, p: O.Params, seed=0, dft=0, scatter=0):
    import torch

    ctx = emg.Context(case.pos, case.d, case.n, case.n, gpu_params(emg, p, seed, dft, scatter),
                      obj=torch.from_numpy(case.z0), probe=torch.from_numpy(case.q0))
    return ctx


def state(ctx):
    import torch

    torch.cuda.synchronize()
    return ctx.obj.cpu().numpy().astype(np.complex128), ctx.probe.cpu().numpy().astype(np.complex128)


def covered_mask(case: Case, idx):
    mask = np.zeros((case.n, case.n), dtype=bool)
    for k in idx:
        r0, c0 = case.pos[k]
        rs, re_ = max(r0, 0), min(r0 + case.m, case.n)
        cs, ce = max(c0, 0), min(c0 + case.m, case.n)
        if re_ > rs and ce > cs:
            mask[rs:re_, cs:ce] = True
    return mask


def log_rel(a, b):
    return math.log10(max(rel_err(a, b), 1e-30))


def jiggle(x, seed):
    """x perturbed by about one FP32 rounding (2^-24 relative), seeded."""
    rng = np.random.default_rng(1000 + seed)
    return x * (1 + 2.0 ** -24 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)))


def oracle_epoch_states(args):
    """FP64 oracle epochs from (z0, q0), optionally jiggled: per epoch the
    end-of-epoch misfit, the running misfit and the state (z, Q).  Runs in a
    spawned worker process."""
    z0, q0, pos, a, orders, p, member = args
    if member is not None:
        z0, q0 = jiggle(z0, member), jiggle(q0, 500 + member)
    z, q = z0, q0
    out = []
    for order in orders:
        z, q, hist = O.run_epochs(z, q, pos, a, order[None, :], p)
        out.append((hist[0]["misfit"], hist[0]["running_misfit"], z.astype(np.complex128), q.astype(np.complex128)))
    return out


def oracle_ensemble_states(z0, q0, pos, a, orders, p, members):
    """The central oracle run and `members` runs from jiggled inputs, in
    parallel spawned processes (the oracle is single-threaded)."""
    import multiprocessing as mp
    import os

    jobs = [(z0, q0, pos, a, orders, p, None)] + [(z0, q0, pos, a, orders, p, s) for s in range(members)]
    procs = min(len(jobs), max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(oracle_epoch_states, jobs)
    return res[0], res[1:]


def epoch_deviations(gpu, central, members, region):
    """Per epoch: the GPU's deviation from the central oracle run, and the
    envelope of the oracle ensemble: the largest deviation between any two of
    its runs (the central one and the jiggled members), as a running maximum
    over epochs.  The GPU passes when it is no farther from the oracle than the
    oracle's own rounding-level runs are from one another.  Quantities: the
    end-of-epoch misfit and the running misfit (relative), and the aligned
    object, probe and RMS phase errors.  Each run is a list of (Phi, running, z, Q)."""
    keys = ("misfit", "running", "object", "probe", "phase")

    def dev(run, ref):
        rows = []
        for (mg, rg, zg, qg), (mo, ro, zo, qo) in zip(run, ref):
            e = O.aligned_errors(zg, qg, zo, qo, region)
            rows.append([abs(mg - mo) / mo, abs(rg - ro) / ro, e["object"], e["probe"], e["phase_rms"]])
        return np.array(rows)

    d_gpu = dev(gpu, central)
    runs = [central] + list(members)
    env = np.max(np.stack([dev(runs[i], runs[j]) for i in range(len(runs)) for j in range(len(runs)) if i != j]),
                 axis=0)
    env = np.maximum.accumulate(env, axis=0)
    return keys, d_gpu, env
