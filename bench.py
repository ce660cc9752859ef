#!/usr/bin/env python3
"""Throughput of the eMAGPIE hot path on GB300: scan positions per second per epoch.

Workload (one "step" = one eMAGPIE epoch over all scan positions): object
512 x 512 complex, probe 128 x 128, 900 scan positions (30 x 30 raster, step
12 px, +-2 px jitter), Poisson noise at 1e4 photons peak, 3 multigrid levels
with 2x averaging restriction and bilinear prolongation, minibatch 64,
alpha 0.05.  Inputs are synthetic and seeded (``synth``): the simulated
measurement of the true object and probe, Poisson-sampled on the host, the
same arrays in both arms.  The L2 cache (129 MB) is flushed by writing a 256 MB buffer before
every timed step; inputs are resident in HBM when a step starts.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(the reference arm); ``--gpus N`` under torchrun runs N independent replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "mg_n512_m128"
METRIC = "scan positions/sec per eMAGPIE epoch"
UNIT = "positions/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_stepc_mg_n512_m128.md")
CLUSTER = 4   # CTAs per position of the step kernel (the library's default for m = 128)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2511_01793_gb300", "csrc", f)
                  for f in ("emg_kernels.cu", "emg_fft.cuh")]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--shard", action="store_true",
                    help="default workload as ONE reconstruction whose minibatches are split across the "
                         "ranks (one all-gather of the slot results per minibatch; strong scaling) instead "
                         "of independent replicas")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="default workload only: skip the short runs of the gradient, batch and precision "
                         "workloads that ride along in the line")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "grad_n1024_m256", "batch64", "prec_n2048_m256"],
                    help="mg_n512_m128: eMAGPIE epochs (default); grad_n1024_m256: exit-wave "
                         "misfit gradient over all positions; batch64: 64 uneven reconstructions, "
                         "one graph launch per epoch; prec_n2048_m256: epochs with the DFT pair on "
                         "tensor cores (BF16 split) against FP32 FFTs, and time to the oracle's misfit")
    return ap.parse_args()


def workload_config(world: int = 1):
    """The workload description, identical in the GPU and the reference arm."""
    p = synth.CONFIGS[WORKLOAD]
    n_pos = p["side"] ** 2
    return {
        "workload": f"{WORKLOAD}: object {p['n']}x{p['n']} c64, probe {p['m']}x{p['m']}, "
                    f"{n_pos} positions ({p['side']}x{p['side']} raster, step {p['step']}, "
                    f"+-{p['jitter']} px jitter), Poisson peak {p['peak']:g}, {p['levels']} levels "
                    f"({p['prolong']} prolongation), minibatch {p['minibatch']}, alpha {p['alpha']}",
        "n": p["n"], "m": p["m"], "n_pos": n_pos, "minibatch": p["minibatch"],
        "levels": p["levels"], "prolong": p["prolong"], "alpha": p["alpha"],
        "l2": "flushed (256 MB write) before every timed step",
        "intensities": "synth.measure_intensities of the true object and probe, Poisson-sampled "
                       "(synth.poisson_noise, seed noise_seed + rank)",
        "parallelism": f"replicas{world}" if world > 1 else "single",
    }


def workload_intensities(w, rank: int = 0) -> np.ndarray:
    """The default workload's data: the simulated measurement, Poisson-sampled on the host."""
    d_clean = synth.measure_intensities(w.z_true, w.q_true, w.pos)
    rng = np.random.Generator(np.random.PCG64(w.params["noise_seed"] + rank))
    return synth.poisson_noise(d_clean, w.params["peak"], rng).astype(np.float32)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP32 pipe peak derived from the unit counts: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def step_flops_per_position(m: int, levels: int) -> float:
    """Algorithmic FLOPs of one position: two 2-D FFTs (5 N log2 N each, N = m^2) plus about
    100 per pixel of pointwise and multigrid work on every level (1 + 1/4 + 1/16 ...)."""
    return 10.0 * m * m * math.log2(m * m) + 100.0 * m * m * sum(4.0 ** -l for l in range(levels))


def recorded_counter(name: str = "dram_bytes_per_launch"):
    """A per-launch figure of the step kernel from the committed ncu summary, if still current.

    The summary carries "kernel_hash: <h>" and "<name>: <n>" lines (DRAM bytes,
    warp-instructions); the figure is dropped (None) once the kernel sources
    have changed since.
    """
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith(("|", "#", " ")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_hash") == kernel_hash():
            return float(fields[name])
    except Exception:
        pass
    return None


def recorded_traffic():
    return recorded_counter("dram_bytes_per_launch")


# Warp-instruction issue peak: 152 SMs x 4 schedulers x 1 instruction per clock x 2.07 GHz
ISSUE_PEAK_GINST = 152 * 4 * 2.07


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(x: float, world: int) -> float:
    """The largest value of x over the ranks of the job (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def init_replicas(world: int, local: int) -> None:
    """One process per GPU; the ranks share nothing but the timing reduction."""
    if world > 1:
        import torch
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ reference arm

def cpu_oracle_sample(w, d, seconds: float):
    """The FP64 oracle (as it stands) on consecutive minibatches of the workload."""
    import oracle as O

    p = w.params
    a = np.sqrt(np.maximum(d.astype(np.float64), 0.0))
    z = np.ones((p["n"], p["n"]), dtype=np.complex128)
    q = O.dp_avg_scale(w.q_init_blurred, d.astype(np.float64))
    order = synth.epoch_orders(len(w.pos), 1, p["order_seed"])[0]
    prm = O.Params(alpha=p["alpha"], levels=p["levels"], minibatch=p["minibatch"], prolong=p["prolong"])
    B = p["minibatch"]
    done, b0 = 0, 0
    t0 = time.perf_counter()
    while b0 < len(order):
        idx = order[b0:b0 + B]
        z, q = O.minibatch_step(z, q, w.pos, a, idx, prm)
        done += len(idx)
        b0 += B
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_oracle_problem(sm, seconds: float):
    """The FP64 oracle (as it stands) on consecutive minibatches of one batch problem."""
    import oracle as O

    a = np.sqrt(np.maximum(sm["d"].astype(np.float64), 0.0))
    z = np.ones((sm["n"], sm["n"]), dtype=np.complex128)
    q = sm["q0"].astype(np.complex128)
    order = O.schedule_permutation(sm["seed"], 0, len(sm["pos"]))
    prm = O.Params(alpha=0.05, levels=sm["levels"], minibatch=sm["B"], prolong="bilinear")
    done, b0 = 0, 0
    t0 = time.perf_counter()
    while b0 < len(order) and time.perf_counter() - t0 < seconds:
        idx = order[b0:b0 + sm["B"]]
        z, q = O.minibatch_step(z, q, sm["pos"], a, idx, prm)
        done += len(idx)
        b0 += sm["B"]
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def _oracle_process(name, path, seconds, barrier, out):
    """One independent oracle process: the bounded sample on intensities read
    from `path`, timed from a barrier shared with the other processes."""
    w = synth.make_workload(name)
    d = np.load(path)
    barrier.wait(timeout=300)
    _, done, dt = cpu_oracle_sample(w, d, seconds)
    out.put((done, dt))


def cpu_oracle_all_cores(w, d, seconds: float):
    """The same sample in one spawned process per host core (the oracle itself is
    single-threaded): positions of all processes / the longest process's time.
    Returns None if a process fails or does not report in time."""
    import multiprocessing as mp
    import queue

    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    res = []
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "d.npy")
        np.save(path, d)
        barrier, out = ctx.Barrier(procs), ctx.Queue()
        workers = [ctx.Process(target=_oracle_process, args=(w.name, path, seconds, barrier, out))
                   for _ in range(procs)]
        for p in workers:
            p.start()
        deadline = time.monotonic() + seconds + 600
        try:
            while len(res) < procs and time.monotonic() < deadline:
                try:
                    res.append(out.get(timeout=5))
                except queue.Empty:
                    if any(p.exitcode not in (None, 0) for p in workers):
                        break
        finally:
            for p in workers:
                if p.is_alive() and len(res) < procs:
                    p.terminate()
                p.join(timeout=60)
    if len(res) < procs:
        return None
    done = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return done / dt, done, dt, procs


def host_intensities(w, rank: int):
    """Noise-free intensities from the library's forward model, Poisson-sampled on the host."""
    import torch

    import paper_2511_01793_gb300 as emg

    p = w.params
    m, N = p["m"], len(w.pos)
    zt = torch.from_numpy(w.z_true.astype(np.complex64)).cuda()
    qt = torch.from_numpy(w.q_true.astype(np.complex64)).cuda()
    pt = torch.from_numpy(w.pos).cuda()
    out = torch.empty((N, m, m), dtype=torch.float32, device="cuda")
    emg.emg_simulate_intensity(zt.data_ptr(), p["n"], p["n"], qt.data_ptr(), m, pt.data_ptr(), N,
                               out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    d_clean = out.cpu().numpy().astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(p["noise_seed"] + rank))
    return synth.poisson_noise(d_clean, p["peak"], rng).astype(np.float32)


def run_reference(args, world, rank):
    if rank != 0:
        return
    w = synth.make_workload(WORKLOAD)
    d = workload_intensities(w, 0)
    per_step = []
    B = w.params["minibatch"]
    for i in range(args.warmup + args.steps):
        rate, done, dt = cpu_oracle_sample(w, d, seconds=0.0)   # exactly one minibatch
        if i >= args.warmup:
            per_step.append((done, dt))
    tot_pos = sum(x[0] for x in per_step)
    tot_t = sum(x[1] for x in per_step)
    value = tot_pos / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one minibatch of {B} positions per step from the initial state"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, world, rank, local):
    import torch

    import paper_2511_01793_gb300 as emg

    torch.cuda.set_device(local)
    init_replicas(world, local)
    emg.build()
    emg.load()
    w = synth.make_workload(WORKLOAD)
    p = w.params
    m, N, B = p["m"], len(w.pos), p["minibatch"]
    d = workload_intensities(w, rank)
    params = emg.emg_default_params(alpha=p["alpha"], levels=p["levels"], minibatch=B,
                                    prolong=emg.EMG_PROLONG_BILINEAR if p["prolong"] == "bilinear"
                                    else emg.EMG_PROLONG_CONST, seed=p["order_seed"] + rank)
    z0 = np.ones((p["n"], p["n"]), dtype=np.complex64)
    q0 = w.q_init_blurred.astype(np.complex64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = emg.Context(w.pos, d, p["n"], p["n"], params, obj=torch.from_numpy(z0),
                          probe=torch.from_numpy(q0), stream=stream)
        emg.emg_normalize_probe(ctx.ctx)
        emg.emg_set_cluster(ctx.ctx, CLUSTER)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

        def barrier():
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()

        for _ in range(args.warmup):
            emg.emg_run_epochs(ctx.ctx, 1)
        emg.emg_profile_read(ctx.ctx)

        def timed_epochs(profiling: bool):
            """K epochs, each timed with CUDA events on the library's stream, L2 flushed before each."""
            emg.emg_set_profiling(ctx.ctx, profiling)
            emg.emg_profile_read(ctx.ctx)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier()
            for i in range(args.steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                emg.emg_run_epochs(ctx.ctx, 1)
                ev[i][1].record(stream)
            barrier()
            pr = emg.emg_profile_read(ctx.ctx)
            emg.emg_set_profiling(ctx.ctx, False)
            return sum(a.elapsed_time(b) for a, b in ev), pr

        # throughput: each epoch replays the captured CUDA graph
        clocks = ClockSampler(local)
        clocks.start()
        total_ms, counts = timed_epochs(False)
        clk = clocks.stop()
        # per-kernel durations: the same K epochs as direct launches bracketed by events
        prof_ms, prof = timed_epochs(True)
        total_ms = max_over_ranks(total_ms, world)
        value = world * N * args.steps / (total_ms / 1e3)
        phi_end = emg.emg_misfit(ctx.ctx)

        # the same epochs with the atomic object scatter (a variant; the default is deterministic)
        pa = emg.emg_default_params(alpha=p["alpha"], levels=p["levels"], minibatch=B,
                                    prolong=emg.EMG_PROLONG_BILINEAR if p["prolong"] == "bilinear"
                                    else emg.EMG_PROLONG_CONST, seed=p["order_seed"] + rank,
                                    scatter=emg.EMG_SCATTER_ATOMIC)
        actx = emg.Context(w.pos, d, p["n"], p["n"], pa, obj=torch.from_numpy(z0), probe=torch.from_numpy(q0),
                           stream=stream)
        emg.emg_normalize_probe(actx.ctx)
        emg.emg_set_cluster(actx.ctx, CLUSTER)
        for _ in range(args.warmup):
            emg.emg_run_epochs(actx.ctx, 1)
        aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        for i in range(args.steps):
            flush.fill_(float(i))
            aev[i][0].record(stream)
            emg.emg_run_epochs(actx.ctx, 1)
            aev[i][1].record(stream)
        barrier()
        atomic_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in aev), world)
        actx.close()

        # end-to-end through the host-buffer entry point (pinned host memory)
        e2e = None
        if not args.no_e2e:
            d_pin = torch.from_numpy(d).pin_memory()
            z_pin = torch.from_numpy(z0.copy()).pin_memory()
            q_pin = torch.empty((m, m), dtype=torch.complex64).pin_memory()
            q_pin.copy_(ctx.probe.cpu())
            dn, zn, qn = d_pin.numpy(), z_pin.numpy(), q_pin.numpy()
            for _ in range(max(1, args.warmup // 2)):
                emg.emg_reconstruct_host(ctx.ctx, dn, zn, qn, 1, running=True)
            t_e2e = 0.0
            for i in range(args.steps):
                flush.fill_(float(i))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                emg.emg_reconstruct_host(ctx.ctx, dn, zn, qn, 1, running=True)
                t_e2e += time.perf_counter() - t0
            t_e2e = max_over_ranks(t_e2e, world)
            e2e = {"value": world * N * args.steps / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": int(d.nbytes + zn.nbytes + qn.nbytes),
                   "d2h_bytes_per_step": int(zn.nbytes + qn.nbytes + 8)}

    # roofline of the dominant kernel (the fused per-position step)
    step_ms, step_launches = prof["step"]
    launches_total = sum(v[1] for v in counts.values())
    alg_bytes_per_pos = 20 * m * m             # patch read 8m^2 + amplitude 4m^2 + patch write 8m^2
    pos_per_launch = N * args.steps / max(step_launches, 1)
    avg_launch_s = step_ms / 1e3 / max(step_launches, 1)
    achieved = alg_bytes_per_pos * pos_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic()       # ncu DRAM bytes of one launch of 64 positions
    if traffic is not None:
        traffic = round(traffic * pos_per_launch / 64)
    kernel_share = {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4) for k, v in prof.items()}
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 5), "peak_source": peak_kind,
                "traffic": traffic, "kernel": f"k_stepc<{m},{CLUSTER}>",
                "algorithmic_bytes_per_launch": int(alg_bytes_per_pos * pos_per_launch),
                "avg_launch_us": round(avg_launch_s * 1e6, 3), "launch_share": kernel_share,
                "timing": "CUDA events around each k_step launch over a second pass of the same "
                          f"{args.steps} epochs (direct launches, {prof_ms / args.steps:.3f} ms/epoch)"}
    flops = step_flops_per_position(m, p["levels"]) * pos_per_launch
    roofline["fp32"] = {"achieved": round(flops / avg_launch_s / 1e12, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                        "unit": "TFLOP/s", "frac": round(flops / avg_launch_s / 1e12 / FP32_PEAK_TFLOPS, 5),
                        "flops_per_launch": int(flops), "peak_source": "derived: 152 SMs x 128 lanes x 2 x 2.07 GHz"}
    inst = recorded_counter("warp_instructions_per_launch")
    if inst is not None:
        # the ncu count is for a launch of 64 positions; scale to this run's average launch
        inst_avg = inst * pos_per_launch / 64
        roofline["issue"] = {"achieved": round(inst_avg / avg_launch_s / 1e9, 2), "peak": round(ISSUE_PEAK_GINST, 2),
                             "unit": "G warp-instructions/s",
                             "frac": round(inst_avg / avg_launch_s / 1e9 / ISSUE_PEAK_GINST, 5),
                             "instructions_per_launch": int(inst_avg),
                             "peak_source": "derived: 152 SMs x 4 schedulers x 2.07 GHz; count from the ncu summary"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(world),
        "e2e": e2e, "gpu_launches": launches_total, "roofline": roofline, "clocks": clk,
        "misfit_end": phi_end,
        "scatter_atomic": {"value": world * N * args.steps / (atomic_ms / 1e3), "ms_per_step": atomic_ms / args.steps,
                           "note": "EMG_SCATTER_ATOMIC (FP32 atomics, not bitwise repeatable); value above is the "
                                   "deterministic default"},
    }
    if world == 1 and not args.no_cpu_baseline:
        rate, done, dt = cpu_oracle_sample(w, d, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{done} positions ({math.ceil(done / B)} minibatches of "
                                          f"{B}) from the initial state, {dt:.1f} s single-thread FP64"}
        par = cpu_oracle_all_cores(w, d, args.cpu_seconds)
        if par is not None:
            rate_all, done_all, dt_all, procs = par
            line["cpu_baseline"]["all_cores"] = {
                "value": rate_all, "unit": UNIT, "cores": procs,
                "sample": f"{procs} independent oracle processes (spawned), each on the sample above; "
                          f"{done_all} positions in {dt_all:.1f} s"}
    ctx.close()
    return line


def run_gpu_grad(args, world, rank, local):
    """One step = Phi and its Wirtinger gradients over all positions (Sec. 2.1)."""
    import torch

    import paper_2511_01793_gb300 as emg

    torch.cuda.set_device(local)
    init_replicas(world, local)
    emg.build()
    emg.load()
    w = synth.make_workload(args.workload)
    p = w.params
    m, N, B = p["m"], len(w.pos), p["minibatch"]
    d = host_intensities(w, rank)
    rng = np.random.default_rng(rank)
    z0 = synth.perturb(w.z_true, 0.2, rng).astype(np.complex64)
    q0 = synth.perturb(w.q_true, 0.2, rng).astype(np.complex64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = emg.Context(w.pos, d, p["n"], p["n"], emg.emg_default_params(alpha=p["alpha"], minibatch=B),
                          stream=stream)
        zd = torch.from_numpy(z0).cuda()
        qd = torch.from_numpy(q0).cuda()
        gz = torch.empty_like(zd)
        gq = torch.empty_like(qd)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

        def step():
            emg.emg_misfit_gradient(ctx.ctx, zd.data_ptr(), qd.data_ptr(), gz.data_ptr(), gq.data_ptr(), False)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        emg.emg_profile_read(ctx.ctx)
        clocks = ClockSampler(local)
        clocks.start()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        counts = emg.emg_profile_read(ctx.ctx)
        total_ms = sum(a.elapsed_time(b) for a, b in ev)
        # gradient-kernel share: time the chunk kernels alone in a second pass
        gms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            emg.emg_misfit_gradient(ctx.ctx, zd.data_ptr(), qd.data_ptr(), 0, 0, False)
            a1.record(stream)
            gms.append((a0, a1))
        torch.cuda.synchronize()
        grad_only_ms = sum(a.elapsed_time(b) for a, b in gms) / args.steps
        # end to end: pinned host state in, gradients and misfit out
        zh = torch.from_numpy(z0).pin_memory()
        qh = torch.from_numpy(q0).pin_memory()
        gzh = torch.empty_like(zh).pin_memory()
        gqh = torch.empty_like(qh).pin_memory()
        t_e2e = 0.0
        for i in range(args.steps + 1):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            zd.copy_(zh, non_blocking=True)
            qd.copy_(qh, non_blocking=True)
            emg.emg_misfit_gradient(ctx.ctx, zd.data_ptr(), qd.data_ptr(), gz.data_ptr(), gq.data_ptr(), True)
            gzh.copy_(gz, non_blocking=True)
            gqh.copy_(gq, non_blocking=True)
            torch.cuda.synchronize()
            if i > 0:
                t_e2e += time.perf_counter() - t0
    total_ms = max_over_ranks(total_ms, world)
    grad_only_ms = max_over_ranks(grad_only_ms, world)
    t_e2e = max_over_ranks(t_e2e, world)
    value = world * N * args.steps / (total_ms / 1e3)
    # the library picks the chunking; each chunk is one k_gradc and one k_grad_reduce launch
    chunks = max(1, round(sum(v[1] for v in counts.values()) / args.steps / 2))
    alg = 28 * m * m          # patch read 8m^2 + amplitude 4m^2 + two gradient patches 16m^2
    achieved = alg * N / (grad_only_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    line = {
        "metric": "scan positions/sec per misfit-gradient evaluation", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: object {p['n']}^2, probe {m}^2, {N} positions in {chunks} launches "
                               "(chunks chosen by the library)",
                   "l2": "flushed (256 MB write) before every timed step"},
        "e2e": {"value": world * N * args.steps / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(z0.nbytes + q0.nbytes),
                "d2h_bytes_per_step": int(z0.nbytes + q0.nbytes + 8)},
        "gpu_launches": sum(v[1] for v in counts.values()),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 5), "peak_source": peak_kind, "traffic": None,
                     "kernel": f"k_gradc<{m}> (+ its sums)",
                     "algorithmic_bytes_per_launch": int(alg * N / chunks),
                     "timing": f"misfit-only gradient kernels {grad_only_ms:.3f} ms per step"},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O

        t0 = time.perf_counter()
        done = 0
        zz, qq = z0.astype(np.complex128), q0.astype(np.complex128)
        a = np.sqrt(np.maximum(d.astype(np.float64), 0.0))
        while done < N and time.perf_counter() - t0 < args.cpu_seconds:
            O.misfit_gradients(qq, zz, w.pos[done:done + 8], a[done:done + 8])
            done += 8
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"gradients of {done} positions, {dt:.1f} s single-thread FP64"}
    ctx.close()
    return line if rank == 0 else None


PREC_WORKLOAD = "prec_n2048_m256"
PREC_TARGET = os.path.join(ROOT, "tests", "golden", f"{PREC_WORKLOAD}_oracle_misfit.txt")


def read_prec_target():
    """The FP64 oracle's misfit after each stored epoch, [(epoch, Phi), ...] (empty if absent)."""
    if not os.path.exists(PREC_TARGET):
        return []
    rows = [ln.split() for ln in open(PREC_TARGET) if ln.strip() and not ln.startswith("#")]
    return [(int(r[0]), float(r[1])) for r in rows]


def run_gpu_prec(args, world, rank, local):
    """The precision workload: the same eMAGPIE epochs with the DFT pair as FP32
    shared-memory FFTs and as BF16-split GEMMs on the tensor cores; throughput
    of both and wall time until each reaches the FP64 oracle's misfit."""
    import torch

    import paper_2511_01793_gb300 as emg

    torch.cuda.set_device(local)
    init_replicas(world, local)
    emg.build()
    emg.load()
    w = synth.make_workload(PREC_WORKLOAD)
    p = w.params
    n, m, N, B = p["n"], p["m"], len(w.pos), p["minibatch"]
    d = host_intensities(w, rank)
    oracle_phi = read_prec_target()
    e_target, phi_target = oracle_phi[-1] if oracle_phi else (None, None)
    max_epochs = 3 * e_target if e_target else 0
    orders = synth.epoch_orders(N, max(max_epochs, args.warmup + args.steps + 2), p["order_seed"])
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        d_dev = torch.from_numpy(d).cuda()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for name, dft in (("fft32", emg.EMG_DFT_FFT32), ("bf16x3", emg.EMG_DFT_BF16X3)):
            params = emg.emg_default_params(alpha=p["alpha"], levels=p["levels"], minibatch=B,
                                            prolong=emg.EMG_PROLONG_BILINEAR, dft=dft)
            ctx = emg.Context(w.pos, d_dev, n, n, params, obj=torch.ones((n, n), dtype=torch.complex64),
                              probe=torch.from_numpy(w.q_init_blurred.astype(np.complex64)), stream=stream)
            emg.emg_normalize_probe(ctx.ctx)
            torch.cuda.synchronize()
            z_init, q_init = ctx.obj.clone(), ctx.probe.clone()
            for e in range(args.warmup):
                emg.emg_run_epochs(ctx.ctx, 1, order=orders[e])
            emg.emg_profile_read(ctx.ctx)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            clocks = ClockSampler(local)
            clocks.start()
            torch.cuda.synchronize()
            for i in range(args.steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                emg.emg_run_epochs(ctx.ctx, 1, order=orders[args.warmup + i])
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
            counts = emg.emg_profile_read(ctx.ctx)
            # per-kind event times over two more epochs of direct launches
            emg.emg_set_profiling(ctx.ctx, True)
            emg.emg_profile_read(ctx.ctx)
            for e in range(2):
                flush.fill_(float(e))
                emg.emg_run_epochs(ctx.ctx, 1, order=orders[e])
            prof = emg.emg_profile_read(ctx.ctx)
            emg.emg_set_profiling(ctx.ctx, False)
            # time to the oracle's misfit, from the initial state, epochs timed alone
            ttt = None
            if max_epochs:
                ctx.obj.copy_(z_init)
                ctx.probe.copy_(q_init)
                emg.emg_set_epoch(ctx.ctx, 0)
                t_ms, phis = 0.0, []
                for e in range(max_epochs):
                    flush.fill_(float(e))
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    emg.emg_run_epochs(ctx.ctx, 1, order=orders[e])
                    a1.record(stream)
                    phi = emg.emg_misfit(ctx.ctx)
                    t_ms += a0.elapsed_time(a1)
                    phis.append(phi)
                    if ttt is None and phi <= phi_target:
                        ttt = {"ms": round(t_ms, 3), "epochs": e + 1, "phi": phi}
                    if ttt is not None and e + 1 >= e_target:
                        break
                if ttt is None:
                    ttt = {"ms": None, "epochs": None}
                # misfit per epoch against the oracle's on the same inputs, schedule and start
                ttt["misfit_vs_oracle"] = [
                    {"epoch": ep, "phi": phis[ep - 1], "oracle": po, "rel": round((phis[ep - 1] - po) / po, 6)}
                    for ep, po in oracle_phi if ep <= len(phis)]
            res[name] = dict(value=world * N * args.steps / (ms / 1e3), ms_per_epoch=ms / args.steps, counts=counts,
                             prof=prof, clocks=clk, ttt=ttt, ctx=ctx)
        # end to end on host buffers through the tensor-core variant
        ctx = res["bf16x3"]["ctx"]
        d_pin = torch.from_numpy(d).pin_memory()
        z_pin = torch.ones((n, n), dtype=torch.complex64).pin_memory()
        q_pin = q_init.cpu().pin_memory()
        dn, zn, qn = d_pin.numpy(), z_pin.numpy(), q_pin.numpy()
        emg.emg_reconstruct_host(ctx.ctx, dn, zn, qn, 1, running=True)
        t_e2e = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            emg.emg_reconstruct_host(ctx.ctx, dn, zn, qn, 1, running=True)
            t_e2e += time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, world)
    tc = res["bf16x3"]
    dft_ms, dft_launches = tc["prof"]["dft"]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    timing = (f"CUDA events around each minibatch's DFT chain over 2 epochs "
              f"({dft_ms / 2:.3f} ms/epoch of {tc['ms_per_epoch']:.3f})")
    if emg.emg_dft_bf16x3_form(m):
        # radix-16 passes: HBM-bound.  Algorithmic bytes per pixel and position:
        # psi (object read 8, split write 8), three split passes (read 8, write 8;
        # the modulus pass also reads a_k, 4), the last pass (read 8, FP32 write 8)
        bytes_mb = B * m * m * (16 + 16 + 20 + 16 + 16)
        achieved = bytes_mb * (N / B) * 2 / (dft_ms / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 5),
                    "peak_source": "measured (copy)" if "hbm_gbs" in peaks else "fallback",
                    "traffic": None, "kernel": "k_tc_rows16 + k_tc_fft16 x4 (radix-16 tensor-core DFT chain)",
                    "bytes_per_minibatch": bytes_mb, "timing": timing}
    else:
        # executed MMA work of the four GEMM passes: 2 (b m) (2m) (2m) flops per pass and product, 3 products
        flops_epoch = 4 * 2 * N * m * (2 * m) * (2 * m) * 3
        achieved = flops_epoch * 2 / (dft_ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        roofline = {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 5),
                    "peak_source": "measured (bf16, sustained)" if peaks else "fallback",
                    "traffic": None, "kernel": "k_tc_dft x4 + k_tc_psi (dense tensor-core DFT chain)",
                    "flops_per_minibatch": 4 * 2 * B * m * (2 * m) * (2 * m) * 3, "timing": timing}
    line = {
        "metric": "scan positions/sec per eMAGPIE epoch (DFT pair on tensor cores, BF16 x3 split)",
        "value": tc["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tc["ms_per_epoch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3/f32", "data": "synthetic",
        "config": {"workload": f"{PREC_WORKLOAD}: object {n}^2, probe {m}^2, {N} positions (64x64 raster, step 28, "
                               f"+-3 px), Poisson peak 1e5, {p['levels']} levels bilinear, minibatch {B}",
                   "l2": "flushed (256 MB write) before every timed epoch; amplitudes 1.07 GB > L2"},
        "fft32": {"value": res["fft32"]["value"], "ms_per_epoch": res["fft32"]["ms_per_epoch"]},
        "time_to_oracle_misfit": {"target": {"epochs": e_target, "phi": phi_target},
                                  "bf16x3": tc["ttt"], "fft32": res["fft32"]["ttt"]},
        "e2e": {"value": world * N * args.steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(dn.nbytes + zn.nbytes +
                                                                                          qn.nbytes),
                "d2h_bytes_per_step": int(zn.nbytes + qn.nbytes + 8)},
        "gpu_launches": sum(v[1] for v in tc["counts"].values()),
        "roofline": roofline,
        "clocks": tc["clocks"],
    }
    if rank != 0:
        for r in res.values():
            r["ctx"].close()
        return None
    if world == 1 and not args.no_cpu_baseline:
        rate, done, dt = cpu_oracle_sample(w, d, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{done} positions from the initial state, {dt:.1f} s single-thread FP64"}
    for r in res.values():
        r["ctx"].close()
    return line


def batch_problems(count: int = 64, seed: int = 1003):
    """64 uneven problems: object side from {256, 512, 768, 1024}, probe side from
    {64, 128, 256} with m <= n/2, 100-2500 positions (raster step m/8, +-2 px
    jitter, capped by the raster that fits), Poisson peak 1e3-1e5 (log-uniform),
    2 or 3 multigrid levels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for i in range(count):
        n = int(rng.choice([256, 512, 768, 1024]))
        m = int(rng.choice([mm for mm in (64, 128, 256) if mm <= n // 2]))
        step = m // 8
        side_fit = (n - m) // step + 1
        side = max(10, min(int(np.sqrt(rng.integers(100, 2501))), side_fit))
        probs.append(dict(n=n, m=m, side=side, step=step, jitter=2, peak=float(10 ** rng.uniform(3, 5)),
                          levels=int(rng.choice([2, 3])), seed=seed * 1000 + i))
    return probs


def run_gpu_batch(args, world, rank, local):
    import torch

    import paper_2511_01793_gb300 as emg

    torch.cuda.set_device(local)
    init_replicas(world, local)
    emg.build()
    emg.load()
    probs = batch_problems()
    stream = torch.cuda.Stream()
    ctxs, total_pos, alg_bytes, tiles, batches = [], 0, 0, {}, {}
    hosts, samples = [], []
    gen = torch.Generator(device="cuda")
    with torch.cuda.stream(stream):
        for pr in probs:
            rng = np.random.Generator(np.random.PCG64(pr["seed"] + rank))
            n, m = pr["n"], pr["m"]
            z_true = synth.make_object(n, n, rng, phi_max=math.pi).astype(np.complex64)
            q_true = synth.make_probe(m, radius=m * 10.0 / 32.0)
            pos = synth.make_scan(n, m, pr["side"], pr["step"], pr["jitter"], rng)
            N = len(pos)
            zt = torch.from_numpy(z_true).cuda()
            qt = torch.from_numpy(q_true.astype(np.complex64)).cuda()
            pt = torch.from_numpy(pos).cuda()
            d = torch.empty((N, m, m), dtype=torch.float32, device="cuda")
            emg.emg_simulate_intensity(zt.data_ptr(), n, n, qt.data_ptr(), m, pt.data_ptr(), N, d.data_ptr(),
                                       stream.cuda_stream)
            gen.manual_seed(pr["seed"] + rank)
            scale = pr["peak"] / float(d.reshape(N, -1).amax(dim=1).mean())
            d = torch.poisson(d * scale, generator=gen) / scale
            params = emg.emg_default_params(alpha=0.05, levels=pr["levels"], minibatch=min(64, N),
                                            prolong=emg.EMG_PROLONG_BILINEAR, seed=pr["seed"])
            ctx = emg.Context(pos, d, n, n, params, obj=torch.ones((n, n), dtype=torch.complex64),
                              probe=torch.from_numpy(synth.blur_probe(q_true, 2.0).astype(np.complex64)),
                              stream=stream)
            emg.emg_normalize_probe(ctx.ctx)
            # B by the largest misfit decrease per second over two trial epochs, then the tiling
            tuned = emg.emg_autotune_search(ctx.ctx, minibatch=sorted({min(b, N) for b in (16, 32, 64)}),
                                            trial_epochs=2, tune_tiling=True, allow_atomic=False)
            tiles[f"m{m}"] = tiles.get(f"m{m}", []) + [tuned["cluster"]]
            batches[f"m{m}"] = batches.get(f"m{m}", []) + [tuned["minibatch"]]
            if not args.no_e2e:
                hosts.append(d.cpu().pin_memory())
            if not samples and rank == 0 and not args.no_cpu_baseline:
                samples.append(dict(pos=pos, d=d.cpu().numpy(), n=n, q0=ctx.probe.cpu().numpy(), levels=pr["levels"],
                                    B=tuned["minibatch"], seed=pr["seed"], m=m))
            del ctx.intensity
            ctxs.append(ctx)
            total_pos += N
            alg_bytes += 20 * m * m * N
        batch = emg.emg_batch_create([c.ctx for c in ctxs])
        for _ in range(args.warmup):
            emg.emg_batch_run_epochs(batch, 1, stream.cuda_stream)
        torch.cuda.synchronize()
        for c in ctxs:
            emg.emg_profile_read(c.ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        clocks.start()
        for i in range(args.steps):
            ev[i][0].record(stream)
            emg.emg_batch_run_epochs(batch, 1, stream.cuda_stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
        launches = sum(sum(v[1] for v in emg.emg_profile_read(c.ctx).values()) for c in ctxs)
        e2e = None
        if hosts:
            # end to end through the public calls: every step uploads every problem's intensities
            # (pinned host memory, read in place by the amplitude kernel) and its state, runs the
            # batch epoch and reads every state back
            z_in = [c.obj.cpu().pin_memory() for c in ctxs]
            q_in = [c.probe.cpu().pin_memory() for c in ctxs]
            z_out = [torch.empty_like(z).pin_memory() for z in z_in]
            q_out = [torch.empty_like(q).pin_memory() for q in q_in]
            t_e2e = 0.0
            for i in range(args.steps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for c, dh, zh, qh in zip(ctxs, hosts, z_in, q_in):
                    emg.emg_set_intensity(c.ctx, dh.data_ptr())
                    c.obj.copy_(zh, non_blocking=True)
                    c.probe.copy_(qh, non_blocking=True)
                emg.emg_batch_run_epochs(batch, 1, stream.cuda_stream)
                for c, zo, qo in zip(ctxs, z_out, q_out):
                    zo.copy_(c.obj, non_blocking=True)
                    qo.copy_(c.probe, non_blocking=True)
                torch.cuda.synchronize()
                if i > 0:      # the first round pays one-time costs
                    t_e2e += time.perf_counter() - t0
            t_e2e = max_over_ranks(t_e2e, world)
            e2e = {"value": world * total_pos * args.steps / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(h.nbytes for h in hosts) + sum(z.nbytes for z in z_in) +
                                             sum(q.nbytes for q in q_in)),
                   "d2h_bytes_per_step": int(sum(z.nbytes for z in z_out) + sum(q.nbytes for q in q_out))}
        emg.emg_batch_destroy(batch)
    value = world * total_pos * args.steps / (total_ms / 1e3)
    achieved = alg_bytes * args.steps / (total_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    line = {
        "metric": "scan positions/sec per epoch over a batch of reconstructions", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch64: {len(probs)} problems, {total_pos} positions per epoch, object "
                               "256-1024, probe 64-256, 2-3 levels, one graph launch per epoch",
                   "l2": f"inputs {alg_bytes / 2.5e9:.1f} GB of amplitudes and patches, larger than L2",
                   "tiling_chosen": {k: sorted(set(v)) for k, v in tiles.items()},
                   "minibatch_chosen": {k: {str(b): v.count(b) for b in sorted(set(v))} for k, v in batches.items()},
                   "autotune": "per problem: B from {16, 32, 64} by misfit decrease per second over two trial "
                               "epochs, then the FFT tiling by epoch time; deterministic scatter"},
        "e2e": e2e, "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 5), "peak_source": peak_kind, "traffic": None,
                     "kernel": "whole epoch graph (algorithmic bytes of all positions / epoch time)"},
        "clocks": clk,
    }
    if samples:
        sm = samples[0]
        rate, done, dt = cpu_oracle_problem(sm, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"problem 0 of the batch (object {sm['n']}^2, probe {sm['m']}^2, "
                                          f"{len(sm['pos'])} positions, B = {sm['B']}): {done} positions from its "
                                          f"initial state, {dt:.1f} s single-thread FP64"}
    for c in ctxs:
        c.close()
    return line if rank == 0 else None


def run_gpu_shard(args, world, rank, local):
    """One reconstruction of the default workload with every minibatch split across the ranks."""
    import torch

    import paper_2511_01793_gb300 as emg
    from paper_2511_01793_gb300.shard import ShardedReconstruction

    torch.cuda.set_device(local)
    init_replicas(world, local)
    emg.build()
    emg.load()
    w = synth.make_workload(WORKLOAD)
    p = w.params
    m, N, B = p["m"], len(w.pos), p["minibatch"]
    d = workload_intensities(w, 0)            # the same data on every rank
    params = emg.emg_default_params(alpha=p["alpha"], levels=p["levels"], minibatch=B,
                                    prolong=emg.EMG_PROLONG_BILINEAR, seed=p["order_seed"])
    stream = torch.cuda.Stream()
    orders = synth.epoch_orders(N, args.warmup + args.steps, p["order_seed"])
    with torch.cuda.stream(stream):
        ctx = emg.Context(w.pos, d, p["n"], p["n"], params, obj=torch.ones((p["n"], p["n"]), dtype=torch.complex64),
                          probe=torch.from_numpy(w.q_init_blurred.astype(np.complex64)), stream=stream)
        emg.emg_normalize_probe(ctx.ctx)
        emg.emg_set_cluster(ctx.ctx, CLUSTER)
        run = ShardedReconstruction(ctx, world, rank)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

        def barrier():
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()

        for e in range(args.warmup):
            run.run_epoch(orders[e])
        emg.emg_profile_read(ctx.ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        clocks.start()
        barrier()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            run.run_epoch(orders[args.warmup + i])
            ev[i][1].record(stream)
        barrier()
        clk = clocks.stop()
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
        launches = sum(v[1] for v in emg.emg_profile_read(ctx.ctx).values())
        phi_end = emg.emg_misfit(ctx.ctx)
    ctx.close()
    if rank != 0:
        return None
    value = N * args.steps / (total_ms / 1e3)       # one reconstruction: the job's positions per second
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(1), parallelism=f"minibatch split over {world} ranks"),
        "e2e": None, "gpu_launches": launches, "roofline": None, "clocks": clk, "misfit_end": phi_end,
        "note": "each minibatch: the ranks step their shares of the slots, one all-gather of the slot results, "
                "the combine on every rank; minibatches run from Python without graph capture",
    }


def compact(line):
    """The figures of a next-row workload that ride along in the default line."""
    if line is None:
        return None
    keep = {k: line.get(k) for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "clocks",
                                     "gpu_launches")}
    keep["workload"] = line["config"]["workload"]
    rf = line.get("roofline") or {}
    keep["roofline"] = {k: rf.get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "kernel")}
    if line.get("e2e"):
        keep["e2e"] = line["e2e"]
    if line.get("cpu_baseline"):
        cb = line["cpu_baseline"]
        keep["cpu_baseline"] = {k: cb.get(k) for k in ("value", "unit", "cores", "kind", "sample")}
    for k in ("fft32", "time_to_oracle_misfit"):
        if k in line:
            keep[k] = line[k]
    return keep


def next_rows(args, world, rank, local):
    """The three next-row workloads, each with a few timed steps, for the default line."""
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = min(args.steps, 5), max(3, min(args.warmup, 3))
    sub.cpu_seconds = min(args.cpu_seconds, 6.0)
    out = {}
    for name, fn in (("grad_n1024_m256", run_gpu_grad), ("batch64", run_gpu_batch),
                     (PREC_WORKLOAD, run_gpu_prec)):
        sub.workload = name
        t0 = time.perf_counter()
        try:
            out[name] = compact(fn(sub, world, rank, local))
        except Exception as exc:  # a failed next row must not cost the main line
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        if out[name] is not None:
            out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def main():
    args = parse_args()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    fn = {"grad_n1024_m256": run_gpu_grad, "batch64": run_gpu_batch, PREC_WORKLOAD: run_gpu_prec}.get(args.workload)
    if args.shard and args.workload == WORKLOAD:
        fn = run_gpu_shard
    if fn is not None:
        line = fn(args, world, rank, local)
    else:
        line = run_gpu(args, world, rank, local)
        if world == 1 and not args.no_next_rows:
            line["next_rows"] = next_rows(args, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
