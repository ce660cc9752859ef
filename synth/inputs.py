"""Seeded generators for the synthetic ptychography workloads.

Every generator takes an explicit ``numpy.random.Generator`` (PCG64) or a seed,
so a workload is a pure function of its configuration.

Recipe (shared by every workload):

* Object (n_rows x n_cols complex): amplitude i.i.d. U[amp_lo, amp_hi]; phase a
  white N(0, 1) field smoothed by a periodic Gaussian filter (sigma px, applied
  as a multiply in the Fourier domain), then affinely mapped so that its
  minimum is -phi_max and its maximum +phi_max.  Stands in for the paper's
  Baboon/Cameraman object (Sec. 4.1).
* Probe (m x m complex): a disk of radius R with a Gaussian edge
  (A = 1 for r <= R, exp(-(r-R)^2 / (2 w^2)) beyond, w = 2 px) and a quadratic
  phase pi (r/R)^2, centred at ((m-1)/2, (m-1)/2).  Stands in for the paper's
  Fresnel zone plate (Sec. 4.1).
* Scan: a side x side raster with step s, centred in the object, plus i.i.d.
  integer jitter U{-J..J} per axis.  Positions are patch top-left corners and
  may leave the object (the selection operator P_k zero-pads, Sec. 2.1).
* Noise: Poisson counting noise at a given peak photon count (Sec. 4.3 uses
  Poisson sampling); the noise percentage follows the definition in Sec. 4.1.
* Initial probe: the true probe blurred by a Gaussian of sigma 2 px applied in
  the Fourier domain (the blur step of the paper's initial-probe recipe,
  Sec. 4.1); the dp_avg normalisation that follows it is part of the method
  and lives with each implementation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------
# Workload definitions
# ---------------------------------------------------------------------------

CONFIGS = {
    # Small parity case: 1 level, noise-free, 75 % overlap (step 8 / m 32).
    # alpha 0.05: with 0.01 the misfit of this probe rises after ~10 epochs even
    # for the batch-1 sweep of the paper, so the run would not converge.
    "parity_n128_m32": dict(
        n=128, m=32, side=10, step=8, jitter=1, radius=10.0, phi_max=math.pi / 2,
        peak=None, alpha=0.05, minibatch=10, levels=1, prolong="const",
        epochs=50, seed=1001,
    ),
    # Performance case: 3 levels, bilinear prolongation, Poisson noise.
    "mg_n512_m128": dict(
        n=512, m=128, side=30, step=12, jitter=2, radius=40.0, phi_max=math.pi,
        peak=1e4, alpha=0.05, minibatch=64, levels=3, prolong="bilinear",
        epochs=100, seed=1002,
    ),
    # Precision case: the DFT pair on tensor cores (BF16 split) against FP32 FFTs.
    "prec_n2048_m256": dict(
        n=2048, m=256, side=64, step=28, jitter=3, radius=80.0, phi_max=math.pi,
        peak=1e5, alpha=0.05, minibatch=256, levels=3, prolong="bilinear",
        epochs=6, seed=1005,
    ),
    # Differentiation case: gradient of the exit-wave misfit at full size.
    "grad_n1024_m256": dict(
        n=1024, m=256, side=40, step=20, jitter=2, radius=80.0, phi_max=math.pi,
        peak=1e4, alpha=0.05, minibatch=64, levels=1, prolong="const",
        epochs=1, seed=1004,
    ),
}


@dataclasses.dataclass
class Workload:
    """Arrays of one synthetic reconstruction problem (all numpy, host)."""

    name: str
    z_true: np.ndarray          # complex128 [n, n]
    q_true: np.ndarray          # complex128 [m, m]
    pos: np.ndarray             # int32 [N, 2] (row, col) top-left corners
    q_init_blurred: np.ndarray  # complex128 [m, m], before dp_avg scaling
    params: dict


# ---------------------------------------------------------------------------
# Generators
# ---------------------------------------------------------------------------

def _periodic_gaussian_filter(field: np.ndarray, sigma: float) -> np.ndarray:
    """Circular Gaussian smoothing of a real 2-D field via its DFT."""
    ny, nx = field.shape
    fy = np.fft.fftfreq(ny)[:, None]
    fx = np.fft.fftfreq(nx)[None, :]
    transfer = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (fx ** 2 + fy ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(field) * transfer))


def make_object(n_rows: int, n_cols: int, rng: np.random.Generator,
                phi_max: float, sigma: float = 4.0,
                amp_lo: float = 0.8, amp_hi: float = 1.0) -> np.ndarray:
    amp = rng.uniform(amp_lo, amp_hi, size=(n_rows, n_cols))
    white = rng.standard_normal(size=(n_rows, n_cols))
    smooth = _periodic_gaussian_filter(white, sigma)
    lo, hi = smooth.min(), smooth.max()
    phase = -phi_max + (smooth - lo) * (2.0 * phi_max / (hi - lo))
    return amp * np.exp(1j * phase)


def make_probe(m: int, radius: float, edge: float = 2.0) -> np.ndarray:
    c = (m - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
    r = np.sqrt(xx ** 2 + yy ** 2)
    amp = np.where(r <= radius, 1.0, np.exp(-((r - radius) ** 2) / (2.0 * edge ** 2)))
    phase = math.pi * (r / radius) ** 2
    return amp * np.exp(1j * phase)


def make_scan(n: int, m: int, side: int, step: int, jitter: int,
              rng: np.random.Generator) -> np.ndarray:
    origin = (n - (m + (side - 1) * step)) // 2
    grid = origin + step * np.arange(side)
    rows, cols = np.meshgrid(grid, grid, indexing="ij")
    pos = np.stack([rows.ravel(), cols.ravel()], axis=1).astype(np.int64)
    if jitter > 0:
        pos += rng.integers(-jitter, jitter + 1, size=pos.shape)
    return pos.astype(np.int32)


def blur_probe(q: np.ndarray, sigma: float = 2.0) -> np.ndarray:
    """Complex Gaussian blur (sigma px) of a probe, applied in Fourier space."""
    m0, m1 = q.shape
    fy = np.fft.fftfreq(m0)[:, None]
    fx = np.fft.fftfreq(m1)[None, :]
    transfer = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (fx ** 2 + fy ** 2))
    return np.fft.ifft2(np.fft.fft2(q) * transfer)


def aberrate_probe(q: np.ndarray, rng: np.random.Generator, sigma: float = 2.0, ramp: float = 7.0,
                   defocus: float = 0.6, astigmatism: float = 0.2, noise: float = 0.01) -> np.ndarray:
    """The paper's aberrated initial probe (Sec. 4.1, probe initialisation):
    the magnitude of q blurred in Fourier space (sigma px), times
    exp(i [a_x x + a_y y + defocus (x^2 + y^2) + astigmatism (x^2 - y^2)]),
    plus complex Gaussian noise of `noise` times the largest magnitude.
    x, y run over [-1, 1] across the probe; (a_x, a_y) has a uniformly drawn
    direction and length ramp / 2, so that the linear phase changes by `ramp`
    radians across the field of view along it.
    """
    m0, m1 = q.shape
    amp = np.abs(blur_probe(np.abs(q).astype(np.complex128), sigma))
    y, x = np.meshgrid(np.linspace(-1.0, 1.0, m0), np.linspace(-1.0, 1.0, m1), indexing="ij")
    theta = rng.uniform(0.0, 2.0 * math.pi)
    ax, ay = 0.5 * ramp * math.cos(theta), 0.5 * ramp * math.sin(theta)
    phase = ax * x + ay * y + defocus * (x ** 2 + y ** 2) + astigmatism * (x ** 2 - y ** 2)
    q0 = amp * np.exp(1j * phase)
    scale = noise * float(amp.max()) / math.sqrt(2.0)
    return q0 + scale * (rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape))


def measure_intensities(z_true: np.ndarray, q_true: np.ndarray, pos: np.ndarray,
                        chunk: int = 64) -> np.ndarray:
    """The simulated experiment: noise-free far-field intensities of a known
    object and probe, |FFT2(Q * patch_k(z))|^2 per scan position (patches
    zero-padded outside the object, DC at [0, 0]), float64 [N, m, m].

    This is the measurement being simulated, not part of any reconstruction:
    it produces the data that both implementations are then given.
    """
    m = q_true.shape[0]
    n_rows, n_cols = z_true.shape
    out = np.empty((len(pos), m, m), dtype=np.float64)
    for c0 in range(0, len(pos), chunk):
        block = np.zeros((min(chunk, len(pos) - c0), m, m), dtype=np.complex128)
        for i, (r0, cc0) in enumerate(pos[c0:c0 + chunk]):
            r0, cc0 = int(r0), int(cc0)
            rs, re_ = max(r0, 0), min(r0 + m, n_rows)
            cs, ce = max(cc0, 0), min(cc0 + m, n_cols)
            if re_ > rs and ce > cs:
                block[i, rs - r0:re_ - r0, cs - cc0:ce - cc0] = z_true[rs:re_, cs:ce]
        out[c0:c0 + len(block)] = np.abs(np.fft.fft2(block * q_true[None])) ** 2
    return out


def poisson_noise(d_clean: np.ndarray, peak: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Poisson counts at ``peak`` photons for the mean per-pattern maximum.

    scale = peak / mean_k(max d_k); d = Poisson(scale * d_clean) / scale, so the
    noisy data keep the units of ``d_clean``.
    """
    per_pattern_max = d_clean.reshape(d_clean.shape[0], -1).max(axis=1)
    scale = peak / float(per_pattern_max.mean())
    counts = rng.poisson(np.maximum(d_clean, 0.0) * scale)
    return counts.astype(np.float64) / scale


def noise_percent(d_noisy: np.ndarray, d_clean: np.ndarray) -> float:
    """Noise amplitude percentage of Sec. 4.1: 100 sqrt(sum|n|^2 / sum|d~|^2)."""
    n = d_noisy - d_clean
    return 100.0 * math.sqrt(float(np.sum(n * n)) / float(np.sum(d_clean * d_clean)))


def epoch_orders(n_pos: int, n_epochs: int, seed: int) -> np.ndarray:
    """One random permutation of the scan indices per epoch, int32 [E, N]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.permutation(n_pos) for _ in range(n_epochs)]).astype(np.int32)


def perturb(x: np.ndarray, rel: float, rng: np.random.Generator) -> np.ndarray:
    """x + complex Gaussian noise of rms ``rel`` * rms(x)."""
    scale = rel * math.sqrt(float(np.mean(np.abs(x) ** 2)))
    noise = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
    return x + scale * noise / math.sqrt(2.0)


def make_workload(name: str, n: Optional[int] = None, **override) -> Workload:
    """Object, probe, scan and blurred initial probe of a named configuration.

    Intensities are not produced here: ``measure_intensities`` simulates them
    on request (the tests use the oracle's forward model instead).
    """
    p = dict(CONFIGS[name])
    p.update(override)
    if n is not None:
        p["n"] = n
    rng = np.random.Generator(np.random.PCG64(p["seed"]))
    z_true = make_object(p["n"], p["n"], rng, p["phi_max"])
    q_true = make_probe(p["m"], p["radius"])
    pos = make_scan(p["n"], p["m"], p["side"], p["step"], p["jitter"], rng)
    q0 = blur_probe(q_true, 2.0)
    p["noise_seed"] = p["seed"] + 7
    p["order_seed"] = p["seed"] + 11
    return Workload(name, z_true, q_true, pos, q0, p)
