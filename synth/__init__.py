"""Seeded synthetic inputs for blind ptychography (object, probe, scan, noise).

This module builds the *inputs* of a reconstruction and nothing of the method:
no Fourier projection, no update rule.  Its one use of the FFT simulates the
experiment (the far-field intensities of a known object and probe), so that
two programs can be given identical data.  Both the FP64 oracle
(tests) and the CUDA library (tests, bench) consume what it produces, so the
two implementations always see identical arrays.

The paper's own test images, zone-plate probe and beamline data (Sec. 4.1,
Sec. 4.4) are not available; the recipes below stand in for them with the same
shapes: an n x n complex object with a smooth phase field, an m x m apodised
probe with quadratic phase, a jittered raster scan and optional Poisson noise.
"""
from .inputs import (  # noqa: F401
    CONFIGS,
    Workload,
    make_object,
    make_probe,
    make_scan,
    blur_probe,
    aberrate_probe,
    measure_intensities,
    poisson_noise,
    noise_percent,
    epoch_orders,
    perturb,
    make_workload,
)
