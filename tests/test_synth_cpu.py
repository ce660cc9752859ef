"""The seeded input generators: the aberrated initial probe of Sec. 4.1."""
import math

import numpy as np

import synth


def test_aberrated_probe_has_the_blurred_magnitude_and_the_stated_phase():
    rng = np.random.default_rng(3)
    m = 64
    q = synth.make_probe(m, radius=20.0)
    q0 = synth.aberrate_probe(q, rng, noise=0.0)
    amp = np.abs(synth.blur_probe(np.abs(q).astype(np.complex128), 2.0))
    assert np.allclose(np.abs(q0), amp, rtol=1e-12, atol=1e-12)
    # phase: linear ramp (7 rad across [-1, 1] along a random direction) + 0.6 defocus + 0.2 astigmatism
    y, x = np.meshgrid(np.linspace(-1, 1, m), np.linspace(-1, 1, m), indexing="ij")
    resid = q0 * np.exp(-1j * (0.6 * (x ** 2 + y ** 2) + 0.2 * (x ** 2 - y ** 2))) / amp
    ph = np.angle(resid[amp > 1e-3 * amp.max()])
    gx = np.angle(resid[m // 2, m // 2 + 1] / resid[m // 2, m // 2]) / (2.0 / (m - 1))
    gy = np.angle(resid[m // 2 + 1, m // 2] / resid[m // 2, m // 2]) / (2.0 / (m - 1))
    assert math.isclose(math.hypot(gx, gy), 3.5, rel_tol=1e-9)       # ramp 7 rad across the field
    assert np.all(np.isfinite(ph))


def test_aberrated_probe_noise_is_one_percent_of_the_peak():
    rng = np.random.default_rng(4)
    q = synth.make_probe(128, radius=40.0)
    clean = synth.aberrate_probe(q, np.random.default_rng(9), noise=0.0)
    noisy = synth.aberrate_probe(q, np.random.default_rng(9), noise=0.01)
    d = noisy - clean
    rms = np.sqrt(np.mean(np.abs(d) ** 2))
    assert abs(rms / np.abs(clean).max() - 0.01) < 0.001
