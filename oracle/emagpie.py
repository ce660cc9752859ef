"""Plain, slow, FP64 reference of eMAGPIE (arXiv 2511.01793).  TEST INFRASTRUCTURE.

This module is the oracle that the CUDA library is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run it.  It shares no code with the CUDA library.

Every function follows one passage of the paper, in the paper's notation
(object z, probe Q, patch operator P_k, data d_k, revised exit wave R_k,
misfit Phi, surrogate Phi~).  numpy's FFT serves as the 2-D DFT primitive and
numpy's complex ``sqrt`` as the principal square root; everything else is
written out per pixel with no blocking or fusion.  Positions within a
minibatch are processed one at a time, in the given order.

Readings where the paper is silent, ambiguous or deviates (the CUDA library
follows the same readings):

* F is the unnormalised forward 2-D DFT and F^-1 carries 1/m^2 (Sec. 4.1: the
  dp_avg probe scaling equals the exit-wave norm only with this convention).
* theta(0) := 0 at every iteration j (Def. 2.1 footnote); the j >= 1 rule of
  Sec. 3 (reuse the previous iterate's phase at exact zeros) is not applied.
* Restriction I_h^H is the 2x2 block average and the paper's prolongation
  I_H^h = 4 (I_h^H)^T is piecewise-constant copy (Sec. 3.2); a cell-centred
  bilinear prolongation with edge clamp is offered as an option.
* 0/0 := 0 in every weight and step ratio (Sec. 3.2 weights).
* L > 2 levels: each coarse level treats the previous level's restricted
  (Q, z, R, u) as its fine problem (the two-level scheme of Sec. 3.2 applied
  recursively; L = 2 is exactly the paper's pair of levels).
* Minibatch of B positions (the paper's sweep has batch 1, Sec. 4.4): all B
  positions see the same snapshot (z, Q); covered object pixels become the
  weighted mean sum_k w_k z~_k / sum_k w_k with w_k = |Q(p - o_k)|^2 +
  eps max|Q|^2, and the probe becomes the plain mean of Q~_k over positions
  whose patch is not identically zero.  B = 1 is the paper's update.  The
  paper fixes nothing beyond B = 1, so B > 1 with overlapping patches is
  pinned by a case worked by hand from these definitions (two overlapping
  patches, an asymmetric probe, the weight floor active).
* Geometric-mean branch: the principal root, negated when Re(root * conj(x))
  < 0; at exactly 0 the principal root is kept (Eq. geomean allows both).
* A patch with max|z_k|^2 = 0 leaves the probe unchanged and is excluded from
  the probe mean.
* Stopping criterion (Sec. 4.1): as printed, the best average includes the
  current one, so "average >= best" would always hold; the best is read as the
  minimum of the earlier averages.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Params", "select_patch", "dft2", "idft2", "unit_phase", "revised_exit_wave",
    "exit_wave_misfit_k", "misfit", "misfit_per_position", "wirtinger_gradients",
    "surrogate_k", "u_probe_reg", "u_object_reg", "restrict", "prolong",
    "mg_weights", "magpie_zplus", "probe_plus", "geometric_mean_aligned",
    "joint_step", "minibatch_step", "run_epochs", "sequential_sweep",
    "forward_intensity", "dp_avg", "dp_avg_scale", "splitmix64_stream",
    "schedule_permutation", "magnitude_error", "illuminated_region",
    "aligned_errors", "misfit_gradients", "stopping_epoch",
]


@dataclasses.dataclass
class Params:
    """Hyper-parameters of one eMAGPIE run.

    alpha     rPIE object constant (Sec. 4: u_Q = alpha (||Q||_inf^2 - |Q|^2))
    levels    multigrid levels L >= 1 for the object step (Sec. 3.2)
    minibatch positions per minibatch B >= 1
    prolong   'const' (I_H^h = 4 (I_h^H)^T) or 'bilinear'
    combine   'wavg' (weighted mean) or 'sum' (sum of per-position corrections)
    w_eps     floor of the object-combine weight, relative to max|Q|^2
    joint     True: geometric-mean joint step (Eq. geomean); False: take z^+ and
              Q^+ as they are (the simultaneous rPIE update of Sec. 2.2)
    """

    alpha: float = 0.01
    levels: int = 1
    minibatch: int = 1
    prolong: str = "const"
    combine: str = "wavg"
    w_eps: float = 1e-6
    joint: bool = True


# ---------------------------------------------------------------------------
# Sec. 2.1: forward model, revised exit wave, misfit, gradients
# ---------------------------------------------------------------------------

def _patch_slices(shape, pos_k, m):
    """Object-side and patch-side slices of the part of patch k inside the object."""
    n_rows, n_cols = shape
    r0, c0 = int(pos_k[0]), int(pos_k[1])
    rs, re_ = max(r0, 0), min(r0 + m, n_rows)
    cs, ce = max(c0, 0), min(c0 + m, n_cols)
    re_ = max(re_, rs)
    ce = max(ce, cs)
    obj = (slice(rs, re_), slice(cs, ce))
    pat = (slice(rs - r0, re_ - r0), slice(cs - c0, ce - c0))
    return obj, pat


def select_patch(z: np.ndarray, pos_k: Sequence[int], m: int) -> np.ndarray:
    """z_k = P_k z: the m x m patch at top-left (row, col); zero outside z (Sec. 2.1)."""
    out = np.zeros((m, m), dtype=np.complex128)
    obj, pat = _patch_slices(z.shape, pos_k, m)
    out[pat] = z[obj]
    return out


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2-D DFT: (F x)[u, v] = sum x[r, c] e^{-2 pi i (ur + vc)/m}."""
    return np.fft.fft2(x)


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse of ``dft2`` (carries the 1/m^2)."""
    return np.fft.ifft2(X)


def unit_phase(Psi: np.ndarray) -> np.ndarray:
    """exp(i theta(Psi)) elementwise, with theta(0) := 0 (Def. 2.1 footnote)."""
    mag = np.abs(Psi)
    out = np.ones_like(Psi)
    nz = mag > 0
    out[nz] = Psi[nz] / mag[nz]
    return out


def revised_exit_wave(Q: np.ndarray, z_k: np.ndarray, a_k: np.ndarray) -> np.ndarray:
    """R_k(Q, z_k) = F^-1( sqrt(d_k) * exp(i theta(F(Q * z_k))) ), Def. 2.1.

    ``a_k`` is sqrt(max(d_k, 0)).
    """
    Psi = dft2(Q * z_k)
    return idft2(a_k * unit_phase(Psi))


def exit_wave_misfit_k(Q: np.ndarray, z_k: np.ndarray, a_k: np.ndarray) -> float:
    """Phi_k = 1/2 || Q * z_k - R_k(Q, z_k) ||^2, Eq. (exit_misfit)."""
    R = revised_exit_wave(Q, z_k, a_k)
    return 0.5 * float(np.sum(np.abs(Q * z_k - R) ** 2))


def misfit_per_position(Q, z, pos, a) -> np.ndarray:
    m = Q.shape[0]
    return np.array([exit_wave_misfit_k(Q, select_patch(z, pos[k], m), a[k])
                     for k in range(len(pos))])


def misfit(Q, z, pos, a) -> float:
    """Phi(Q, z) = sum_k Phi_k, Eq. (exit_misfit)."""
    return float(np.sum(misfit_per_position(Q, z, pos, a)))


def wirtinger_gradients(Q, z_k, a_k):
    """grad_{z_k} Phi_k = conj(Q) (Q z_k - R_k), grad_Q Phi_k = conj(z_k) (Q z_k - R_k).

    CR-calculus gradients (d/dx + i d/dy) of Sec. 2.1.
    """
    R = revised_exit_wave(Q, z_k, a_k)
    e = Q * z_k - R
    return np.conj(Q) * e, np.conj(z_k) * e


def misfit_gradients(Q, z, pos, a):
    """Phi(Q, z) and its gradients over all positions (Sec. 2.1, Eq. exit_misfit).

    grad_z Phi = sum_k P_k^T [conj(Q) (Q z_k - R_k)] (patch pixels outside the
    object drop out), grad_Q Phi = sum_k conj(z_k) (Q z_k - R_k).
    """
    m = Q.shape[0]
    gz = np.zeros_like(z)
    gq = np.zeros_like(Q)
    phi = 0.0
    for k in range(len(pos)):
        z_k = select_patch(z, pos[k], m)
        phi += exit_wave_misfit_k(Q, z_k, a[k])
        g_zk, g_q = wirtinger_gradients(Q, z_k, a[k])
        obj, pat = _patch_slices(z.shape, pos[k], m)
        gz[obj] += g_zk[pat]
        gq += g_q
    return phi, gz, gq


def forward_intensity(Q, z, pos) -> np.ndarray:
    """Noise-free data d_k = |F(Q * P_k z)|^2 of Sec. 2.1, float64 [N, m, m]."""
    m = Q.shape[0]
    return np.stack([np.abs(dft2(Q * select_patch(z, pos[k], m))) ** 2
                     for k in range(len(pos))])


# ---------------------------------------------------------------------------
# Sec. 3: surrogate, regularisers, one-variable steps, joint step
# ---------------------------------------------------------------------------

def surrogate_k(Q, z_k, R_fixed) -> float:
    """Phi~_k(Q, z_k; j) = 1/2 || Q z_k - R_k(Q^(j), z_k^(j)) ||^2, Eq. (quadratic_surrogate)."""
    return 0.5 * float(np.sum(np.abs(Q * z_k - R_fixed) ** 2))


def u_probe_reg(Q: np.ndarray, alpha: float) -> np.ndarray:
    """u_Q(Q) = alpha (||Q||_inf^2 - |Q|^2), the rPIE object-step weight (Sec. 2.2, Sec. 4)."""
    absQ2 = np.abs(Q) ** 2
    return alpha * (absQ2.max() - absQ2)


def u_object_reg(z_k: np.ndarray) -> np.ndarray:
    """u_z(z_k) = ||z_k||_inf^2 - |z_k|^2, the ePIE probe-step weight (Sec. 4)."""
    absz2 = np.abs(z_k) ** 2
    return absz2.max() - absz2


def _safe_div(num, den):
    """num / den elementwise with 0/0 (den == 0) read as 0."""
    num = np.asarray(num)
    den = np.asarray(den)
    shape = np.broadcast_shapes(num.shape, den.shape)
    out = np.zeros(shape, dtype=np.result_type(num, den, np.float64))
    numb = np.broadcast_to(num, shape)
    denb = np.broadcast_to(den, shape)
    nz = denb != 0
    out[nz] = numb[nz] / denb[nz]
    return out


def restrict(x: np.ndarray) -> np.ndarray:
    """I_h^H: average of each 2x2 block (Sec. 3.2)."""
    return 0.25 * (x[0::2, 0::2] + x[1::2, 0::2] + x[0::2, 1::2] + x[1::2, 1::2])


def _bilinear_1d(y: np.ndarray, axis: int) -> np.ndarray:
    """Cell-centred linear interpolation to twice the size along ``axis``.

    Fine cell 2i takes 3/4 y[i] + 1/4 y[i-1], fine cell 2i+1 takes
    3/4 y[i] + 1/4 y[i+1]; indices beyond the edge are clamped.
    """
    y = np.moveaxis(y, axis, 0)
    n = y.shape[0]
    out = np.empty((2 * n,) + y.shape[1:], dtype=y.dtype)
    for i in range(n):
        lo = y[max(i - 1, 0)]
        hi = y[min(i + 1, n - 1)]
        out[2 * i] = 0.75 * y[i] + 0.25 * lo
        out[2 * i + 1] = 0.75 * y[i] + 0.25 * hi
    return np.moveaxis(out, 0, axis)


def prolong(y: np.ndarray, kind: str = "const") -> np.ndarray:
    """I_H^h.  'const': 4 (I_h^H)^T, i.e. copy each coarse value to its 2x2 block."""
    if kind == "const":
        return np.repeat(np.repeat(y, 2, axis=0), 2, axis=1)
    if kind == "bilinear":
        return _bilinear_1d(_bilinear_1d(y, 0), 1)
    raise ValueError(kind)


def mg_weights(Q: np.ndarray, kind: str = "const"):
    """W_z, W_R, W_u^H of Eq. (def_weights), with 0/0 := 0.

    W_z   = |Q|^2 / (I_H^h I_h^H |Q|^2)
    W_R   = (I_H^h Q_H) * W_z / Q,   Q_H = I_h^H Q
    W_u^H = |Q_H|^2 / (I_h^H |Q|^2)
    """
    absQ2 = np.abs(Q) ** 2
    restricted_absQ2 = restrict(absQ2)
    Wz = _safe_div(absQ2, prolong(restricted_absQ2, kind))
    QH = restrict(Q)
    WR = _safe_div(prolong(QH, kind) * Wz, Q)
    WuH = _safe_div(np.abs(QH) ** 2, restricted_absQ2)
    return Wz, WR, WuH


def magpie_zplus(Q, z_k, R, u, levels: int, kind: str = "const") -> np.ndarray:
    """Object-patch step of MAGPIE (Sec. 3.2), returning z_k^+.

    One level: the proximal minimiser of Eq. (zplus_proximal),
        z^+ = z + conj(Q) / (u + |Q|^2) * (R - Q z).
    Two or more levels: restrict the terms (Eq. downsampled_terms), take the
    coarse closed-form step, prolongate the coarse correction into z', then
    take the fine closed-form step from z' (the three closed forms of
    Sec. 3.2).  The coarse problem is solved by this same function.
    """
    fine_gain = _safe_div(np.conj(Q), u + np.abs(Q) ** 2)
    if levels <= 1:
        return z_k + fine_gain * (R - Q * z_k)
    Wz, WR, WuH = mg_weights(Q, kind)
    QH = restrict(Q)
    zH = restrict(Wz * z_k)
    RH = restrict(WR * R)
    uH = WuH * restrict(u)
    zH_hat = magpie_zplus(QH, zH, RH, uH, levels - 1, kind)
    z_prime = z_k + prolong(zH_hat - zH, kind)
    return z_prime + fine_gain * (R - Q * z_prime)


def probe_plus(Q, z_k, R) -> np.ndarray:
    """Q^+ of Eq. (qplus_proximal) with the ePIE weight u_z (Sec. 4).

    Q^+ = Q + conj(z_k) / (u_z(z_k) + |z_k|^2) * (R - Q z_k).
    """
    u_z = u_object_reg(z_k)
    return Q + _safe_div(np.conj(z_k), u_z + np.abs(z_k) ** 2) * (R - Q * z_k)


def geometric_mean_aligned(x: np.ndarray, x_plus: np.ndarray) -> np.ndarray:
    """x~ with x~^2 = x * x^+ and |arg(x~ conj(x))| <= pi/2, Eq. (geomean)."""
    root = np.sqrt(x * x_plus)
    flip = np.real(root * np.conj(x)) < 0
    root[flip] = -root[flip]
    return root


def joint_step(Q, z_k, a_k, alpha: float, levels: int = 1, kind: str = "const",
               joint: bool = True):
    """One eMAGPIE position update (Sec. 3, Sec. 3.2, Sec. 4).

    Returns a dict with the revised exit wave R, the one-variable minimisers
    z^+ (MAGPIE) and Q^+ (ePIE), the geometric-mean joint step (z~, Q~),
    mu = ||z_k||_inf^2, and the sampled surrogate before and after.
    """
    R = revised_exit_wave(Q, z_k, a_k)
    u = u_probe_reg(Q, alpha)
    z_plus = magpie_zplus(Q, z_k, R, u, levels, kind)
    Q_plus = probe_plus(Q, z_k, R)
    if joint:
        z_t = geometric_mean_aligned(z_k, z_plus)
        Q_t = geometric_mean_aligned(Q, Q_plus)
    else:
        z_t, Q_t = z_plus, Q_plus
    mu = float(np.max(np.abs(z_k) ** 2))
    return dict(R=R, z_plus=z_plus, Q_plus=Q_plus, z_t=z_t, Q_t=Q_t, mu=mu,
                u_Q=u, u_z=u_object_reg(z_k),
                surrogate_before=surrogate_k(Q, z_k, R),
                surrogate_after=surrogate_k(Q_t, z_t, R))


# ---------------------------------------------------------------------------
# Minibatch reading and the stochastic sweep (Sec. 3, footnote on j; Sec. 4.4)
# ---------------------------------------------------------------------------

def minibatch_step(z, Q, pos, a, idx, params: Params, out: Optional[dict] = None):
    """Apply one minibatch of positions ``idx`` to (z, Q); returns (z, Q).

    All positions use the same snapshot (z, Q).  Object pixels covered by the
    minibatch become sum_k w_k z~_k / sum_k w_k (``combine='wavg'``) or
    z + sum_k (z~_k - z_k) (``combine='sum'``); the probe becomes the mean of
    Q~_k (or Q + sum_k (Q~_k - Q)) over positions with mu_k > 0.
    If ``out`` is a dict it receives per-position diagnostics.  B = 1 and
    non-overlapping minibatches are pinned against the paper's sequential
    sweep; B > 1 with overlapping patches against a hand-worked case.
    """
    m = Q.shape[0]
    absQ2 = np.abs(Q) ** 2
    M_Q = float(absQ2.max())
    num = np.zeros_like(z)
    den = np.zeros(z.shape)
    corr = np.zeros_like(z)
    covered = np.zeros(z.shape, dtype=bool)
    q_sum = np.zeros_like(Q)
    q_count = 0
    diag = []
    for k in idx:
        z_k = select_patch(z, pos[k], m)
        st = joint_step(Q, z_k, a[k], params.alpha, params.levels, params.prolong, params.joint)
        diag.append(st)
        w = absQ2 + params.w_eps * M_Q
        obj, pat = _patch_slices(z.shape, pos[k], m)
        num[obj] += w[pat] * st["z_t"][pat]
        den[obj] += w[pat]
        corr[obj] += st["z_t"][pat] - z_k[pat]
        covered[obj] = True
        if st["mu"] > 0:
            if params.combine == "wavg":
                q_sum += st["Q_t"]
            else:
                q_sum += st["Q_t"] - Q
            q_count += 1
    z_new = z.copy()
    if params.combine == "wavg":
        z_new[covered] = num[covered] / den[covered]
        Q_new = q_sum / q_count if q_count > 0 else Q.copy()
    elif params.combine == "sum":
        z_new[covered] = z[covered] + corr[covered]
        Q_new = Q + q_sum
    else:
        raise ValueError(params.combine)
    if out is not None:
        out["positions"] = diag
        out["sampled_misfit"] = float(sum(d["surrogate_before"] for d in diag))
    return z_new, Q_new


def run_epochs(z, Q, pos, a, orders, params: Params, eval_misfit: bool = True):
    """Run one epoch per row of ``orders`` (a permutation of 0..N-1 each).

    Each epoch splits its permutation into consecutive minibatches of
    ``params.minibatch`` positions (the last may be shorter).  Returns
    (z, Q, history) with per-epoch sampled (running) and end-of-epoch misfit.
    """
    N = len(pos)
    B = params.minibatch
    hist = []
    for order in orders:
        running = 0.0
        for b0 in range(0, N, B):
            info = {}
            z, Q = minibatch_step(z, Q, pos, a, order[b0:b0 + B], params, out=info)
            running += info["sampled_misfit"]
        rec = dict(running_misfit=running)
        if eval_misfit:
            rec["misfit"] = misfit(Q, z, pos, a)
        hist.append(rec)
    return z, Q, hist


def sequential_sweep(z, Q, pos, a, order, params: Params):
    """The paper's own sweep (batch 1): for each k in order, z_k <- z~_k, Q <- Q~."""
    m = Q.shape[0]
    z = z.copy()
    Q = Q.copy()
    for k in order:
        z_k = select_patch(z, pos[k], m)
        st = joint_step(Q, z_k, a[k], params.alpha, params.levels, params.prolong, params.joint)
        obj, pat = _patch_slices(z.shape, pos[k], m)
        z[obj] = st["z_t"][pat]
        Q = st["Q_t"]
    return z, Q


# ---------------------------------------------------------------------------
# Sec. 4.1: probe normalisation, metrics
# ---------------------------------------------------------------------------

def dp_avg(d: np.ndarray) -> float:
    """dp_avg = sqrt(sum_ij dbar_ij) / m with dbar the mean pattern (Sec. 4.1)."""
    m = d.shape[-1]
    dbar = np.mean(d, axis=0)
    return float(np.sqrt(np.sum(dbar)) / m)


def dp_avg_scale(Q0: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Q0 <- Q0 * dp_avg / ||Q0||_2 (Sec. 4.1)."""
    return Q0 * (dp_avg(d) / float(np.sqrt(np.sum(np.abs(Q0) ** 2))))


def magnitude_error(z, z_true) -> float:
    """|| |z| - |z*| ||_2, the paper's error metric (Sec. 4.1)."""
    return float(np.sqrt(np.sum((np.abs(z) - np.abs(z_true)) ** 2)))


def illuminated_region(Q_ref, pos, shape, frac: float = 0.1) -> np.ndarray:
    """Pixels whose summed illumination sum_k |Q(p - o_k)|^2 >= frac * max."""
    m = Q_ref.shape[0]
    illum = np.zeros(shape)
    absQ2 = np.abs(Q_ref) ** 2
    for k in range(len(pos)):
        obj, pat = _patch_slices(shape, pos[k], m)
        illum[obj] += absQ2[pat]
    return illum >= frac * illum.max()


def aligned_errors(z, Q, z_ref, Q_ref, region) -> dict:
    """Errors after removing the (c, 1/c) scale/phase ambiguity of blind ptychography.

    c = <z, z_ref>_region / <z, z>_region minimises || c z - z_ref ||; the probe
    is compared as Q / c.  Returns relative object and probe errors and the
    RMS wrapped phase difference over the region.
    """
    zr = z[region]
    zrefr = z_ref[region]
    c = np.vdot(zr, zrefr) / np.vdot(zr, zr)
    obj = float(np.linalg.norm(c * zr - zrefr) / np.linalg.norm(zrefr))
    phase = np.angle(c * zr * np.conj(zrefr))
    prb = float(np.linalg.norm(Q / c - Q_ref) / np.linalg.norm(Q_ref))
    return dict(c=c, object=obj, probe=prb, phase_rms=float(np.sqrt(np.mean(phase ** 2))))


def stopping_epoch(r: Sequence[float], window: int = 5, patience: int = 10, floor: float = 0.0) -> int:
    """The outer iteration (1-based) at which the run of Sec. 4.1 stops, or 0.

    r[t-1] is the residual r_t = Phi(Q^(t), z^(t)) after iteration t.  For
    t >= window the moving average rbar_t = (1/window) sum_{i<window} r_{t-i}
    is formed.  A check at t counts when rbar_t is not below the best of the
    earlier averages; any improvement resets the count.  The run stops at the
    first t at which the count reaches `patience`.  With floor > 0 (the noise
    residual of Sec. 4.3: Phi at the true object and probe on the noisy data),
    it also stops at the first t with r_t < 0.9 floor.
    """
    best = None
    count = 0
    for t in range(1, len(r) + 1):
        if floor > 0.0 and r[t - 1] < 0.9 * floor:
            return t
        if t < window:
            continue
        avg = sum(r[t - 1 - i] for i in range(window)) / window
        if best is not None and avg >= best:
            count += 1
            if count >= patience:
                return t
        else:
            count = 0
            best = avg
    return 0


# ---------------------------------------------------------------------------
# Default schedule: SplitMix64 + Fisher-Yates (used when no order is given)
# ---------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1


def splitmix64_stream(state: int):
    """SplitMix64 (Steele, Lea, Flood 2014): yields successive 64-bit outputs."""
    state &= _MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        x = state
        x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK64
        yield x ^ (x >> 31)


def schedule_permutation(seed: int, epoch: int, n_pos: int) -> List[int]:
    """Permutation of 0..N-1 for one epoch.

    Generator state = seed + epoch * 0x9E3779B97F4A7C15 (mod 2^64); then the
    Fisher-Yates shuffle of the identity, i from N-1 down to 1, swapping
    element i with element (next() mod (i + 1)).
    """
    gen = splitmix64_stream((seed + epoch * 0x9E3779B97F4A7C15) & _MASK64)
    perm = list(range(n_pos))
    for i in range(n_pos - 1, 0, -1):
        j = next(gen) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm
