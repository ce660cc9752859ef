"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a naive DFT,
hand-derived golden values, closed forms, brute-force minimisation, the
paper's propositions (Prop. 3.1, Prop. 3.2, the MAGPIE properties of
Sec. 3.2) and exact invariants (equivariance, fixed point, batch-1
equivalence with the sequential sweep).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


# ---------------------------------------------------------------- Sec. 2.1: F

@pytest.mark.parametrize("m", [2, 4, 8])
def test_dft2_is_the_unnormalised_dft(m):
    rng = np.random.default_rng(m)
    x = _crandn(rng, m, m)
    ref = np.zeros((m, m), dtype=complex)
    for u in range(m):
        for v in range(m):
            s = 0j
            for r in range(m):
                for c in range(m):
                    s += x[r, c] * complex(math.cos(-2 * math.pi * (u * r + v * c) / m),
                                           math.sin(-2 * math.pi * (u * r + v * c) / m))
            ref[u, v] = s
    assert np.max(np.abs(O.dft2(x) - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(O.idft2(O.dft2(x)) - x)) <= 1e-14 * m * m


def test_dft2_golden_delta():
    g = _load("dft_delta_4x4.txt")
    x = np.zeros((4, 4), dtype=complex)
    x[1, 2] = 1.0
    X = O.dft2(x)
    for u, v, re, im in g:
        assert abs(X[int(u), int(v)] - complex(re, im)) < 1e-15


def test_parseval_unnormalised():
    rng = np.random.default_rng(1)
    x = _crandn(rng, 16, 16)
    assert np.isclose(np.sum(np.abs(O.dft2(x)) ** 2), 256 * np.sum(np.abs(x) ** 2), rtol=1e-13)


# ------------------------------------------------- Def. 2.1: revised exit wave

def _random_problem(rng, m):
    Q = _crandn(rng, m, m)
    z = _crandn(rng, m, m)
    a = np.abs(_crandn(rng, m, m)) * m
    return Q, z, a


def test_revised_exit_wave_has_the_data_modulus():
    rng = np.random.default_rng(2)
    Q, z, a = _random_problem(rng, 8)
    R = O.revised_exit_wave(Q, z, a)
    assert np.max(np.abs(np.abs(O.dft2(R)) - a)) < 1e-12 * a.max()


def test_revised_exit_wave_is_the_nearest_feasible_point():
    rng = np.random.default_rng(3)
    Q, z, a = _random_problem(rng, 8)
    psi = Q * z
    R = O.revised_exit_wave(Q, z, a)
    d_best = np.linalg.norm(psi - R)
    for _ in range(300):
        other = O.idft2(a * np.exp(1j * rng.uniform(-np.pi, np.pi, a.shape)))
        assert d_best <= np.linalg.norm(psi - other) + 1e-12


def test_revised_exit_wave_phase_at_zero_is_zero():
    rng = np.random.default_rng(4)
    a = np.abs(_crandn(rng, 4, 4))
    R = O.revised_exit_wave(np.zeros((4, 4), complex), np.ones((4, 4), complex), a)
    assert np.allclose(O.dft2(R), a, atol=1e-14)


def test_misfit_equals_fourier_amplitude_misfit():
    rng = np.random.default_rng(5)
    Q, z, a = _random_problem(rng, 8)
    phi = O.exit_wave_misfit_k(Q, z, a)
    alt = np.sum((np.abs(O.dft2(Q * z)) - a) ** 2) / (2 * 64)
    assert np.isclose(phi, alt, rtol=1e-12)


# ------------------------------------------------------------------ Prop. 3.1

def test_prop31_objective_agreement_and_majorization():
    rng = np.random.default_rng(6)
    Qj, zj, a = _random_problem(rng, 8)
    Rj = O.revised_exit_wave(Qj, zj, a)
    assert np.isclose(O.exit_wave_misfit_k(Qj, zj, a), O.surrogate_k(Qj, zj, Rj), rtol=1e-13)
    for scale in (1e-3, 1e-1, 1.0):
        for _ in range(20):
            Q = Qj + scale * _crandn(rng, 8, 8)
            z = zj + scale * _crandn(rng, 8, 8)
            assert O.exit_wave_misfit_k(Q, z, a) <= O.surrogate_k(Q, z, Rj) * (1 + 1e-12) + 1e-12


def _fd_wirtinger(f, x, h=1e-6):
    """Central-difference d/dRe + i d/dIm of a real function of a complex array."""
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        e = np.zeros_like(x)
        e[idx] = h
        gr = (f(x + e) - f(x - e)) / (2 * h)
        gi = (f(x + 1j * e) - f(x - 1j * e)) / (2 * h)
        g[idx] = gr + 1j * gi
    return g


def test_prop31_first_order_agreement():
    rng = np.random.default_rng(7)
    Q, z, a = _random_problem(rng, 4)
    gz, gq = O.wirtinger_gradients(Q, z, a)
    fz = _fd_wirtinger(lambda zz: O.exit_wave_misfit_k(Q, zz, a), z)
    fq = _fd_wirtinger(lambda qq: O.exit_wave_misfit_k(qq, z, a), Q)
    assert np.max(np.abs(gz - fz)) < 1e-6 * np.max(np.abs(gz))
    assert np.max(np.abs(gq - fq)) < 1e-6 * np.max(np.abs(gq))
    # and the surrogate's gradient at the iterate is the same closed form
    R = O.revised_exit_wave(Q, z, a)
    sz = _fd_wirtinger(lambda zz: O.surrogate_k(Q, zz, R), z)
    assert np.max(np.abs(gz - sz)) < 1e-6 * np.max(np.abs(gz))


# ------------------------------------------ Eq. zplus/qplus proximal minimisers

def test_one_variable_steps_are_the_proximal_minimisers():
    from scipy.optimize import minimize

    rng = np.random.default_rng(8)
    m = 2
    Q, z0, a = _random_problem(rng, m)
    R = O.revised_exit_wave(Q, z0, a)
    u = O.u_probe_reg(Q, 0.3)

    def obj_z(v):
        zz = v[:m * m].reshape(m, m) + 1j * v[m * m:].reshape(m, m)
        return 0.5 * np.sum(np.abs(Q * zz - R) ** 2) + 0.5 * np.sum(u * np.abs(zz - z0) ** 2)

    v0 = np.concatenate([z0.real.ravel(), z0.imag.ravel()])
    res = minimize(obj_z, v0, method="BFGS", options=dict(gtol=1e-12, maxiter=10000))
    z_bf = res.x[:4].reshape(m, m) + 1j * res.x[4:].reshape(m, m)
    assert np.max(np.abs(O.magpie_zplus(Q, z0, R, u, 1) - z_bf)) < 1e-6

    uz = O.u_object_reg(z0)

    def obj_q(v):
        qq = v[:m * m].reshape(m, m) + 1j * v[m * m:].reshape(m, m)
        return 0.5 * np.sum(np.abs(qq * z0 - R) ** 2) + 0.5 * np.sum(uz * np.abs(qq - Q) ** 2)

    v0 = np.concatenate([Q.real.ravel(), Q.imag.ravel()])
    res = minimize(obj_q, v0, method="BFGS", options=dict(gtol=1e-12, maxiter=10000))
    q_bf = res.x[:4].reshape(m, m) + 1j * res.x[4:].reshape(m, m)
    assert np.max(np.abs(O.probe_plus(Q, z0, R) - q_bf)) < 1e-6


# ------------------------------------------------------ Eq. geomean, Prop. 3.2

def test_geometric_mean_golden():
    for xr, xi, pr, pi_, yr, yi in _load("geomean_cases.txt"):
        y = O.geometric_mean_aligned(np.array([complex(xr, xi)]), np.array([complex(pr, pi_)]))
        assert abs(y[0] - complex(yr, yi)) < 1e-15


def test_geometric_mean_properties():
    rng = np.random.default_rng(9)
    x = _crandn(rng, 1000)
    xp = _crandn(rng, 1000)
    y = O.geometric_mean_aligned(x, xp)
    assert np.max(np.abs(y * y - x * xp)) < 1e-14 * np.max(np.abs(x * xp))
    assert np.all(np.real(y * np.conj(x)) >= 0)
    c = rng.uniform(0.5, 2.0, 1000)
    assert np.allclose(O.geometric_mean_aligned(x, c * c * x), c * x, rtol=1e-14)


def test_prop32_golden_pixels():
    rows = _load("prop32_scalar.txt")
    Q = np.array([[2.0 + 0j, 3.0 + 0j]])
    z = np.array([[1.0 + 0j, 2.0 + 0j]])
    R = np.array([[3.0 + 0j, 5.0 + 0j]])
    u = O.u_probe_reg(Q, 0.2)
    uz = O.u_object_reg(z)
    zp = O.magpie_zplus(Q, z, R, u, 1)
    qp = O.probe_plus(Q, z, R)
    zt = O.geometric_mean_aligned(z, zp)
    qt = O.geometric_mean_aligned(Q, qp)
    for i, (q, zz, d, uq, uzz, zplus, qplus, ztil, qtil, res, fac) in enumerate(rows):
        assert abs(u[0, i] - uq) < 1e-15 and abs(uz[0, i] - uzz) < 1e-15
        assert abs(zp[0, i] - zplus) < 1e-15
        assert abs(qp[0, i] - qplus) < 1e-15
        assert abs(zt[0, i] - ztil) < 1e-15
        assert abs(qt[0, i] - qtil) < 1e-15
        assert abs(abs(qt[0, i] * zt[0, i] - d) - res) < 1e-14
        assert res <= fac * abs(q * zz - d) + 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_prop32_per_pixel_descent_bound(seed):
    rng = np.random.default_rng(100 + seed)
    m = 8
    Q, z, a = _random_problem(rng, m)
    st = O.joint_step(Q, z, a, alpha=rng.uniform(0.01, 0.5), levels=1)
    d = st["R"]
    e = np.abs(Q * z - d)
    alpha_r = st["u_Q"] / (np.abs(Q) ** 2 + st["u_Q"])
    beta_r = st["u_z"] / (np.abs(z) ** 2 + st["u_z"])
    lhs = np.abs(st["Q_t"] * st["z_t"] - d)
    assert np.all(lhs <= np.maximum(alpha_r, beta_r) * e + 1e-12 * e.max())
    assert st["surrogate_after"] < st["surrogate_before"]


# ------------------------------------------------------------ Sec. 3.2 MAGPIE

def _as_matrix(fn, n_in):
    cols = []
    for i in range(n_in * n_in):
        e = np.zeros(n_in * n_in)
        e[i] = 1.0
        cols.append(fn(e.reshape(n_in, n_in)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("m", [4, 8])
def test_restriction_prolongation_identities(m):
    Ir = _as_matrix(O.restrict, m)                       # (m/2)^2 x m^2
    Ip = _as_matrix(lambda y: O.prolong(y, "const"), m // 2)   # m^2 x (m/2)^2
    assert np.allclose(Ir @ Ip, np.eye((m // 2) ** 2), atol=0)
    assert np.allclose(Ip, 4 * Ir.T, atol=0)
    Ib = _as_matrix(lambda y: O.prolong(y, "bilinear"), m // 2)
    assert np.allclose(Ib.sum(axis=1), 1.0)              # reproduces constants
    assert np.all(Ib >= 0)


def test_bilinear_prolongation_reproduces_linear_fields_inside():
    n = 8
    i = np.arange(n)
    coarse = 3.0 * i[:, None] - 2.0 * i[None, :] + 1.0
    fine = O.prolong(coarse, "bilinear")
    f = (np.arange(2 * n) + 0.5) / 2 - 0.5                # coarse coordinate of fine centres
    ref = 3.0 * f[:, None] - 2.0 * f[None, :] + 1.0
    assert np.allclose(fine[1:-1, 1:-1], ref[1:-1, 1:-1], atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_mg_weight_bounds(seed):
    rng = np.random.default_rng(200 + seed)
    Q = _crandn(rng, 16, 16) * (rng.uniform(size=(16, 16)) > 0.3)   # exact zeros too
    Wz, WR, WuH = O.mg_weights(Q, "const")
    assert np.max(np.abs(Wz)) <= 4 + 1e-12
    assert np.max(np.abs(WR)) <= 4 + 1e-12
    assert np.max(np.abs(WuH)) <= 1 + 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_mg_consistency_and_descent_direction(seed):
    rng = np.random.default_rng(300 + seed)
    m = 16
    Q, z, a = _random_problem(rng, m)
    R = O.revised_exit_wave(Q, z, a)
    u = O.u_probe_reg(Q, 0.1)
    Wz, WR, WuH = O.mg_weights(Q, "const")
    QH = O.restrict(Q)
    zH = O.restrict(Wz * z)
    RH = O.restrict(WR * R)
    uH = WuH * O.restrict(u)
    fine = O.surrogate_k(Q, z, R)
    coarse = O.surrogate_k(QH, zH, RH)
    assert coarse <= 0.25 * np.max(np.abs(WR)) ** 2 * fine * (1 + 1e-12)
    g_fine = np.conj(Q) * (Q * z - R)
    g_coarse = np.conj(QH) * (QH * zH - RH)
    assert np.linalg.norm(g_coarse) <= 0.5 * np.max(np.abs(WuH)) * np.linalg.norm(g_fine) * (1 + 1e-12)
    zH_hat = O.magpie_zplus(QH, zH, RH, uH, 1)
    direction = O.prolong(zH_hat - zH, "const")
    assert np.real(np.vdot(g_fine, direction)) <= 1e-12 * np.linalg.norm(g_fine) * np.linalg.norm(direction)


@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("kind", ["const", "bilinear"])
def test_flat_probe_gives_exact_division(levels, kind):
    rng = np.random.default_rng(400 + levels)
    m = 16
    c = 1.7 * np.exp(0.4j)
    Q = np.full((m, m), c)
    z = _crandn(rng, m, m)
    R = _crandn(rng, m, m)
    u = O.u_probe_reg(Q, 0.25)
    assert np.all(u == 0)
    assert np.allclose(O.magpie_zplus(Q, z, R, u, levels, kind), R / c, atol=1e-13)


def test_two_level_blockwise_constant_probe_closed_form():
    """Q and u constant on 2x2 blocks: z+ = z + G r + a_r I_H^h(G_b I_h^H r).

    With such a probe W_z = W_R = W_u^H = 1, so the coarse correction is the
    block gain times the block mean of r = R - Q z, and the fine step
    from z' = z + I_H^h c leaves a fraction a_r = u/(u+|Q|^2) of it.
    """
    rng = np.random.default_rng(500)
    m = 8
    qb = _crandn(rng, m // 2, m // 2)
    Q = np.repeat(np.repeat(qb, 2, 0), 2, 1)
    z = _crandn(rng, m, m)
    R = _crandn(rng, m, m)
    u = O.u_probe_reg(Q, 0.3)
    r = R - Q * z
    G = np.conj(Q) / (u + np.abs(Q) ** 2)
    ar = u / (u + np.abs(Q) ** 2)
    expect = np.empty_like(z)
    for bi in range(m // 2):
        for bj in range(m // 2):
            blk = (slice(2 * bi, 2 * bi + 2), slice(2 * bj, 2 * bj + 2))
            gb = G[2 * bi, 2 * bj]
            corr = gb * r[blk].mean()
            expect[blk] = z[blk] + G[blk] * r[blk] + ar[blk] * corr
    assert np.allclose(O.magpie_zplus(Q, z, R, u, 2, "const"), expect, atol=1e-13)


def test_two_level_coarse_step_is_restricted_fine_step_for_blockwise_modulus():
    """|Q| constant on each 2x2 block (phases free): the coarse correction is I_h^H(G r).

    Then W_z = 1, W_R = Q_H conj(Q) / rho^2 and W_u^H = |Q_H|^2 / rho^2, and the
    coarse gain with u_H = W_u^H I_h^H u reduces the coarse step exactly to the
    block average of the fine rPIE step G r, G = conj(Q)/(u + |Q|^2) (Sec. 3.2,
    'automatic regularisation transfer').
    """
    rng = np.random.default_rng(510)
    m = 8
    rho = np.repeat(np.repeat(rng.uniform(0.5, 2.0, (m // 2, m // 2)), 2, 0), 2, 1)
    Q = rho * np.exp(1j * rng.uniform(-np.pi, np.pi, (m, m)))
    z = _crandn(rng, m, m)
    R = _crandn(rng, m, m)
    u = O.u_probe_reg(Q, 0.3)
    G = np.conj(Q) / (u + np.abs(Q) ** 2)
    c = O.restrict(G * (R - Q * z))
    z_prime = z + O.prolong(c, "const")
    expect = z_prime + G * (R - Q * z_prime)
    assert np.allclose(O.magpie_zplus(Q, z, R, u, 2, "const"), expect, atol=1e-13)


def _fraction_blocks(name):
    """[block] headers followed by rows of exact fractions (a hand-derived fixture)."""
    from fractions import Fraction

    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                blocks[cur] = []
            else:
                blocks[cur].append([float(Fraction(t)) for t in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def _bilinear_fixture_inputs():
    Q = np.outer([2.0, 1.0, 1.0, 1.0], [1.0, 1.0, 1.0, 2.0]).astype(complex)
    return Q, np.ones((4, 4), dtype=complex), 2 * Q, np.ones((4, 4))


def test_two_level_bilinear_step_golden():
    """Eq. def_weights and the two-level closed forms with bilinear prolongation, against the
    hand-worked separable 4 x 4 case (a non-flat probe, so the coarse correction matters)."""
    g = _fraction_blocks("magpie_bilinear_m4_l2.txt")
    Q, z, R, u = _bilinear_fixture_inputs()
    Wz, WR, WuH = O.mg_weights(Q, "bilinear")
    assert np.max(np.abs(Wz - g["Wz"])) <= 1e-15
    assert np.max(np.abs(WR - g["WR"])) <= 1e-15
    assert np.max(np.abs(WuH - g["WuH"])) <= 1e-15
    zp = O.magpie_zplus(Q, z, R, u, 2, "bilinear")
    assert np.max(np.abs(zp - g["zplus"])) <= 1e-14
    # the fine step does not erase the coarse correction here: z+ differs from R/Q
    assert np.max(np.abs(zp - R / Q)) > 0.05


def test_two_level_bilinear_golden_catches_constant_weights(monkeypatch):
    """Planted mistake: piecewise-constant S inside the weights while the correction stays
    bilinear.  The hand-worked fixture must reject it."""
    g = _fraction_blocks("magpie_bilinear_m4_l2.txt")
    Q, z, R, u = _bilinear_fixture_inputs()
    import oracle.emagpie as OE

    real = OE.mg_weights
    monkeypatch.setattr(OE, "mg_weights", lambda Q_, kind="const": real(Q_, "const"))
    zp = O.magpie_zplus(Q, z, R, u, 2, "bilinear")
    assert np.max(np.abs(zp - g["zplus"])) > 1e-3


def _overlap_fixture():
    rows = {}
    env = {"sqrt": math.sqrt, "__builtins__": {}}
    with open(os.path.join(GOLDEN, "minibatch_overlap_m2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            mode, what, *vals = [t.strip() for t in line.split("|")]
            rows[(mode, what)] = np.array([eval(v, env) for v in vals])
    z = np.full((2, 4), 0.6 + 0.8j)
    Q = np.array([[2.0, 1.0], [3.0, 1.0]], dtype=complex)
    pos = np.array([[0, 0], [0, 1]], dtype=np.int32)
    a = np.array([[[14.0, 6.0], [2.0, 2.0]], [[21.0, 9.0], [3.0, 3.0]]])
    return rows, z, Q, pos, a


@pytest.mark.parametrize("mode", ["wavg", "sum"])
def test_overlapping_minibatch_combine_golden(mode):
    """The minibatch reading at B = 2 with overlapping patches and a non-flat probe, against
    the hand-worked fixture: weights from the right probe pixel, the w_eps max|Q|^2 floor,
    the shared snapshot, uncovered pixels untouched."""
    rows, z, Q, pos, a = _overlap_fixture()
    p = O.Params(alpha=0.5, levels=1, minibatch=2, combine=mode, w_eps=1.0 / 9.0)
    z_new, Q_new = O.minibatch_step(z, Q, pos, a, [0, 1], p)
    expect = np.stack([rows[(mode, "row0")], rows[(mode, "row1")]]) * z
    assert np.max(np.abs(z_new - expect)) <= 1e-14
    assert np.max(np.abs(Q_new - rows[(mode, "probe")][0] * Q)) <= 1e-14
    # the order of the positions in the minibatch does not matter
    z_rev, Q_rev = O.minibatch_step(z, Q, pos, a, [1, 0], p)
    assert np.max(np.abs(z_rev - expect)) <= 1e-14


def test_overlapping_minibatch_golden_catches_a_dropped_floor():
    """Planted mistake: the weight floor w_eps max|Q|^2 left out.  Only the doubly covered
    pixels move, and the fixture rejects them."""
    rows, z, Q, pos, a = _overlap_fixture()
    p = O.Params(alpha=0.5, levels=1, minibatch=2, combine="wavg", w_eps=0.0)
    z_new, _ = O.minibatch_step(z, Q, pos, a, [0, 1], p)
    expect = np.stack([rows[("wavg", "row0")], rows[("wavg", "row1")]]) * z
    assert abs(z_new[0, 1] - expect[0, 1]) > 1e-3 and abs(z_new[1, 1] - expect[1, 1]) > 1e-3
    others = np.ones((2, 4), dtype=bool)
    others[:, 1] = False
    assert np.max(np.abs(z_new[others] - expect[others])) <= 1e-14


def test_overlapping_minibatch_golden_catches_a_transposed_weight():
    """Planted mistake: the combine weight read from the transposed probe pixel, in a copy of
    the oracle's source.  The asymmetric probe of the fixture makes the doubly covered pixels
    move."""
    import sys
    import types

    import oracle.emagpie as OE

    src = open(OE.__file__).read()
    right = 'num[obj] += w[pat] * st["z_t"][pat]\n        den[obj] += w[pat]'
    wrong = 'num[obj] += w.T[pat] * st["z_t"][pat]\n        den[obj] += w.T[pat]'
    assert src.count(right) == 1
    mutant = types.ModuleType("oracle_mutant_wT")
    sys.modules[mutant.__name__] = mutant
    try:
        exec(compile(src.replace(right, wrong), "oracle_mutant_wT", "exec"), mutant.__dict__)
        rows, z, Q, pos, a = _overlap_fixture()
        p = mutant.Params(alpha=0.5, levels=1, minibatch=2, combine="wavg", w_eps=1.0 / 9.0)
        z_new, _ = mutant.minibatch_step(z, Q, pos, a, [0, 1], p)
    finally:
        del sys.modules[mutant.__name__]
    expect = np.stack([rows[("wavg", "row0")], rows[("wavg", "row1")]]) * z
    assert np.max(np.abs(z_new - expect)) > 1e-3


# ------------------------------------------------- whole-step invariants

def _tiny_workload(levels, m=16, n=40, side=4, step=6):
    rng = np.random.default_rng(600 + levels)
    z_true = synth.make_object(n, n, rng, phi_max=1.0, sigma=2.0)
    Q_true = synth.make_probe(m, radius=m / 4)
    pos = synth.make_scan(n, m, side, step, 1, rng)
    d = O.forward_intensity(Q_true, z_true, pos)
    return z_true, Q_true, pos, np.sqrt(d)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_truth_is_a_fixed_point_with_zero_misfit(levels):
    z_true, Q_true, pos, a = _tiny_workload(levels)
    assert O.misfit(Q_true, z_true, pos, a) <= 1e-24 * np.sum(a ** 2)
    p = O.Params(alpha=0.05, levels=levels, minibatch=5)
    z1, Q1 = O.minibatch_step(z_true, Q_true, pos, a, list(range(5)), p)
    assert np.max(np.abs(z1 - z_true)) < 1e-12
    assert np.max(np.abs(Q1 - Q_true)) < 1e-12


@pytest.mark.parametrize("levels,kind", [(1, "const"), (2, "const"), (3, "bilinear")])
def test_scale_equivariance_of_the_minibatch_step(levels, kind):
    z_true, Q_true, pos, a = _tiny_workload(levels)
    rng = np.random.default_rng(700)
    z = synth.perturb(z_true, 0.3, rng)
    Q = synth.perturb(Q_true, 0.3, rng)
    c = 0.7 * np.exp(1.1j)
    p = O.Params(alpha=0.05, levels=levels, minibatch=6, prolong=kind)
    idx = [3, 0, 7, 12, 5, 9]
    z1, Q1 = O.minibatch_step(z, Q, pos, a, idx, p)
    z2, Q2 = O.minibatch_step(z / c, c * Q, pos, a, idx, p)
    assert np.max(np.abs(z2 - z1 / c)) < 1e-12 * np.max(np.abs(z1))
    assert np.max(np.abs(Q2 - c * Q1)) < 1e-12 * np.max(np.abs(Q1))


@pytest.mark.parametrize("levels", [1, 2])
def test_batch_one_equals_the_papers_sequential_sweep(levels):
    z_true, Q_true, pos, a = _tiny_workload(levels)
    rng = np.random.default_rng(800)
    z = np.ones_like(z_true)
    Q = synth.blur_probe(Q_true, 2.0)
    order = rng.permutation(len(pos))
    p = O.Params(alpha=0.05, levels=levels, minibatch=1)
    z_mb, Q_mb, _ = O.run_epochs(z, Q, pos, a, [order], p, eval_misfit=False)
    z_sq, Q_sq = O.sequential_sweep(z, Q, pos, a, order, p)
    assert np.max(np.abs(z_mb - z_sq)) < 1e-13 * np.max(np.abs(z_sq))
    assert np.max(np.abs(Q_mb - Q_sq)) < 1e-13 * np.max(np.abs(Q_sq))


def test_sum_combine_equals_weighted_mean_without_overlap():
    z_true, Q_true, pos, a = _tiny_workload(1, m=16, n=64, side=4, step=16)
    rng = np.random.default_rng(900)
    z = synth.perturb(z_true, 0.2, rng)
    Q = synth.perturb(Q_true, 0.2, rng)
    idx = [0, 2, 8, 10]          # patches 16 px apart on a 16 px probe: disjoint
    pw = O.Params(alpha=0.05, minibatch=4, combine="wavg")
    ps = O.Params(alpha=0.05, minibatch=4, combine="sum")
    zw, _ = O.minibatch_step(z, Q, pos, a, idx, pw)
    zs, _ = O.minibatch_step(z, Q, pos, a, idx, ps)
    assert np.max(np.abs(zw - zs)) < 1e-13


def test_weighted_combine_follows_the_illumination():
    """Where one patch's probe is dark and the other's bright, the bright one wins."""
    rng = np.random.default_rng(950)
    m, n = 16, 40
    Q = synth.perturb(np.ones((m, m), complex), 0.2, rng)
    Q[:, : m // 2] = 0.0                       # left half of the probe is dark
    z = synth.perturb(np.ones((n, n), complex), 0.3, rng)
    pos = np.array([[10, 10], [10, 18]], dtype=np.int32)   # B is 8 px right of A
    a = np.abs(_crandn(rng, 2, m, m)) * m
    p = O.Params(alpha=0.05, minibatch=2)
    z1, _ = O.minibatch_step(z, Q, pos, a, [0, 1], p)
    zB, _ = O.minibatch_step(z, Q, pos, a, [1], p)
    # object columns 18..25: patch A sees probe columns 8..15 (bright), patch B 0..7 (dark)
    zA, _ = O.minibatch_step(z, Q, pos, a, [0], p)
    region = (slice(10, 26), slice(18, 26))
    assert np.max(np.abs(z1[region] - zA[region])) < 1e-5 * np.max(np.abs(zA[region]))
    # object columns 26..33 are covered by B only (its bright half)
    region = (slice(10, 26), slice(26, 34))
    assert np.max(np.abs(z1[region] - zB[region])) < 1e-13


def test_dp_avg_restores_the_exit_wave_norm():
    """With |z| = 1 and every patch inside the object, dp_avg = ||Q*||_2 (Sec. 4.1, unnormalised F)."""
    rng = np.random.default_rng(1000)
    m, n = 16, 48
    Q_true = synth.make_probe(m, radius=4.0) * 3.0
    z = np.exp(1j * rng.uniform(-1, 1, (n, n)))
    pos = synth.make_scan(n, m, 4, 8, 0, rng)
    d = O.forward_intensity(Q_true, z, pos)
    Q0 = O.dp_avg_scale(synth.blur_probe(Q_true, 2.0), d)
    assert np.isclose(np.linalg.norm(Q0), np.linalg.norm(Q_true), rtol=1e-12)


def test_misfit_decreases_on_noise_free_data():
    z_true, Q_true, pos, a = _tiny_workload(1)
    z = np.ones_like(z_true)
    Q = O.dp_avg_scale(synth.blur_probe(Q_true, 2.0), a ** 2)
    orders = synth.epoch_orders(len(pos), 5, 3)
    p = O.Params(alpha=0.01, levels=1, minibatch=4)
    phi0 = O.misfit(Q, z, pos, a)
    _, _, hist = O.run_epochs(z, Q, pos, a, orders, p)
    assert hist[-1]["misfit"] < 0.5 * phi0


# ------------------------------------------------------------------ schedule

def test_splitmix64_reference_outputs():
    # Published reference outputs of SplitMix64 (Steele, Lea, Flood 2014;
    # the splitmix64.c reference generator) for seed 1234567.
    g = O.splitmix64_stream(1234567)
    assert [next(g) for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_schedule_is_a_permutation():
    for e in range(3):
        p = O.schedule_permutation(42, e, 97)
        assert sorted(p) == list(range(97))
    assert O.schedule_permutation(42, 0, 97) != O.schedule_permutation(42, 1, 97)


def test_fifty_epoch_trajectory_is_sensitive_at_rounding_level():
    """Why the 50-epoch GPU/oracle bound is taken from an oracle ensemble.

    Two FP64 oracle runs of the small configuration whose initial object
    differs by 1e-7 relative end more than 1e-3 apart in misfit: a fixed 1e-3
    agreement after 50 epochs is out of reach for any FP32 implementation.
    """
    w = synth.make_workload("parity_n128_m32")
    pr = w.params
    d = O.forward_intensity(w.q_true, w.z_true, w.pos)
    a = np.sqrt(d)
    q0 = O.dp_avg_scale(w.q_init_blurred, d)
    z0 = np.ones((pr["n"], pr["n"]), complex)
    orders = synth.epoch_orders(len(w.pos), pr["epochs"], pr["order_seed"])
    p = O.Params(alpha=pr["alpha"], levels=1, minibatch=pr["minibatch"])
    _, _, h1 = O.run_epochs(z0, q0, w.pos, a, orders, p)
    rng = np.random.default_rng(0)
    zp = z0 * (1 + 1e-7 * (rng.standard_normal(z0.shape) + 1j * rng.standard_normal(z0.shape)))
    _, _, h2 = O.run_epochs(zp, q0, w.pos, a, orders, p)
    m1 = np.array([h["misfit"] for h in h1])
    m2 = np.array([h["misfit"] for h in h2])
    assert np.max(np.abs(m2 - m1) / m1) > 1e-3
    assert m1[-1] < 1e-2 * m1[0] * 10   # while the run itself converges


def test_whole_object_gradient_matches_central_differences():
    """The summed gradients of Phi over all positions (Sec. 2.1) against FD."""
    z_true, Q_true, pos, a = _tiny_workload(1, m=8, n=20, side=3, step=4)
    rng = np.random.default_rng(1100)
    z = synth.perturb(z_true, 0.3, rng)
    Q = synth.perturb(Q_true, 0.3, rng)
    phi, gz, gq = O.misfit_gradients(Q, z, pos, a)
    assert np.isclose(phi, O.misfit(Q, z, pos, a), rtol=1e-13)
    fz = _fd_wirtinger(lambda zz: O.misfit(Q, zz, pos, a), z, h=1e-6)
    fq = _fd_wirtinger(lambda qq: O.misfit(qq, z, pos, a), Q, h=1e-6)
    assert np.max(np.abs(gz - fz)) < 1e-5 * np.max(np.abs(gz))
    assert np.max(np.abs(gq - fq)) < 1e-5 * np.max(np.abs(gq))


# ---------------------------------------------------------------------------
# Stopping criterion and noise-floor rule (Sec. 4.1, Sec. 4.3), hand-worked sequences

def test_stopping_rule_never_fires_on_a_strictly_decreasing_residual():
    r = [1.0 / t for t in range(1, 200)]
    assert O.stopping_epoch(r, 5, 10) == 0


def test_stopping_rule_on_a_constant_residual_fires_after_patience_checks():
    # t = 5 sets the first average (no earlier best); t = 6 .. 15 are ten checks without improvement
    assert O.stopping_epoch([1.0] * 40, 5, 10) == 15
    assert O.stopping_epoch([1.0] * 40, 3, 4) == 7


def test_stopping_rule_counts_from_the_last_improvement():
    # averages: t=5: 3, t=6: 2.2, t=7: 1.6, t=8: 1.2, t=9: 1.0, then 1.0 from t = 10 on
    r = [5, 4, 3, 2, 1] + [1] * 30
    assert O.stopping_epoch(r, 5, 10) == 19
    # an improvement in between restarts the count
    r2 = [5, 4, 3, 2, 1] + [1] * 6 + [0.5] + [0.5] * 30
    # t=12 average 0.9 < 1.0 resets; averages fall to 0.5 at t=16, then ten flat checks end at t=26
    assert O.stopping_epoch(r2, 5, 10) == 26


def test_noise_floor_rule_stops_at_the_first_residual_below_nine_tenths_of_the_floor():
    r = [10.0, 5.0, 3.0, 2.5, 2.0]
    assert O.stopping_epoch(r, 5, 10, floor=3.0) == 4     # 2.5 < 2.7
    assert O.stopping_epoch(r, 5, 10, floor=2.0) == 0     # never below 1.8
    assert O.stopping_epoch(r, 5, 10, floor=20.0) == 1    # 10 < 18 already
