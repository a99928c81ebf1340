"""Pins of the oracle's RKL2 super-time-step (Sec. 3, Fig. 2, Eq. 5).

The RKL2 scheme is built so that one super-step multiplies an eigenvector of M with
eigenvalue lam by R_s(lam dt) = a_s + b_s P_s(1 + w1 lam dt) (P_s Legendre,
a_s = 1 - b_s, w1 = 4/(s^2+s-2)); it is second order (R = 1 + z + z^2/2 + O(z^3)),
stable for |z| <= (s^2+s-2)/2 and its mid-spectrum amplification is a_s ~ 1/2
(Sec. 6).  These fix the coefficients (including the M0 weight) independently.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import eval_legendre

from paper_1610_01265_gb300 import synth


def b_exact(j):
    if j <= 2:
        return Fraction(1, 3)
    return Fraction(j * j + j - 2, 2 * j * (j + 1))


def R_closed(s, z):
    w1 = 4.0 / (s * s + s - 2)
    bs = float(b_exact(s))
    return (1 - bs) + bs * eval_legendre(s, 1 + w1 * z)


@pytest.mark.parametrize("ratio,s,s_odd", [(100, 20, 21), (500, 45, 45), (1000, 63, 63), (10000, 200, 201),
                                           (1.0, 2, 3), (0.01, 2, 3)])
def test_stage_count(oracle_mod, ratio, s, s_odd):
    """Eq. 5: smallest s with (s^2 + s - 2)/4 >= dt/dt_E (at least 2), odd when forced."""
    O = oracle_mod
    got = O.rkl2_stages(ratio)
    assert got == s
    assert (got * got + got - 2) / 4 >= ratio
    if got > 2:
        assert ((got - 1) ** 2 + (got - 1) - 2) / 4 < ratio
    assert O.rkl2_stages(ratio, force_odd=True) == s_odd


@pytest.mark.parametrize("s", [2, 3, 5, 20, 63])
def test_coefficients_exact(oracle_mod, s):
    """Coefficient list of Sec. 3 recomputed in exact rational arithmetic."""
    O = oracle_mod
    mu, nu, mut, gt = O.rkl2_coeffs(s)
    w1 = Fraction(4, s * s + s - 2)
    assert mut[1] == pytest.approx(float(w1 / 3), rel=1e-15)
    for j in range(2, s + 1):
        m = Fraction(2 * j - 1, j) * b_exact(j) / b_exact(j - 1)
        n = -Fraction(j - 1, j) * b_exact(j) / b_exact(j - 2)
        assert mu[j] == pytest.approx(float(m), rel=1e-14)
        assert nu[j] == pytest.approx(float(n), rel=1e-14)
        assert mut[j] == pytest.approx(float(w1 * m), rel=1e-14)
        assert gt[j] == pytest.approx(float(-(1 - b_exact(j - 1)) * w1 * m), rel=1e-14)


def stability_fn(O, s, z):
    """Fig. 2 recurrence with the oracle's coefficients applied to the scalar problem
    y' = z y / dt (z an array of samples or a numpy Polynomial in z)."""
    mu, nu, mut, gt = O.rkl2_coeffs(s)
    Y0 = 1.0 + 0.0 * z
    M0 = z
    Ym2, Ym1 = Y0, Y0 + mut[1] * M0
    for j in range(2, s + 1):
        Y = mu[j] * Ym1 + nu[j] * Ym2 + (1 - mu[j] - nu[j]) * Y0 + mut[j] * z * Ym1 + gt[j] * M0
        Ym2, Ym1 = Ym1, Y
    return Ym1


@pytest.mark.parametrize("s", [2, 3, 4, 7, 20, 45])
def test_stability_polynomial(oracle_mod, s):
    O = oracle_mod
    c = stability_fn(O, s, np.polynomial.Polynomial([0.0, 1.0])).coef
    assert c[0] == pytest.approx(1.0, abs=1e-13)
    assert c[1] == pytest.approx(1.0, rel=1e-12)
    assert c[2] == pytest.approx(0.5, rel=1e-11)
    zmax = (s * s + s - 2) / 2.0
    zs = np.linspace(-zmax, 0.0, 4001)
    closed = R_closed(s, zs)
    assert np.abs(stability_fn(O, s, zs) - closed).max() < 1e-11
    assert np.abs(closed).max() <= 1.0 + 1e-12
    bs = float(b_exact(s))
    assert R_closed(s, -zmax) == pytest.approx((1 - bs) + (-1) ** s * bs, abs=1e-12)


def test_mid_spectrum_amplification_near_half(oracle_mod):
    """Sec. 6: with many stages RKL2 damps mid-to-high modes only by about a_s ~ 1/2."""
    for s in (45, 200):
        zmax = (s * s + s - 2) / 2.0
        zs = np.linspace(-0.6 * zmax, -0.4 * zmax, 101)
        R = R_closed(s, zs)
        a_s = 1 - float(b_exact(s))
        assert np.abs(R - a_s).max() < 0.1
        assert abs(a_s - 0.5) < 0.01


def ring_case(O, nph=16):
    nr, nth = 4, 5
    g = O.Grid(synth.r_faces(nr), nth, nph)
    one = np.ones(g.shape)
    S, W = O.assemble_conduction(g, 1e6 * one, np.stack([0 * one, 0 * one, one]), 1e8 * one)
    phi = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    return g, S, W, phi, one


@pytest.mark.parametrize("ratio", [0.7, 10.0, 100.0, 1000.0])
def test_superstep_on_eigenvectors(oracle_mod, ratio):
    """One super-step multiplies each ring eigenmode by R_s(lam dt) exactly."""
    O = oracle_mod
    g, S, W, phi, one = ring_case(O)
    dtE, _ = O.gershgorin_dt(g, S, W)
    dt = ratio * dtE
    s = O.rkl2_stages(ratio)
    for m in (1, 4, 7):
        u = np.cos(m * phi)[:, None, None] * one
        lam = (O.apply_F(g, S, W, u) / u)[0]
        out = O.rkl2_superstep(g, S, W, u, dt, s)
        expect = R_closed(s, lam * dt)[None] * u
        assert np.abs(out - expect).max() <= 1e-12


def test_second_order_local_error(oracle_mod):
    """Local error against exp(lam dt) scales as dt^3: halving dt cuts it by ~8."""
    O = oracle_mod
    g, S, W, phi, one = ring_case(O)
    dtE, _ = O.gershgorin_dt(g, S, W)
    u = np.cos(2 * phi)[:, None, None] * one
    lam = (O.apply_F(g, S, W, u) / u)[0]
    errs = []
    for dt in (0.4 * dtE, 0.2 * dtE, 0.1 * dtE):
        out = O.rkl2_superstep(g, S, W, u, dt, 5)
        errs.append(np.abs(out - np.exp(lam * dt)[None] * u).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, errs


def test_superstep_matches_matrix_exponential(oracle_mod):
    """Full operator (synthetic fields): a small super-step agrees with expm(dt M) u to O(dt^3)."""
    from scipy.linalg import expm

    O = oracle_mod
    c = synth.conduction_case(4, 4, 6, seed=2)
    g = O.Grid(c["rf"], 4, 6)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dtE, _ = O.gershgorin_dt(g, S, W)
    M = -O.dense(g, S) / W[:, None]
    u = c["T"].ravel()
    errs = []
    for dt in (0.02 * dtE, 0.01 * dtE):
        out = O.rkl2_superstep(g, S, W, c["T"], dt, 4).ravel()
        errs.append(np.abs(out - expm(dt * M) @ u).max())
    assert errs[0] / errs[1] > 6.0


def test_superstep_conserves_energy(oracle_mod):
    """sum W u is conserved by every stage (K 1 = 0)."""
    O = oracle_mod
    c = synth.conduction_case(16, 12, 24, seed=1)
    g = O.Grid(c["rf"], 12, 24)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dtE, _ = O.gershgorin_dt(g, S, W)
    out = O.rkl2_superstep(g, S, W, c["T"], 1000 * dtE, O.rkl2_stages(1000))
    e0 = (W * c["T"].ravel()).sum()
    e1 = (W * out.ravel()).sum()
    assert abs(e1 - e0) <= 1e-13 * abs(e0)
    assert np.isfinite(out).all()
    assert out.max() <= c["T"].max() * (1 + 1e-12) and out.min() >= c["T"].min() * (1 - 1e-12)


# ---------------- RKL1 (Sec. 6 remark: extra stages damp the highest mode) ----------------

def rkl1_fn(O, s, z):
    mu, nu, mut = O.rkl1_coeffs(s)
    Ym2 = 1.0 + 0.0 * z
    Ym1 = Ym2 + mut[1] * z
    for j in range(2, s + 1):
        Y = mu[j] * Ym1 + nu[j] * Ym2 + mut[j] * z * Ym1
        Ym2, Ym1 = Ym1, Y
    return Ym1


@pytest.mark.parametrize("s", [1, 2, 3, 8, 25])
def test_rkl1_stability_polynomial(oracle_mod, s):
    """RKL1 is built so that R_s(z) = P_s(1 + w1 z), w1 = 2/(s^2+s): first order, |R| <= 1 on
    [-(s^2+s), 0] and |R| = 1 at its left end (no damping of the highest mode)."""
    O = oracle_mod
    w1 = 2.0 / (s * s + s)
    c = rkl1_fn(O, s, np.polynomial.Polynomial([0.0, 1.0])).coef
    assert c[0] == pytest.approx(1.0, abs=1e-13) and c[1] == pytest.approx(1.0, rel=1e-12)
    zs = np.linspace(-(s * s + s), 0.0, 2001)
    closed = eval_legendre(s, 1 + w1 * zs)
    assert np.abs(rkl1_fn(O, s, zs) - closed).max() < 1e-11
    assert np.abs(closed).max() <= 1 + 1e-12
    assert abs(abs(closed[0]) - 1.0) < 1e-12


def test_rkl1_extra_stages_damp_the_highest_mode(oracle_mod):
    """With one or more stages beyond the minimum, |R| at the largest |z| the step reaches
    drops below one (Sec. 6)."""
    for ratio in (10.0, 100.0, 1000.0):
        s = 1
        while (s * s + s) / 2 < ratio:
            s += 1
        zmax = 2 * ratio  # dt |lambda|max = 2 dt/dt_E
        for extra in (1, 2, 5):
            se = s + extra
            r = abs(eval_legendre(se, 1 - 2 * zmax / (se * se + se)))
            assert r < 1 - 1e-3


@pytest.mark.parametrize("ratio", [3.0, 40.0, 400.0])
def test_rkl1_superstep_on_eigenvectors(oracle_mod, ratio):
    O = oracle_mod
    g, S, W, phi, one = ring_case(O)
    dtE, _ = O.gershgorin_dt(g, S, W)
    s = O.rkl1_stages(ratio)
    assert (s * s + s) / 2 >= ratio and (s == 1 or ((s - 1) ** 2 + s - 1) / 2 < ratio)
    for m in (1, 5):
        u = np.cos(m * phi)[:, None, None] * one
        lam = (O.apply_F(g, S, W, u) / u)[0]
        out = O.rkl1_superstep(g, S, W, u, ratio * dtE, s + 1)
        w1 = 2.0 / ((s + 1) ** 2 + s + 1)
        assert np.abs(out - eval_legendre(s + 1, 1 + w1 * lam * ratio * dtE)[None] * u).max() <= 1e-12


def test_exact_s_step_damps_the_edge_for_odd_s():
    """Sec. 6: choosing s first and dt = dt_E (s^2+s-2)/4 exactly, the RKL2 factor at the
    highest mode is a_s + (-1)^s b_s, which is 2/(s(s+1)) for odd s (near zero); one stage
    more than needed for the same dt leaves it near a_s ~ 1/2 at the edge."""
    for s in (5, 21, 45):
        zedge = -(s * s + s - 2) / 2.0
        assert R_closed(s, zedge) == pytest.approx(2.0 / (s * (s + 1)), rel=1e-10)
        assert R_closed(s + 1, zedge) > 0.3
