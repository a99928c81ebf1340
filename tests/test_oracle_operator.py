"""Pins of the oracle's discrete operators against facts fixed outside the oracle.

Each test checks the oracle against mathematics the paper fixes (Sec. 4.1-4.2,
App. B) -- closed forms, invariants, exact integrals, a textbook special case and
second-order convergence to the continuum operator -- chosen so that a dropped
term, a wrong sign, index or area would fail one of them.
"""
import math

import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

R_SUN = 6.96e10
K_B = 1.380649e-16


def case(nr, nth, nph, seed=1):
    import oracle as O

    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    return g, c, S, W


def test_cell_volumes_fill_the_shell(oracle_mod):
    """Sum of cell volumes = (4 pi / 3)(2.5^3 - 1) R_sun^3 exactly (W = V when 3 k n = 1)."""
    O = oracle_mod
    for nr, nth, nph in [(5, 4, 3), (16, 12, 24)]:
        g = O.Grid(synth.r_faces(nr), nth, nph)
        one = np.ones(g.shape)
        _, W = O.assemble_conduction(g, one * 1e6, np.stack([one, 0 * one, 0 * one]), one / (3 * K_B))
        exact = 4.0 * math.pi / 3.0 * (2.5**3 - 1.0) * R_SUN**3
        assert abs(W.sum() - exact) / exact < 1e-13
        _, Wv = O.assemble_viscosity(g, one, one)
        assert abs(Wv.sum() - exact) / exact < 1e-13


@pytest.mark.parametrize("dims", [(4, 6, 8), (6, 5, 7), (5, 4, 3), (1, 3, 4)])
def test_symmetric_zero_rowsum_psd(oracle_mod, dims):
    """K = -S is symmetric, K 1 = 0 (zero-flux r faces) and S is positive semi-definite."""
    O = oracle_mod
    g, c, S, W = case(*dims)
    D = O.dense(g, S)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() <= 1e-15 * scale
    assert np.abs(D.sum(axis=1)).max() <= 1e-14 * scale
    ev = np.linalg.eigvalsh(D)
    assert ev.min() >= -1e-14 * ev.max()


def test_psd_with_random_directions(oracle_mod):
    """The energy form stays positive semi-definite for arbitrary per-cell bhat."""
    O = oracle_mod
    rng = np.random.default_rng(7)
    for nr, nth, nph in [(4, 6, 8), (6, 5, 7)]:
        g = O.Grid(synth.r_faces(nr), nth, nph)
        b = rng.standard_normal((3, nph, nth, nr))
        b /= np.linalg.norm(b, axis=0)
        T = rng.uniform(5e5, 2e6, g.shape)
        n = rng.uniform(1e6, 1e8, g.shape)
        S, _ = O.assemble_conduction(g, T, b, n)
        ev = np.linalg.eigvalsh(O.dense(g, S))
        assert ev.min() >= -1e-14 * ev.max()


def test_energy_matches_hessian(oracle_mod):
    """u^T S u = 2 Q(u) and e_i^T S e_j = Q(e_i + e_j) - Q(e_i) - Q(e_j) (polarisation)."""
    O = oracle_mod
    g, c, S, W = case(4, 5, 6, seed=3)
    D = O.dense(g, S)
    u = synth.random_field(g.shape, 11)
    Q = O.energy_conduction(g, c["T"], c["bhat"], c["n"], u)
    assert abs(u.ravel() @ D @ u.ravel() - 2.0 * Q) <= 1e-12 * abs(2.0 * Q)
    rng = np.random.default_rng(0)
    scale = np.abs(D).max()
    for _ in range(40):
        i, j = rng.integers(0, g.N, 2)
        ei = np.zeros(g.N); ei[i] = 1.0
        ej = np.zeros(g.N); ej[j] = 1.0
        q = lambda v: O.energy_conduction(g, c["T"], c["bhat"], c["n"], v.reshape(g.shape))  # noqa
        pol = q(ei + ej) - q(ei) - q(ej) if i != j else 2.0 * q(ei)
        assert abs(pol - D[i, j]) <= 1e-12 * scale


def test_stencil_width_is_19_points(oracle_mod):
    """Interior rows have exactly p = 19 non-zeros (App. B: p = 19 for conduction)."""
    O = oracle_mod
    g, c, S, W = case(6, 6, 8)
    D = O.dense(g, S)
    nnz = (D != 0).sum(axis=1).reshape(g.shape)
    assert nnz[:, 1:-1, 1:-1].max() == 19
    assert (nnz[:, 1:-1, 1:-1] == 19).mean() > 0.9


def test_conservation_and_symmetry_at_scale(oracle_mod):
    """sum W F(u) = 0 (energy conservation) and <u, S v> = <v, S u> on a 24x32x48 grid."""
    O = oracle_mod
    g, c, S, W = case(24, 32, 48)
    u = synth.random_field(g.shape, 1)
    v = synth.random_field(g.shape, 2)
    Fu = O.apply_F(g, S, W, u)
    Fv = O.apply_F(g, S, W, v)
    wf = np.abs(W * Fu.ravel()).sum()
    assert abs((W * Fu.ravel()).sum()) <= 1e-13 * wf
    a = (u.ravel() * W * Fv.ravel()).sum()
    b = (v.ravel() * W * Fu.ravel()).sum()
    assert abs(a - b) <= 1e-13 * np.abs(u.ravel() * W * Fv.ravel()).sum()


def test_ring_eigenmodes(oracle_mod):
    """bhat = phi-hat, uniform T: cos(m phi) is an exact eigenvector on every (r, theta) ring
    with eigenvalue proportional to 4 sin^2(m dphi / 2) (circulant 3-point ring operator)."""
    O = oracle_mod
    nr, nth, nph = 5, 6, 16
    g = O.Grid(synth.r_faces(nr), nth, nph)
    one = np.ones(g.shape)
    b = np.stack([0 * one, 0 * one, one])
    S, W = O.assemble_conduction(g, 1e6 * one, b, 1e8 * one)
    phi = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    lams = {}
    for m in (1, 3, 5):
        u = np.cos(m * phi)[:, None, None] * one
        F = O.apply_F(g, S, W, u)
        lam = (F / u)[0]
        resid = F - lam[None] * u
        assert np.abs(resid).max() <= 1e-12 * np.abs(F).max()
        lams[m] = lam
    dph = 2 * np.pi / nph
    for m in (3, 5):
        ratio = lams[m] / lams[1]
        expect = math.sin(m * dph / 2) ** 2 / math.sin(dph / 2) ** 2
        assert np.allclose(ratio, expect, rtol=1e-12)
    assert (lams[1] < 0).all()


def _textbook_laplacian(rf, nth, nph, kappa, u):
    """Independent numpy finite-volume div(kappa grad u) on the spherical grid (7 points)."""
    rfc = np.asarray(rf) * R_SUN
    nr = len(rf) - 1
    dt, dp = np.pi / nth, 2 * np.pi / nph
    tf = np.arange(nth + 1) * dt
    tcn = (np.arange(nth) + 0.5) * dt
    rc = 0.5 * (rfc[1:] + rfc[:-1])
    vol = (rfc[1:] ** 3 - rfc[:-1] ** 3)[None, None, :] / 3 * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :, None] * dp
    div = np.zeros_like(u)
    # radial faces
    Ar = rfc[1:-1][None, None, :] ** 2 * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :, None] * dp
    kf = 0.5 * (kappa[:, :, 1:] + kappa[:, :, :-1])
    fl = kf * Ar * (u[:, :, 1:] - u[:, :, :-1]) / (rc[1:] - rc[:-1])[None, None, :]
    div[:, :, :-1] += fl
    div[:, :, 1:] -= fl
    # theta faces
    At = 0.5 * (rfc[1:] ** 2 - rfc[:-1] ** 2)[None, None, :] * np.sin(tf[1:-1])[None, :, None] * dp
    kf = 0.5 * (kappa[:, 1:, :] + kappa[:, :-1, :])
    fl = kf * At * (u[:, 1:, :] - u[:, :-1, :]) / (rc[None, None, :] * dt)
    div[:, :-1, :] += fl
    div[:, 1:, :] -= fl
    # phi faces (periodic)
    Ap = 0.5 * (rfc[1:] ** 2 - rfc[:-1] ** 2)[None, None, :] * dt
    up = np.roll(u, -1, axis=0)
    kf = 0.5 * (kappa + np.roll(kappa, -1, axis=0))
    fl = kf * Ap * (up - u) / (rc[None, None, :] * np.sin(tcn)[None, :, None] * dp)
    div += fl
    div -= np.roll(fl, 1, axis=0)
    return div, vol


def test_isotropic_reduction_is_textbook_laplacian(oracle_mod):
    """With bhat bhat^T replaced by I (test hook) the operator is the textbook 7-point FV
    spherical Laplacian; edge couplings vanish exactly."""
    O = oracle_mod
    nr, nth, nph = 7, 6, 8
    c = synth.conduction_case(nr, nth, nph, seed=2)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], isotropic=True)
    assert np.abs(S[:, 7:]).max() == 0.0
    u = synth.random_field(g.shape, 5)
    kappa = 9e-7 * c["T"] ** 2.5
    div, vol = _textbook_laplacian(c["rf"], nth, nph, kappa, u)
    F = O.apply_F(g, S, W, u)
    expect = div / (3 * K_B * c["n"] * vol)
    assert np.abs(F - expect).max() <= 1e-12 * np.abs(expect).max()


def test_viscosity_constant_coefficients_textbook(oracle_mod):
    """Viscosity with constant mu = nu rho is the textbook 7-point Laplacian, W = rho V."""
    O = oracle_mod
    nr, nth, nph = 6, 5, 8
    g = O.Grid(synth.r_faces(nr), nth, nph)
    rho = np.full(g.shape, 2.0)
    nu = np.full(g.shape, 3.0)
    S, W = O.assemble_viscosity(g, rho, nu)
    D = O.dense(g, S)
    assert np.abs(D - D.T).max() <= 1e-15 * np.abs(D).max()
    u = synth.random_field(g.shape, 9)
    div, vol = _textbook_laplacian(g.rf, nth, nph, rho * nu, u)
    F = O.apply_F(g, S, W, u)
    expect = div / (rho * vol)
    assert np.abs(F - expect).max() <= 1e-12 * np.abs(expect).max()


def test_manufactured_solution_second_order(oracle_mod):
    """F(T) converges at second order to div(kappa0 T^5/2 b b . grad T)/(3 k n) for smooth
    analytic T, b, n (away from the poles and the radial boundaries)."""
    sp = pytest.importorskip("sympy")
    O = oracle_mod
    r, t, p = sp.symbols("r t p", positive=True)
    Tx = 1e6 * (1 + 0.3 * sp.sin(2 * r) * sp.cos(t) + 0.2 * sp.sin(t) ** 2 * sp.cos(p))
    kap = 9e-7 * Tx ** sp.Rational(5, 2)
    b = [1 + 0.2 * sp.cos(p) * sp.sin(t), 0.5 * sp.sin(t) * sp.cos(t) + 0.1 * r, 0.4 * sp.sin(p + r)]
    nx = 1e8 * r**-6
    gT = [sp.diff(Tx, r) / R_SUN, sp.diff(Tx, t) / (r * R_SUN), sp.diff(Tx, p) / (r * R_SUN * sp.sin(t))]
    bdg = sum(b[i] * gT[i] for i in range(3))
    q = [kap * b[i] * bdg for i in range(3)]
    div = (sp.diff(r**2 * q[0], r) / r**2 + sp.diff(sp.sin(t) * q[1], t) / (r * sp.sin(t))
           + sp.diff(q[2], p) / (r * sp.sin(t))) / R_SUN
    Fx = div / (3 * K_B * nx)
    fT, fF, fn = (sp.lambdify((r, t, p), e, "numpy") for e in (Tx, Fx, nx))
    fb = [sp.lambdify((r, t, p), e, "numpy") for e in b]
    errs = []
    for m in (1, 2, 4):
        nr, nth, nph = 8 * m, 8 * m, 16 * m
        rf = synth.r_faces(nr)
        R, Tt, P = np.broadcast_arrays(*synth.sample_points(nr, nth, nph, rf))
        g = O.Grid(rf, nth, nph)
        T = fT(R, Tt, P)
        B = np.stack([np.broadcast_to(f(R, Tt, P), R.shape) for f in fb])
        S, W = O.assemble_conduction(g, T, B, fn(R, Tt, P) * np.ones_like(R))
        F = O.apply_F(g, S, W, T)
        Fe = fF(R, Tt, P)
        mask = (R > 1.3) & (R < 2.2) & (Tt > np.pi / 4) & (Tt < 3 * np.pi / 4)
        errs.append(np.abs(F - Fe)[mask].max() / np.abs(Fe[mask]).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-2
    assert orders.min() > 1.7, (errs, orders)


def test_gershgorin_bounds(oracle_mod):
    """App. B: |lambda|max <= max row sum (so dt_E |lambda|max <= 2) and the bound is within
    sqrt(p) = sqrt(19) of |lambda|max for these symmetric-like operators."""
    O = oracle_mod
    for dims, seed in [((4, 6, 8), 1), ((6, 5, 7), 2), ((5, 8, 6), 3)]:
        g, c, S, W = case(*dims, seed=seed)
        dt, lam_g = O.gershgorin_dt(g, S, W)
        assert dt == pytest.approx(2.0 / lam_g, rel=1e-15)
        M = -O.dense(g, S) / W[:, None]
        lam = np.abs(np.linalg.eigvals(M)).max()
        assert lam <= lam_g * (1 + 1e-12)
        assert lam_g <= math.sqrt(19) * lam
    # viscosity: p = 7 in the Cartesian-component reading
    g = O.Grid(synth.r_faces(6), 5, 8)
    v = synth.viscosity_case(6, 5, 8, seed=1)
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    dt, lam_g = O.gershgorin_dt(g, S, W)
    lam = np.abs(np.linalg.eigvals(-O.dense(g, S) / W[:, None])).max()
    assert lam <= lam_g * (1 + 1e-12) and lam_g <= math.sqrt(7) * lam


def test_beta_tcut_factor(oracle_mod):
    """beta_Tcut flag (Sec. 4.1, the printed factor): cells below 5e5 K have kappa0 T^{5/2}
    multiplied by (T / 5e5)^{5/2}; others are unchanged.  With uniform T and bhat the
    operator is linear in kappa, so the flagged operator at 2e5 K is (0.4)^{5/2} times the
    plain one."""
    O = oracle_mod
    nr, nth, nph = 6, 4, 6
    g = O.Grid(synth.r_faces(nr), nth, nph)
    one = np.ones(g.shape)
    b = np.stack([one, 0 * one, 0 * one])
    S_lo, _ = O.assemble_conduction(g, 2e5 * one, b, one, beta_tcut=True)
    S_lo0, _ = O.assemble_conduction(g, 2e5 * one, b, one)
    assert np.allclose(S_lo, 0.4**2.5 * S_lo0, rtol=1e-14, atol=0)
    S_hi, _ = O.assemble_conduction(g, 8e5 * one, b, one, beta_tcut=True)
    S_hi0, _ = O.assemble_conduction(g, 8e5 * one, b, one)
    assert np.array_equal(S_hi, S_hi0)
