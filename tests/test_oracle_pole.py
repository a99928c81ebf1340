"""Pins of the oracle's across-pole option (Sec. 4.2 boundaries: the theta-difference next to
a pole taken across it, the ghost beyond the pole being the cell at phi + pi of the same
row) against what the mathematics fixes:

* the assembled operator is the Hessian of the discrete energy, entry by entry, by brute
  force polarisation of the energy evaluated from its face definition;
* symmetric, zero row sums (conservation); unlike the mirror-ghost operator it is not
  positive semi-definite to rounding: the energy gains cross terms through the pole whose
  matching normal term (across a pole face of zero area) is absent, which leaves one or two
  slightly negative eigenvalues, shrinking as the theta grid is refined;
* for bhat = phi-hat the cross terms with theta vanish, so the option changes nothing;
* consistency through the pole: for bhat = x-hat, uniform kappa and u = x (Cartesian),
  div(kappa bhat bhat . grad u) = 0; the mirror ghost leaves an O(1) residual in the pole
  rows that does not shrink under refinement, the across-pole ghost (a true centred
  difference along the meridian continued through the pole) converges;
* PCG, RKL2 and Gershgorin see the antipodal couplings: BE equals a dense solve, the
  Gershgorin bound equals the dense row sums, RKL2 conserves sum W u.
"""
import numpy as np
import pytest

import oracle as O
from paper_1610_01265_gb300 import synth


def tiny(seed=3, dims=(3, 4, 6)):
    nr, nth, nph = dims
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    return g, c


def test_pole_hessian_is_the_energy_by_polarisation():
    g, c = tiny()
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], across_pole=True)
    D = O.dense(g, S)
    N = g.N
    E = lambda u: O.energy_conduction(g, c["T"], c["bhat"], c["n"], u.reshape(g.shape), across_pole=True)  # noqa: E731
    e = np.eye(N)
    q = np.array([E(e[i]) for i in range(N)])
    H = np.empty((N, N))
    for i in range(N):
        H[i, i] = 2.0 * q[i]
        for j in range(i + 1, N):
            H[i, j] = H[j, i] = E(e[i] + e[j]) - q[i] - q[j]
    scale = np.abs(D).max()
    assert np.abs(H - D).max() <= 1e-12 * scale
    # the antipodal couplings are really there (and differ from the mirror operator)
    Sm, _ = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    assert np.abs(S[:, 19:]).max() > 1e-3 * scale
    assert np.abs(O.dense(g, Sm) - D).max() > 1e-3 * scale


def _scaled_eigs(g, S, W):
    D = O.dense(g, S)
    d = 1.0 / np.sqrt(W)
    return np.linalg.eigvalsh(d[:, None] * (0.5 * (D + D.T)) * d[None, :])


def test_pole_operator_symmetric_conservative():
    g, c = tiny(seed=5, dims=(4, 6, 8))
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], across_pole=True)
    D = O.dense(g, S)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() <= 1e-14 * scale
    assert np.abs(D.sum(axis=1)).max() <= 1e-13 * scale


def test_pole_operator_spectrum():
    """The mirror operator is PSD to rounding; the across-pole one has at most two negative
    eigenvalues (of W^-1/2 S W^-1/2), small and shrinking under theta refinement."""
    ratios = []
    for dims in ((4, 6, 8), (8, 8, 16), (8, 16, 32)):
        g, c = tiny(seed=5 if dims[1] == 6 else 1, dims=dims)
        Sm, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True)
        lm = _scaled_eigs(g, Sm, W)
        assert lm.min() >= -1e-13 * lm.max()
        S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True, across_pole=True)
        lam = _scaled_eigs(g, S, W)
        assert (lam < -1e-12 * lam.max()).sum() <= 2
        ratios.append(-lam.min() / lam.max())
    assert ratios[0] < 1e-4 and ratios[1] < ratios[0] and ratios[2] < ratios[1]
    # antipodal entries only in the pole rows
    rows = np.nonzero(np.abs(S[:, 19:]).max(axis=1))[0]
    j = (rows // g.nr) % g.nth
    assert set(j.tolist()) <= {0, g.nth - 1}


def test_pole_option_changes_nothing_for_azimuthal_field():
    g, c = tiny(seed=2, dims=(4, 6, 8))
    b = np.zeros_like(c["bhat"])
    b[2] = 1.0  # bhat = phi-hat: no cross term with theta
    S0, _ = O.assemble_conduction(g, c["T"], b, c["n"])
    S1, _ = O.assemble_conduction(g, c["T"], b, c["n"], across_pole=True)
    assert np.array_equal(S0, S1)


def _x_case(nth, nr=6):
    nph = 2 * nth
    rf = np.linspace(1.0, 1.5, nr + 1)
    g = O.Grid(rf, nth, nph)
    rc = 0.5 * (rf[1:] + rf[:-1])
    th = (np.arange(nth) + 0.5) * np.pi / nth
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    P, Th, R = np.meshgrid(ph, th, rc, indexing="ij")
    bx = np.stack([np.sin(Th) * np.cos(P), np.cos(Th) * np.cos(P), -np.sin(P)])  # x-hat in (r, t, p)
    T = np.full(R.shape, 1e6)
    n = np.full(R.shape, 1e8)
    u = R * np.sin(Th) * np.cos(P)  # the Cartesian coordinate x
    return g, T, bx, n, u


def _pole_row_residual(nth, across):
    g, T, b, n, u = _x_case(nth)
    S, W = O.assemble_conduction(g, T, b, n, across_pole=across)
    F = O.apply_F(g, S, W, u)
    scale = -O.apply_F(g, np.abs(S), W, np.abs(u))
    rel = np.abs(F) / scale
    return max(rel[:, 0, 1:-1].max(), rel[:, -1, 1:-1].max())


def test_pole_consistency_through_the_pole():
    mirror = [_pole_row_residual(n, False) for n in (16, 32, 64)]
    across = [_pole_row_residual(n, True) for n in (16, 32, 64)]
    assert min(mirror) > 2e-2  # the mirror ghost is inconsistent at the pole
    assert across[0] / across[1] > 3.0 and across[1] / across[2] > 3.0  # ~ second order
    assert across[2] < 1e-3


def test_pole_solvers_see_the_antipodal_couplings():
    g, c = tiny(seed=7, dims=(4, 6, 8))
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], across_pole=True)
    D = O.dense(g, S)
    dte, lam = O.gershgorin_dt(g, S, W)
    assert lam == pytest.approx((np.abs(D).sum(axis=1) / W).max(), rel=1e-14)
    dt = 30 * dte
    x, it, rel, st = O.be_pcg(g, S, W, c["T"], dt, pc=O.PC_JACOBI, rtol=1e-14, maxit=5000)
    assert st == 0
    xd = np.linalg.solve(np.diag(W) + dt * D, W * c["T"].ravel())
    assert np.linalg.norm(x.ravel() - xd) <= 1e-11 * np.linalg.norm(xd)
    s = O.rkl2_stages(dt / dte)
    y = O.rkl2_superstep(g, S, W, c["T"], dt, s)
    assert abs(np.sum(W * y.ravel()) - np.sum(W * c["T"].ravel())) <= 1e-13 * np.sum(W * c["T"].ravel())


def test_pole_option_needs_an_antipodal_cell():
    for dims in ((3, 4, 7), (3, 1, 8), (3, 4, 4)):
        g, c = tiny(dims=dims)
        with pytest.raises(ValueError):
            O.assemble_conduction(g, c["T"], c["bhat"], c["n"], across_pole=True)
