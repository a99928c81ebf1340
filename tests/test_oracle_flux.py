"""Pins of the oracle's flux-form (non-symmetric) conduction operator.

Row c of the flux form is minus the divergence of the face fluxes
A_f (D_f^aa g_f + sum_b D_f^ab ghat_b) through the six faces of c (the "standard" scheme
Sec. 4.2 refers to; Sec. 2.1 uses PCG on such slightly non-symmetric operators).  Facts
fixed outside the oracle: its symmetric part is the Hessian of the discrete energy
(pinned separately in test_oracle_operator.py), it annihilates constants and conserves
sum W u (zero row and column sums), it reduces to the symmetric operator when the
tensor is isotropic, each row depends only on the coefficients of the cell and its six
face neighbours (what makes it a divergence of face fluxes, and what its transpose
lacks), it converges at second order to the continuum operator, and BE + PCG on it
reaches the dense solution."""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

from test_oracle_operator import K_B, R_SUN


def _ops(O, dims, seed=1, **kw):
    c = synth.conduction_case(*dims, seed=seed)
    g = O.Grid(c["rf"], dims[1], dims[2])
    Ss, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], **kw)
    Sf, W2 = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], flux_form=True, **kw)
    assert np.array_equal(W, W2)
    return g, c, Ss, Sf, W


@pytest.mark.parametrize("dims", [(4, 6, 8), (5, 4, 3), (1, 3, 4)])
def test_symmetric_part_is_the_energy_hessian(oracle_mod, dims):
    O = oracle_mod
    g, c, Ss, Sf, W = _ops(O, dims)
    Ds, Df = O.dense(g, Ss), O.dense(g, Sf)
    scale = np.abs(Ds).max()
    assert np.abs(0.5 * (Df + Df.T) - Ds).max() <= 1e-13 * scale
    asym = np.linalg.norm(Df - Df.T) / np.linalg.norm(Df)
    if dims[0] > 1:
        assert 0.01 < asym < 0.5, asym


def test_conservation_and_constants(oracle_mod):
    O = oracle_mod
    g, c, Ss, Sf, W = _ops(O, (6, 5, 7), seed=2)
    D = O.dense(g, Sf)
    scale = np.abs(D).max()
    assert np.abs(D.sum(axis=1)).max() <= 1e-13 * scale * 19  # S 1 = 0
    assert np.abs(D.sum(axis=0)).max() <= 1e-13 * scale * 19  # 1^T S = 0: sum W u conserved


def test_isotropic_tensor_gives_the_symmetric_operator(oracle_mod):
    O = oracle_mod
    g, c, Ss, Sf, W = _ops(O, (5, 6, 8), seed=3, isotropic=True)
    assert np.abs(Sf - Ss).max() <= 1e-14 * np.abs(Ss).max()


def test_rows_depend_only_on_face_neighbours(oracle_mod):
    """Changing bhat at cell x changes row c of the flux form only if x is c or one of its
    six face neighbours; the symmetric form (and the transpose of the flux form) also
    reach the edge neighbours."""
    O = oracle_mod
    dims = (6, 6, 8)
    c = synth.conduction_case(*dims, seed=4)
    g = O.Grid(c["rf"], dims[1], dims[2])
    nr, nth, nph = dims
    k, j, i = 3, 2, 2
    x = (k, j + 1, i + 1)  # an edge neighbour of (k, j, i)
    b2 = c["bhat"].copy()
    b2[:, x[0], x[1], x[2]] = [0.0, 0.6, 0.8]
    row = (k * nth + j) * nr + i
    Sf1, _ = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], flux_form=True)
    Sf2, _ = O.assemble_conduction(g, c["T"], b2, c["n"], flux_form=True)
    Ss1, _ = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    Ss2, _ = O.assemble_conduction(g, c["T"], b2, c["n"])
    assert np.array_equal(Sf1[row], Sf2[row])
    assert not np.array_equal(Ss1[row], Ss2[row])
    # a face neighbour does change the row
    b3 = c["bhat"].copy()
    b3[:, k, j + 1, i] = [0.0, 0.6, 0.8]
    Sf3, _ = O.assemble_conduction(g, c["T"], b3, c["n"], flux_form=True)
    assert not np.array_equal(Sf1[row], Sf3[row])


def test_manufactured_solution_second_order_flux_form(oracle_mod):
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
        S, W = O.assemble_conduction(g, T, B, fn(R, Tt, P) * np.ones_like(R), flux_form=True)
        F = O.apply_F(g, S, W, T)
        Fe = fF(R, Tt, P)
        mask = (R > 1.3) & (R < 2.2) & (Tt > np.pi / 4) & (Tt < 3 * np.pi / 4)
        errs.append(np.abs(F - Fe)[mask].max() / np.abs(Fe[mask]).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-2
    assert orders.min() > 1.7, (errs, orders)


@pytest.mark.parametrize("pc", [1, 2])
def test_be_pcg_on_the_nonsymmetric_system(oracle_mod, pc):
    O = oracle_mod
    dims = (6, 6, 8)
    g, c, Ss, Sf, W = _ops(O, dims, seed=5)
    dte, _ = O.gershgorin_dt(g, Sf, W)
    dt = 50 * dte
    A = np.diag(W) + dt * O.dense(g, Sf)
    x_ref = np.linalg.solve(A, W * c["T"].ravel())
    x, its, rel, st = O.be_pcg(g, Sf, W, c["T"], dt, pc=pc, block=(2, 3, 4), rtol=1e-12, maxit=5000)
    assert st == 0
    assert np.linalg.norm(x.ravel() - x_ref) <= 1e-8 * np.linalg.norm(x_ref - c["T"].ravel())
