"""Pins of the oracle's backward-Euler + PCG step (Sec. 2, Eqs. 2-4, Fig. 1, App. A).

BE solves (W + dt S) x = W u^n, the W-scaled symmetric form of Eq. 4.  The pins:
a dense direct solve, the closed-form BE factor 1/(1 - lam dt) on eigenmodes, the
defining property of zero-fill ILU ((LU)_ij = A_ij on the pattern), exact LU when
the block pattern is complete or tridiagonal (one PCG iteration), PC2 with one cell
per block being PC1 (Sec. 2.3), and conservation up to the residual.
"""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth


def case(O, nr, nth, nph, seed=1):
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dtE, _ = O.gershgorin_dt(g, S, W)
    return g, c, S, W, dtE


@pytest.mark.parametrize("pc,block", [(1, (1, 1, 1)), (2, (2, 3, 2)), (2, (4, 6, 4))])
@pytest.mark.parametrize("ratio", [1.0, 100.0, 10000.0])
def test_matches_dense_solve(oracle_mod, pc, block, ratio):
    O = oracle_mod
    g, c, S, W, dtE = case(O, 4, 6, 8)
    dt = ratio * dtE
    A = np.diag(W) + dt * O.dense(g, S)
    x_ref = np.linalg.solve(A, W * c["T"].ravel())
    x, it, rel, st = O.be_pcg(g, S, W, c["T"], dt, pc=pc, block=block, rtol=1e-14, maxit=2000)
    assert st == 0
    assert rel <= 1e-14
    assert np.linalg.norm(x.ravel() - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_eigenmode_closed_form(oracle_mod):
    """BE multiplies an eigenmode with eigenvalue lam by 1/(1 - lam dt) (Eq. 3)."""
    O = oracle_mod
    nr, nth, nph = 4, 5, 16
    g = O.Grid(synth.r_faces(nr), nth, nph)
    one = np.ones(g.shape)
    S, W = O.assemble_conduction(g, 1e6 * one, np.stack([0 * one, 0 * one, one]), 1e8 * one)
    dtE, _ = O.gershgorin_dt(g, S, W)
    phi = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    u = np.cos(3 * phi)[:, None, None] * one
    lam = (O.apply_F(g, S, W, u) / u)[0]
    for pc, blk in ((1, (1, 1, 1)), (2, (4, 5, 4))):
        x, it, rel, st = O.be_pcg(g, S, W, u, 500 * dtE, pc=pc, block=blk, rtol=1e-14)
        assert st == 0
        assert np.abs(x - u / (1 - lam * 500 * dtE)[None]).max() <= 1e-12


def test_ilu0_defining_property(oracle_mod):
    """Zero-fill ILU: L unit lower, U upper, (L U)_ij = A_ij for every (i, j) of the block's
    19-point pattern; couplings leaving the block are dropped."""
    O = oracle_mod
    g, c, S, W, dtE = case(O, 4, 6, 6, seed=2)
    blk = (4, 3, 3)
    A19 = O.build_A(S, W, 50 * dtE)
    LU19 = O.bilu0_factor(g, A19, blk)
    off = O.offsets()
    nr, nth, nph = g.nr, g.nth, g.nph

    def local_cells(bi, bj, bk):
        cells = []
        for lk in range(blk[2]):
            for lj in range(blk[1]):
                for li in range(blk[0]):
                    cells.append((bi * blk[0] + li, bj * blk[1] + lj, bk * blk[2] + lk))
        return cells

    for bi, bj, bk in [(0, 0, 0), (0, 1, 1)]:
        cells = local_cells(bi, bj, bk)
        pos = {cl: n for n, cl in enumerate(cells)}
        m = len(cells)
        Ab = np.zeros((m, m))
        LUb = np.zeros((m, m))
        pattern = np.zeros((m, m), dtype=bool)
        for n, (i, j, k) in enumerate(cells):
            cidx = (k * nth + j) * nr + i
            for s in range(19):
                q = (i + off[s, 0], j + off[s, 1], k + off[s, 2])
                if q in pos:
                    Ab[n, pos[q]] = A19[cidx, s]
                    LUb[n, pos[q]] = LU19[cidx, s]
                    pattern[n, pos[q]] = True
        L = np.tril(LUb, -1) + np.eye(m)
        U = np.triu(LUb)
        prod = L @ U
        scale = np.abs(Ab).max()
        assert np.abs((prod - Ab)[pattern]).max() <= 1e-13 * scale
        # symmetric A: U = diag(U) L^T
        assert np.abs(U - np.diag(np.diag(U)) @ (L.T)).max() <= 1e-12 * np.abs(U).max()


def test_complete_pattern_block_is_exact_lu(oracle_mod):
    """A 2 x 2 x 1 block couples all four cells (faces and edges), so ILU0 is exact LU and
    PCG with such blocks on a grid of one block converges in one iteration."""
    O = oracle_mod
    c = synth.conduction_case(2, 2, 3, seed=4)
    g = O.Grid(c["rf"], 2, 3)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dtE, _ = O.gershgorin_dt(g, S, W)
    A19 = O.build_A(S, W, 10 * dtE)
    LU = O.bilu0_factor(g, A19, (2, 2, 1))
    A = np.diag(W) + 10 * dtE * O.dense(g, S)
    r = synth.random_field(g.shape, 3)
    z = O.bilu0_apply(g, LU, (2, 2, 1), r)
    # on each phi-layer the block solve is exact; cross-layer couplings are dropped
    for k in range(3):
        sl = slice(4 * k, 4 * k + 4)
        assert np.allclose(A[sl, sl] @ z.ravel()[sl], r.ravel()[sl], rtol=1e-13, atol=0)


def test_radial_lines_tridiagonal_one_iteration(oracle_mod):
    """bhat = rhat makes every radial line an independent tridiagonal system; blocks of one
    full radial line make ILU0 exact, so PCG converges in one iteration."""
    O = oracle_mod
    nr, nth, nph = 8, 4, 6
    c = synth.conduction_case(nr, nth, nph, seed=1)
    g = O.Grid(c["rf"], nth, nph)
    one = np.ones(g.shape)
    S, W = O.assemble_conduction(g, c["T"], np.stack([one, 0 * one, 0 * one]), c["n"])
    dtE, _ = O.gershgorin_dt(g, S, W)
    x, it, rel, st = O.be_pcg(g, S, W, c["T"], 1000 * dtE, pc=2, block=(nr, 1, 1), rtol=1e-12)
    assert st == 0 and it == 1 and rel <= 1e-13


def test_unit_blocks_equal_jacobi(oracle_mod):
    """Sec. 2.3: PC2 with one cell per block is PC1, iterate for iterate."""
    O = oracle_mod
    g, c, S, W, dtE = case(O, 6, 6, 8)
    for k in (1, 5, 17):
        x1, i1, r1, _ = O.be_pcg(g, S, W, c["T"], 300 * dtE, pc=1, fixed_iters=k)
        x2, i2, r2, _ = O.be_pcg(g, S, W, c["T"], 300 * dtE, pc=2, block=(1, 1, 1), fixed_iters=k)
        assert i1 == i2 == k
        assert np.array_equal(x1, x2) and r1 == r2


def test_conservation_up_to_residual(oracle_mod):
    """1^T S = 0, so sum W x - sum W u^n = 1^T r exactly in exact arithmetic."""
    O = oracle_mod
    g, c, S, W, dtE = case(O, 8, 8, 16)
    u = c["T"]
    for pc in (1, 2):
        x, it, rel, st = O.be_pcg(g, S, W, u, 1000 * dtE, pc=pc, block=(4, 4, 4), rtol=1e-10)
        assert st == 0
        bnorm = np.linalg.norm(W * u.ravel())
        drift = abs((W * x.ravel()).sum() - (W * u.ravel()).sum())
        assert drift <= np.sqrt(g.N) * rel * bnorm * 1.01 + 1e-14 * bnorm


def test_initial_guess_and_zero_iterations(oracle_mod):
    """x0 = exact solution converges with 0 iterations; a given x0 is honoured."""
    O = oracle_mod
    g, c, S, W, dtE = case(O, 4, 6, 8)
    dt = 100 * dtE
    A = np.diag(W) + dt * O.dense(g, S)
    xs = np.linalg.solve(A, W * c["T"].ravel())
    x, it, rel, st = O.be_pcg(g, S, W, c["T"], dt, rtol=1e-10, x0=xs.reshape(g.shape))
    assert st == 0 and it == 0
    x, it, rel, st = O.be_pcg(g, S, W, c["T"], dt, rtol=1e-10, maxit=3)
    assert st == 1 and it == 3


def test_breakdown_detected(oracle_mod):
    """An indefinite system (negative dt large enough) reports breakdown, not garbage."""
    O = oracle_mod
    g, c, S, W, dtE = case(O, 4, 6, 8)
    u = synth.random_field(g.shape, 2)
    x, it, rel, st = O.be_pcg(g, S, W, u, -50 * dtE, rtol=1e-12, maxit=500)
    assert st in (1, 2)
    assert st == 2 or rel > 1e-12
