"""Parity at the benchmark's own size (128 x 192 x 384 cells, the launch configuration
bench.py times): CUDA path vs oracle on the full grid for the operator, one RKL2
super-step and BE+PCG at a fixed number of iterations, plus properties that hold at any
size (conservation of sum W u by RKL2, symmetry <u, S v> = <v, S u>)."""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (128, 192, 384)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def full(oracle_mod):
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    B.build()
    O = oracle_mod
    c = synth.conduction_case(*DIMS, seed=1)
    g = O.Grid(c["rf"], DIMS[1], DIMS[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    ctx = R.Context(c["rf"], DIMS[1], DIMS[2])
    dte = ctx.set_conduction(T, b, n)
    yield O, R, torch, c, g, S, W, ctx, T, dte
    ctx.close()


def test_fullsize_operator_and_dt_exp(full):
    O, R, torch, c, g, S, W, ctx, T, dte = full
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-13)
    u = synth.random_field(g.shape, 21)
    Fu = torch.empty_like(T)
    ctx.apply_F(torch.from_numpy(u.reshape(-1)).cuda(), Fu)
    F_o = O.apply_F(g, S, W, u)
    scale = -O.apply_F(g, np.abs(S), W, np.abs(u))
    F = Fu.cpu().numpy().reshape(g.shape)
    assert np.all(np.abs(F - F_o) <= 1e-12 * scale + 1e-300)
    assert _rel(F, F_o) <= 1e-12
    # symmetry of S at full size, through the GPU operator: <u, W F(v)> = <v, W F(u)>
    v = synth.random_field(g.shape, 22)
    Fv = torch.empty_like(T)
    ctx.apply_F(torch.from_numpy(v.reshape(-1)).cuda(), Fv)
    Wg = W.reshape(g.shape)
    a = float(np.sum(u * Wg * Fv.cpu().numpy().reshape(g.shape)))
    bsum = float(np.sum(v * Wg * F))
    assert abs(a - bsum) <= 1e-12 * float(np.sum(np.abs(u * Wg * F_o)))


def test_fullsize_rkl2_superstep(full):
    O, R, torch, c, g, S, W, ctx, T, dte = full
    u = T.clone()
    s = ctx.rkl2_superstep(u, 100 * dte, dte)
    assert s == 20
    ref = O.rkl2_superstep(g, S, W, c["T"], 100 * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    assert _rel(out, ref) <= 1e-12
    e0 = float(np.sum(W * c["T"].ravel()))
    assert abs(float(np.sum(W * out.ravel())) - e0) <= 1e-13 * abs(e0)


@pytest.mark.parametrize("pc", [1, 2])
def test_fullsize_be_pcg_fixed_iterations(full, pc):
    O, R, torch, c, g, S, W, ctx, T, dte = full
    u = T.clone()
    code, its, rel = ctx.be_pcg_solve(u, 1000 * dte, pc=pc, block=(8, 8, 8), rtol=0.0, maxit=6)
    assert code == R.RKL_ENOTCONV and its == [6]
    x, it_o, rel_o, st = O.be_pcg(g, S, W, c["T"], 1000 * dte, pc=pc, block=(8, 8, 8), fixed_iters=6)
    assert _rel(u.cpu().numpy().reshape(g.shape), x) <= 1e-12
    assert rel[0] == pytest.approx(rel_o, rel=1e-6)
