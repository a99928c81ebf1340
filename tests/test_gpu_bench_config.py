"""Parity on exactly what bench.py times: 128 x 192 x 384 cells, seed 1, conduction with
beta_Tcut (Sec. 4.1), RKL2 super-steps at dt / dt_exp = 1000 and 10000 (s = 63, 200;
Fig. 2), BE + PCG (Fig. 1) converged to rtol 1e-10 with point Jacobi and 8 x 8 x 8
block ILU0 (App. A) at 100, 1000 and 10000 dt_exp, and viscosity on the three Cartesian
components at 500 dt_exp (RKL2 s = 45, both preconditioners).

Tolerances:
* RKL2 super-step: relative L2 <= 1e-12 against the oracle (the FP64 per-large-step
  tolerance), sum W u conserved to 1e-13;
* BE at a fixed number of iterations: relative L2 <= 1e-12 against the oracle;
* BE to rtol: the true FP64 residual ||W u^n - (W + dt S) x|| (formed with the oracle's
  operator) <= 2 rtol ||W u^n||, and the iteration count within one of the oracle's
  converged count (live oracle solves at 100 dt_exp; at 1000 and 10000 dt_exp, and for
  viscosity, the counts the committed script tests/golden/make_bench_config_iters.py
  wrote from the oracle).
"""
import json
import os

import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (128, 192, 384)
RTOL = 1e-10
BLOCK = (8, 8, 8)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bench_config_iters.json")


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _true_relres(O, g, S, W, u0, x, dt):
    """||W u^n - (W + dt S) x|| / ||W u^n|| with the oracle's operator (S x = -W F(x))."""
    Wg = W.reshape(g.shape)
    x = np.asarray(x).reshape(g.shape)
    r = Wg * (u0 - x + dt * O.apply_F(g, S, W, x))
    return float(np.linalg.norm(r) / np.linalg.norm(Wg * u0))


@pytest.fixture(scope="module")
def cond(oracle_mod):
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    B.build()
    O = oracle_mod
    c = synth.conduction_case(*DIMS, seed=1)
    assert (c["T"] < 5e5).any()  # beta_Tcut acts on this input
    g = O.Grid(c["rf"], DIMS[1], DIMS[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    ctx = R.Context(c["rf"], DIMS[1], DIMS[2])
    dte = ctx.set_conduction(T, b, n, beta_tcut=True)
    yield O, R, torch, c, g, S, W, ctx, T, dte
    ctx.close()


@pytest.fixture(scope="module")
def visc(oracle_mod):
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    B.build()
    O = oracle_mod
    v = synth.viscosity_case(*DIMS, seed=1)
    g = O.Grid(v["rf"], DIMS[1], DIMS[2])
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    ctx = R.Context(v["rf"], DIMS[1], DIMS[2])
    dte = ctx.set_viscosity(dev(v["rho"]), dev(v["nu"]))
    yield O, R, torch, v, g, S, W, ctx, dev(v["v"]), dte
    ctx.close()


def test_bench_dt_exp_beta_tcut(cond):
    O, R, torch, c, g, S, W, ctx, T, dte = cond
    assert dte == pytest.approx(O.gershgorin_dt(g, S, W)[0], rel=1e-13)
    gold = _golden()["conduction"]["dt_exp"]
    assert dte == pytest.approx(gold, rel=1e-12)


@pytest.mark.parametrize("ratio,s_expect", [(1000.0, 63), (10000.0, 200)])
def test_bench_rkl2_superstep(cond, ratio, s_expect):
    O, R, torch, c, g, S, W, ctx, T, dte = cond
    u = T.clone()
    s = ctx.rkl2_superstep(u, ratio * dte, dte)
    assert s == s_expect
    ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    assert _rel(out, ref) <= 1e-12
    e0 = float(np.sum(W * c["T"].ravel()))
    assert abs(float(np.sum(W * out.ravel())) - e0) <= 1e-13 * abs(e0)


@pytest.mark.parametrize("pc", [1, 2])
@pytest.mark.parametrize("ratio", [100.0, 1000.0, 10000.0])
def test_bench_be_pcg_converged(cond, pc, ratio):
    O, R, torch, c, g, S, W, ctx, T, dte = cond
    dt = ratio * dte
    u = T.clone()
    code, its, rel = ctx.be_pcg_solve(u, dt, pc=pc, block=BLOCK, rtol=RTOL, maxit=20000)
    assert code == R.RKL_OK and rel[0] <= RTOL
    x = u.cpu().numpy()
    assert _true_relres(O, g, S, W, c["T"], x, dt) <= 2 * RTOL
    name = {1: "jacobi", 2: "bilu0"}[pc]
    if ratio == 100.0:  # live oracle solve
        x_o, it_o, rel_o, st = O.be_pcg(g, S, W, c["T"], dt, pc=pc, block=BLOCK, rtol=RTOL, maxit=20000)
        assert st == 0 and abs(its[0] - it_o) <= 1
        # both solutions lie within the residual-implied distance of the exact one
        assert _rel(x.reshape(g.shape), x_o) <= 1e-6
    else:
        it_o = _golden()["conduction"][f"{name}_{int(ratio)}"]["iters"]
        assert abs(its[0] - it_o) <= 1


def test_bench_viscosity_rkl2(visc):
    O, R, torch, v, g, S, W, ctx, V, dte = visc
    u = V.clone()
    s = ctx.rkl2_superstep(u, 500 * dte, dte, ncomp=3)
    assert s == 45
    out = u.cpu().numpy().reshape(3, *g.shape)
    for q in range(3):
        ref = O.rkl2_superstep(g, S, W, v["v"][q], 500 * dte, s)
        assert _rel(out[q], ref) <= 1e-12


def test_bench_viscosity_be_bilu0_fixed_iterations(visc):
    O, R, torch, v, g, S, W, ctx, V, dte = visc
    u = V.clone()
    code, its, rel = ctx.be_pcg_solve(u, 500 * dte, pc=2, block=BLOCK, rtol=0.0, maxit=6, ncomp=3)
    assert code == R.RKL_ENOTCONV and its == [6, 6, 6]
    out = u.cpu().numpy().reshape(3, *g.shape)
    for q in range(3):
        x, *_ = O.be_pcg(g, S, W, v["v"][q], 500 * dte, pc=2, block=BLOCK, fixed_iters=6, pattern=7)
        assert _rel(out[q], x) <= 1e-12


@pytest.mark.parametrize("pc", [1, 2])
def test_bench_viscosity_be_converged(visc, pc):
    O, R, torch, v, g, S, W, ctx, V, dte = visc
    dt = 500 * dte
    u = V.clone()
    code, its, rel = ctx.be_pcg_solve(u, dt, pc=pc, block=BLOCK, rtol=RTOL, maxit=20000, ncomp=3)
    assert code == R.RKL_OK and max(rel) <= RTOL
    out = u.cpu().numpy().reshape(3, *g.shape)
    name = {1: "jacobi", 2: "bilu0"}[pc]
    gold = _golden()["viscosity"][f"{name}_500"]["iters"]
    for q in range(3):
        assert _true_relres(O, g, S, W, v["v"][q], out[q], dt) <= 2 * RTOL
        assert abs(its[q] - gold[q]) <= 1
