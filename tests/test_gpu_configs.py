"""The two other full-size workloads, each checked against the oracle on the whole grid:

* mixed precision at 256 x 384 x 768 (75.5 M cells): FP32 stages with FP64 recurrence
  coefficients, and FP32 PCG inside FP64 iterative refinement;
* viscosity on three velocity components at 192 x 288 x 576 (31.9 M cells) at
  dt = 500 dt_exp, FP64 and mixed precision, RKL2 and BE + PCG (Jacobi).

RKL2 results are compared element by element with the oracle's super-step (FP64: 1e-12
relative L2; mixed: the bound 4 s u32 ||change|| derived in test_gpu_mixed.py); BE results
by their true FP64 residual evaluated with the oracle's operator.  The oracle assembles
the full operator on the host (about 11 GB for 75.5 M cells), so these tests also need
that much host memory.
"""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def R():
    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg

    B.build()
    return rklpcg


def dev(a):
    import torch

    return torch.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)


def _residual_ok(O, g, S, W, u0, x, dt, rtol=1e-10):
    Wg = W.reshape(g.shape)
    res = Wg * (u0 - x + dt * O.apply_F(g, S, W, x))
    return np.linalg.norm(res) <= 2 * rtol * np.linalg.norm(Wg * u0)


def test_mixed_precision_256x384x768(oracle_mod, R):
    O = oracle_mod
    nr, nth, nph = 256, 384, 768
    c = synth.conduction_case(nr, nth, nph, seed=1)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], nth, nph, prec=R.RKL_F32MIX)
    T = dev(c["T"])
    dte = ctx.set_conduction(T, dev(c["bhat"]), dev(c["n"]))
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-12)
    u = T.clone()
    s = ctx.rkl2_superstep(u, 100 * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], 100 * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    assert np.linalg.norm(out - ref) <= 4 * s * U32 * np.linalg.norm(ref - c["T"])
    del ref, out
    u = T.clone()
    code, its, rel = ctx.be_pcg_solve(u, 100 * dte, pc=R.RKL_PC_JACOBI, rtol=1e-10, maxit=20000)
    assert code == R.RKL_OK and rel[0] <= 1e-10
    assert _residual_ok(O, g, S, W, c["T"], u.cpu().numpy().reshape(g.shape), 100 * dte)
    ctx.close()


@pytest.fixture(scope="module")
def visc_case(oracle_mod):
    nr, nth, nph = 192, 288, 576
    v = synth.viscosity_case(nr, nth, nph, seed=1)
    g = oracle_mod.Grid(v["rf"], nth, nph)
    S, W = oracle_mod.assemble_viscosity(g, v["rho"], v["nu"])
    return v, g, S, W


@pytest.mark.parametrize("prec", ["f64", "mix"])
def test_viscosity_192x288x576(oracle_mod, R, visc_case, prec):
    O = oracle_mod
    v, g, S, W = visc_case
    ctx = R.Context(v["rf"], g.nth, g.nph, prec=R.RKL_F64 if prec == "f64" else R.RKL_F32MIX)
    dte = ctx.set_viscosity(dev(v["rho"]), dev(v["nu"]))
    vel = dev(v["v"])
    u = vel.clone()
    s = ctx.rkl2_superstep(u, 500 * dte, dte, ncomp=3)
    out = u.cpu().numpy().reshape((3,) + g.shape)
    for q in range(3):
        ref = O.rkl2_superstep(g, S, W, v["v"][q], 500 * dte, s)
        err = np.linalg.norm(out[q] - ref)
        if prec == "f64":
            assert err <= 1e-12 * np.linalg.norm(ref)
        else:
            assert err <= 4 * s * U32 * np.linalg.norm(ref - v["v"][q])
    u = vel.clone()
    code, its, rel = ctx.be_pcg_solve(u, 500 * dte, pc=R.RKL_PC_JACOBI, rtol=1e-10, maxit=20000, ncomp=3)
    assert code == R.RKL_OK and max(rel) <= 1e-10
    out = u.cpu().numpy().reshape((3,) + g.shape)
    for q in range(3):
        assert _residual_ok(O, g, S, W, v["v"][q], out[q], 500 * dte)
    ctx.close()
