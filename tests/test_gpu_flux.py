"""The non-symmetric flux form of conduction (RKL_FLUX_FORM) against the oracle.

Same bars as the symmetric operator (test_gpu_parity.py): the operator, dt_exp, RKL2
super-steps and BE + PCG at a fixed number of iterations within 1e-12 relative L2 of the
oracle (the arithmetic is the same FP64 sums in another order); converged BE + PCG by
its true FP64 residual with the oracle's operator; the mixed-precision path by the
bounds of test_gpu_mixed.py; and the full-size grid of the benchmark.
"""
import ctypes

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


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _setup(O, R, dims, seed=1, prec=None, tcut=False):
    nr, nth, nph = dims
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=tcut, flux_form=True)
    ctx = R.Context(c["rf"], nth, nph, prec=R.RKL_F64 if prec is None else prec)
    dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]), beta_tcut=tcut, flux_form=True)
    return c, g, S, W, ctx, dte


@pytest.mark.parametrize("dims", [(16, 12, 24), (32, 32, 64), (7, 5, 3)])
def test_operator_and_dt_exp(oracle_mod, R, dims):
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, dims, tcut=True)
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-13)
    u = synth.random_field(g.shape, 5)
    Fu = dev(np.zeros(g.N))
    ctx.apply_F(dev(u), Fu)
    F = Fu.cpu().numpy().reshape(g.shape)
    F_o = O.apply_F(g, S, W, u)
    scale = -O.apply_F(g, np.abs(S), W, np.abs(u))
    assert np.all(np.abs(F - F_o) <= 1e-12 * scale + 1e-300)
    ctx.close()


@pytest.mark.parametrize("ratio", [30.0, 1000.0])
def test_rkl2_superstep(oracle_mod, R, ratio):
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, (32, 32, 64), seed=2)
    u = dev(c["T"])
    s = ctx.rkl2_superstep(u, ratio * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
    assert _rel(u.cpu().numpy().reshape(g.shape), ref) <= 1e-12
    # the flux form conserves sum W u exactly in exact arithmetic (zero column sums)
    e0 = float(np.sum(W * c["T"].ravel()))
    assert abs(float(np.sum(W * u.cpu().numpy())) - e0) <= 1e-13 * abs(e0)
    ctx.close()


@pytest.mark.parametrize("pc,block", [(1, (8, 8, 8)), (2, (8, 8, 8)), (2, (4, 6, 8))])
def test_be_pcg_fixed_iterations(oracle_mod, R, pc, block):
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, (32, 24, 64), seed=3)
    u = dev(c["T"])
    code, its, rel = ctx.be_pcg_solve(u, 300 * dte, pc=pc, block=block, rtol=0.0, maxit=7)
    assert code == R.RKL_ENOTCONV and its == [7]
    x, it_o, rel_o, st = O.be_pcg(g, S, W, c["T"], 300 * dte, pc=pc, block=block, fixed_iters=7)
    assert _rel(u.cpu().numpy().reshape(g.shape), x) <= 1e-12
    assert rel[0] == pytest.approx(rel_o, rel=1e-6)
    ctx.close()


# CG with point Jacobi stalls on the flux form once dt >= ~100 dt_exp (the antisymmetric
# part, scaled by dt, outweighs W); block ILU0 converges at 1000 dt_exp in about as many
# iterations as on the symmetric form.  Both regimes are tested where they converge.
@pytest.mark.parametrize("pc,ratio", [(1, 30.0), (2, 1000.0)])
@pytest.mark.parametrize("prec", ["f64", "mix"])
def test_be_pcg_converged_true_residual(oracle_mod, R, pc, ratio, prec):
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, (32, 32, 64), seed=4, prec=R.RKL_F64 if prec == "f64" else R.RKL_F32MIX)
    u = dev(c["T"])
    dt = ratio * dte
    code, its, rel = ctx.be_pcg_solve(u, dt, pc=pc, block=(8, 8, 8), rtol=1e-10, maxit=20000)
    assert code == R.RKL_OK and rel[0] <= 1e-10
    x = u.cpu().numpy().reshape(g.shape)
    Wg = W.reshape(g.shape)
    res = Wg * (c["T"] - x + dt * O.apply_F(g, S, W, x))
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(Wg * c["T"])
    if prec == "f64":
        x_o, it_o, _, st = O.be_pcg(g, S, W, c["T"], dt, pc=pc, block=(8, 8, 8), rtol=1e-10)
        assert st == 0 and abs(its[0] - it_o) <= 1
    ctx.close()


def test_mixed_rkl2(oracle_mod, R):
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, (32, 32, 64), seed=5, prec=R.RKL_F32MIX)
    u = dev(c["T"])
    s = ctx.rkl2_superstep(u, 1000 * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], 1000 * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    assert np.linalg.norm(out - ref) <= 4 * s * U32 * np.linalg.norm(ref - c["T"])
    ctx.close()


def test_switching_forms_on_one_context(oracle_mod, R):
    """A context moves between the symmetric and the flux form (full rows need more
    coefficient storage; the switch reallocates it) and back."""
    O = oracle_mod
    dims = (16, 12, 24)
    c = synth.conduction_case(*dims, seed=6)
    g = O.Grid(c["rf"], dims[1], dims[2])
    ctx = R.Context(c["rf"], dims[1], dims[2])
    u = synth.random_field(g.shape, 7)
    for flux in (False, True, False, True):
        S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], flux_form=flux)
        ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]), flux_form=flux)
        Fu = dev(np.zeros(g.N))
        ctx.apply_F(dev(u), Fu)
        assert _rel(Fu.cpu().numpy().reshape(g.shape), O.apply_F(g, S, W, u)) <= 1e-12
    ctx.close()


def test_invalid_uses(R):
    import torch

    c = synth.conduction_case(8, 6, 8, seed=1)
    v = synth.viscosity_case(8, 6, 8, seed=1)
    ctx = R.Context(v["rf"], 6, 8)
    lib = R.load()
    dte = ctypes.c_double(0.0)
    code = lib.set_coeffs(ctx.handle, R.RKL_OP_VISCOSITY, dev(v["rho"]).data_ptr(), None,
                          dev(v["nu"]).data_ptr(), 0.0, R.RKL_FLUX_FORM, ctypes.byref(dte))
    assert code == R.RKL_EINVAL
    ctx.close()
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    u = T.clone()
    g = R._Grid(8, 6, 8, np.ascontiguousarray(c["rf"]).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    code = lib.rkl2_superstep_noalloc(ctypes.byref(g), T.data_ptr(), b.data_ptr(), n.data_ptr(), 9e-7,
                                      R.RKL_FLUX_FORM, u.data_ptr(), 1.0, 0, 0,
                                      torch.cuda.current_stream().cuda_stream, None, None)
    assert code == R.RKL_EINVAL
    assert torch.equal(u, T)


def test_fullsize_flux_form(oracle_mod, R):
    """128 x 192 x 384 (the benchmark's grid): operator and one RKL2 super-step."""
    O = oracle_mod
    c, g, S, W, ctx, dte = _setup(O, R, (128, 192, 384), seed=1, tcut=True)
    u = dev(c["T"])
    s = ctx.rkl2_superstep(u, 100 * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], 100 * dte, s)
    assert _rel(u.cpu().numpy().reshape(g.shape), ref) <= 1e-12
    ctx.close()
