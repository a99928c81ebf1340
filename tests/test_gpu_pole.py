"""Across-pole theta-ghosts (set_coeffs flag RKL_ACROSS_POLE; Sec. 4.2 boundaries): CUDA
path against the oracle's across-pole operator on seeded inputs.

Tolerances as in test_gpu_parity.py: apply_F per cell within 1e-12 of W^-1 |S| |u| and
1e-12 relative L2; dt_exp 1e-13 relative; one RKL2 super-step and BE at a fixed number of
CG iterations (Jacobi, and block ILU0, which drops the across-pole couplings on both
sides) 1e-12 relative L2; mixed precision within its FP32 bound / to the FP64 rtol.
"""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

GRIDS = [(5, 8, 12), (16, 12, 24), (32, 32, 64)]


@pytest.fixture(scope="module")
def R():
    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg

    B.build()
    rklpcg.load()
    return rklpcg


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).cuda().view(-1)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _setup(O, R, torch, dims, seed=1, prec=None, beta_tcut=True):
    nr, nth, nph = dims
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=beta_tcut, across_pole=True)
    ctx = R.Context(c["rf"], nth, nph, prec=R.RKL_F64 if prec is None else prec)
    dte = ctx.set_conduction(_dev(torch, c["T"]), _dev(torch, c["bhat"]), _dev(torch, c["n"]), beta_tcut=beta_tcut,
                             across_pole=True)
    return c, g, S, W, ctx, dte


@pytest.mark.parametrize("dims", GRIDS)
def test_pole_apply_F_and_dt_exp(oracle_mod, R, torch_cuda, dims):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = _setup(O, R, torch, dims)
    assert dte == pytest.approx(O.gershgorin_dt(g, S, W)[0], rel=1e-13)
    u = synth.random_field(g.shape, 11)
    Fu = torch.empty(g.N, dtype=torch.float64, device="cuda")
    ctx.apply_F(_dev(torch, u), Fu)
    F = Fu.cpu().numpy().reshape(g.shape)
    F_o = O.apply_F(g, S, W, u)
    scale = -O.apply_F(g, np.abs(S), W, np.abs(u))
    assert np.all(np.abs(F - F_o) <= 1e-12 * scale + 1e-300)
    assert _rel(F, F_o) <= 1e-12
    # the option is really on: the pole rows differ from the mirror-ghost operator
    Sm, _ = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True)
    Fm = O.apply_F(g, Sm, W, u)
    assert np.abs(F - Fm)[:, (0, -1), :].max() > 1e-6 * np.abs(Fm).max()
    ctx.close()


@pytest.mark.parametrize("dims", GRIDS[1:])
def test_pole_rkl2_superstep(oracle_mod, R, torch_cuda, dims):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = _setup(O, R, torch, dims)
    u = _dev(torch, c["T"])
    s = ctx.rkl2_superstep(u, 100 * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], 100 * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    assert _rel(out, ref) <= 1e-12
    e0 = float(np.sum(W * c["T"].ravel()))
    assert abs(float(np.sum(W * out.ravel())) - e0) <= 1e-13 * abs(e0)
    ctx.close()


@pytest.mark.parametrize("pc,block,dims", [(1, (8, 8, 8), (16, 12, 24)), (2, (4, 4, 4), (16, 12, 24)),
                                           (1, (8, 8, 8), (32, 32, 64)), (2, (8, 8, 8), (32, 32, 64))])
def test_pole_be_pcg_fixed_iterations(oracle_mod, R, torch_cuda, pc, block, dims):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = _setup(O, R, torch, dims)
    u = _dev(torch, c["T"])
    code, its, rel = ctx.be_pcg_solve(u, 300 * dte, pc=pc, block=block, rtol=0.0, maxit=8)
    assert code == R.RKL_ENOTCONV and its == [8]
    x, *_ = O.be_pcg(g, S, W, c["T"], 300 * dte, pc=pc, block=block, fixed_iters=8)
    assert _rel(u.cpu().numpy().reshape(g.shape), x) <= 1e-12
    ctx.close()


def test_pole_be_pcg_converged_true_residual(oracle_mod, R, torch_cuda):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = _setup(O, R, torch, (32, 32, 64))
    dt = 300 * dte
    for pc in (1, 2):
        u = _dev(torch, c["T"])
        code, its, rel = ctx.be_pcg_solve(u, dt, pc=pc, block=(8, 8, 8), rtol=1e-10, maxit=5000)
        assert code == R.RKL_OK
        x = u.cpu().numpy().reshape(g.shape)
        Wg = W.reshape(g.shape)
        r = Wg * (c["T"] - x + dt * O.apply_F(g, S, W, x))
        assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(Wg * c["T"])
        _, it_o, _, st = O.be_pcg(g, S, W, c["T"], dt, pc=pc, block=(8, 8, 8), rtol=1e-10, maxit=5000)
        assert st == 0 and abs(it_o - its[0]) <= 1
    ctx.close()


def test_pole_mixed_precision(oracle_mod, R, torch_cuda):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = _setup(O, R, torch, (32, 32, 64), prec=R.RKL_F32MIX)
    u = _dev(torch, c["T"])
    s = ctx.rkl2_superstep(u, 100 * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], 100 * dte, s)
    err = np.linalg.norm(u.cpu().numpy().reshape(g.shape) - ref)
    assert err <= 4 * s * 2.0 ** -24 * np.linalg.norm(ref - c["T"])
    dt = 300 * dte
    u = _dev(torch, c["T"])
    code, its, rel = ctx.be_pcg_solve(u, dt, pc=R.RKL_PC_BILU0, block=(8, 8, 8), rtol=1e-10, maxit=5000)
    assert code == R.RKL_OK
    x = u.cpu().numpy().reshape(g.shape)
    Wg = W.reshape(g.shape)
    r = Wg * (c["T"] - x + dt * O.apply_F(g, S, W, x))
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(Wg * c["T"])
    ctx.close()


def test_pole_rejected_where_it_cannot_apply(R, torch_cuda):
    torch = torch_cuda
    for dims, kw in (((4, 4, 7), {}), ((4, 1, 8), {}), ((4, 4, 8), {"flux_form": True})):
        c = synth.conduction_case(*dims, seed=1)
        with R.Context(c["rf"], dims[1], dims[2]) as ctx:
            with pytest.raises(R.RklError) as e:
                ctx.set_conduction(_dev(torch, c["T"]), _dev(torch, c["bhat"]), _dev(torch, c["n"]), across_pole=True,
                                   **kw)
            assert e.value.code == R.RKL_EINVAL
