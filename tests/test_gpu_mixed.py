"""Mixed-precision path (RKL_F32MIX) against the FP64 oracle.

RKL2: the stages run in FP32 on the increments delta_j = Y_j - Y_0 (M0 and Y_0 + delta_s
in FP64).  Each stage rounds delta to FP32 (unit roundoff u = 2^-24) and the recurrence
carries earlier roundings with weights of order one, so the error of the result is a
modest multiple of s * u * ||delta||; the tests require
    ||u_mix - u_oracle|| <= 4 s u ||u_oracle - u_0||      (s = number of stages).
BE: FP64 iterative refinement around FP32 PCG stops on the FP64 residual, so the result
must meet the same true-residual bound as the FP64 solver, ||r|| <= 2 rtol ||W u||.
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

    return torch.from_numpy(np.array(a, dtype=np.float64)).cuda()


# nr a multiple of 4 up to 256 runs the phi-marching kernels fed by bulk copies: (128, 20,
# 9), (256, 10, 7) and (32, 70, 5) have several theta tiles with halo rows on both sides,
# (128, 40, 96) phi chunks long enough for the steady refill of the copy rings, (36, 11,
# 13), (132, 6, 8) and (8, 5, 6) tiles with idle threads; (37, 11, 13) and (260, 6, 4) run
# the one-cell-per-thread kernels
@pytest.mark.parametrize("dims", [(16, 12, 24), (32, 32, 64), (36, 11, 13), (132, 6, 8), (8, 5, 6),
                                  (128, 20, 9), (256, 10, 7), (32, 70, 5), (128, 40, 96), (37, 11, 13),
                                  (260, 6, 4)])
@pytest.mark.parametrize("ratio", [100.0, 1000.0, 10000.0])
def test_mixed_rkl2_conduction(oracle_mod, R, dims, ratio):
    O = oracle_mod
    c = synth.conduction_case(*dims, seed=1)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], dims[1], dims[2], prec=R.RKL_F32MIX)
    dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]))
    u = dev(c["T"])
    s = ctx.rkl2_superstep(u, ratio * dte, dte)
    ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
    out = u.cpu().numpy().reshape(g.shape)
    err = np.linalg.norm(out - ref)
    change = np.linalg.norm(ref - c["T"])
    assert err <= 4 * s * U32 * change, (err / change, s)
    # conservation holds to FP32 accuracy of the increments
    e0 = float(np.sum(W * c["T"].ravel()))
    assert abs(float(np.sum(W * out.ravel())) - e0) <= 4 * s * U32 * float(np.sum(np.abs(W * (ref - c["T"]).ravel())))
    ctx.close()


# viscosity through the phi-marching bulk-copy kernels ((128, 20, 9), (256, 10, 7): several
# theta tiles; (36, 11, 13): idle threads) and the one-cell-per-thread ones ((37, 11, 13))
@pytest.mark.parametrize("dims", [(16, 12, 24), (128, 20, 9), (256, 10, 7), (36, 11, 13), (37, 11, 13)])
def test_mixed_rkl2_viscosity(oracle_mod, R, dims):
    O = oracle_mod
    v = synth.viscosity_case(*dims, seed=2)
    g = O.Grid(v["rf"], dims[1], dims[2])
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    ctx = R.Context(v["rf"], dims[1], dims[2], prec=R.RKL_F32MIX)
    dte = ctx.set_viscosity(dev(v["rho"]), dev(v["nu"]))
    u = dev(v["v"])
    s = ctx.rkl2_superstep(u, 500 * dte, dte, ncomp=3)
    out = u.cpu().numpy().reshape((3,) + g.shape)
    for q in range(3):
        ref = O.rkl2_superstep(g, S, W, v["v"][q], 500 * dte, s)
        assert np.linalg.norm(out[q] - ref) <= 4 * s * U32 * np.linalg.norm(ref - v["v"][q])
    ctx.close()


# (37, 11, 13) runs the one-cell-per-thread FP32 SpMV, the others the phi-marching one fed
# by bulk copies ((36, 11, 13) and (132, 6, 8) with idle threads, (128, 40, 96) with
# several theta tiles and longer phi chunks); block ILU0 on thin (nr, nth, 1) blocks is a
# weaker preconditioner than Jacobi (1161 vs 703 FP64 iterations at 1e4 dt_exp on
# 37 x 11 x 13), so those cases run at 100 dt_exp
@pytest.mark.parametrize("pc,ratio,dims", [(1, 100.0, (32, 32, 64)), (2, 100.0, (32, 32, 64)),
                                           (1, 10000.0, (32, 32, 64)), (2, 10000.0, (32, 32, 64)),
                                           (1, 10000.0, (37, 11, 13)), (2, 100.0, (37, 11, 13)),
                                           (1, 10000.0, (36, 11, 13)), (2, 100.0, (36, 11, 13)),
                                           (1, 1000.0, (132, 6, 8)), (1, 1000.0, (128, 40, 96)),
                                           (2, 1000.0, (128, 40, 96))])
def test_mixed_be_meets_fp64_residual(oracle_mod, R, pc, ratio, dims):
    O = oracle_mod
    block = (8, 8, 8) if all(n % 8 == 0 for n in dims) else (dims[0], dims[1], 1)
    c = synth.conduction_case(*dims, seed=3)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], dims[1], dims[2], prec=R.RKL_F32MIX)
    dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]))
    u = dev(c["T"])
    code, its, rel = ctx.be_pcg_solve(u, ratio * dte, pc=pc, block=block, rtol=1e-10, maxit=20000)
    assert code == R.RKL_OK and rel[0] <= 1e-10
    xg = u.cpu().numpy().reshape(g.shape)
    Wg = W.reshape(g.shape)
    res = Wg * (c["T"] - xg + ratio * dte * O.apply_F(g, S, W, xg))
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(Wg * c["T"])
    x64, it64, rel64, st = O.be_pcg(g, S, W, c["T"], ratio * dte, pc=pc, block=block, rtol=1e-10)
    assert its[0] <= 3 * it64 + 50  # FP32 correction solves restart CG a few times
    ctx.close()


@pytest.mark.parametrize("pc,dims,block", [(2, (16, 12, 24), (4, 4, 4)), (1, (128, 20, 16), (8, 4, 8)),
                                           (2, (128, 20, 16), (8, 4, 8))])
def test_mixed_be_viscosity_three_components(oracle_mod, R, pc, dims, block):
    O = oracle_mod
    v = synth.viscosity_case(*dims, seed=1)
    g = O.Grid(v["rf"], dims[1], dims[2])
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    ctx = R.Context(v["rf"], dims[1], dims[2], prec=R.RKL_F32MIX)
    dte = ctx.set_viscosity(dev(v["rho"]), dev(v["nu"]))
    u = dev(v["v"])
    code, its, rel = ctx.be_pcg_solve(u, 500 * dte, pc=pc, block=block, rtol=1e-10, maxit=20000, ncomp=3)
    assert code == R.RKL_OK and max(rel) <= 1e-10
    out = u.cpu().numpy().reshape((3,) + g.shape)
    Wg = W.reshape(g.shape)
    for q in range(3):
        res = Wg * (v["v"][q] - out[q] + 500 * dte * O.apply_F(g, S, W, out[q]))
        assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(Wg * v["v"][q])
    ctx.close()
