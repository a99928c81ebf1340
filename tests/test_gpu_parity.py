"""GPU (C-ABI) vs oracle parity on seeded synthetic inputs.

Tolerances (FP64 both sides, different summation orders and coefficient rounding):
* apply_F: |F_gpu - F_oracle| <= 1e-12 * (W^-1 |S| |u|) per cell (the size of the terms
  that cancel in the stencil sum) and relative L2 <= 1e-12;
* one RKL2 super-step, one BE step at a fixed number of CG iterations:
  relative L2 <= 1e-12 (the per-large-step tolerance of the FP64 path);
* BE to rtol: same iteration count within 1, both residuals <= rtol;
* dt_exp (Gershgorin): relative 1e-13.
"""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

GRIDS = [(5, 7, 9), (16, 12, 24), (32, 32, 64)]


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


def dev(torch, a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def cond_setup(O, R, torch, dims, seed=1):
    nr, nth, nph = dims
    c = synth.conduction_case(nr, nth, nph, seed)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], nth, nph)
    dte = ctx.set_conduction(dev(torch, c["T"]), dev(torch, c["bhat"]), dev(torch, c["n"]))
    return c, g, S, W, ctx, dte


def visc_setup(O, R, torch, dims, seed=1):
    nr, nth, nph = dims
    v = synth.viscosity_case(nr, nth, nph, seed)
    g = O.Grid(v["rf"], nth, nph)
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    ctx = R.Context(v["rf"], nth, nph)
    dte = ctx.set_viscosity(dev(torch, v["rho"]), dev(torch, v["nu"]))
    return v, g, S, W, ctx, dte


def check_F(O, g, S, W, u, F_gpu):
    F_o = O.apply_F(g, S, W, u)
    scale = -O.apply_F(g, np.abs(S), W, np.abs(u))
    assert np.all(np.abs(F_gpu - F_o) <= 1e-12 * scale + 1e-300)
    assert rel_l2(F_gpu, F_o) <= 1e-12


@pytest.mark.parametrize("dims", GRIDS)
def test_apply_F_conduction(oracle_mod, R, torch_cuda, dims):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = cond_setup(O, R, torch, dims)
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-13)
    for u in (c["T"], synth.random_field(g.shape, 5)):
        Fu = torch.empty(g.N, dtype=torch.float64, device="cuda")
        ctx.apply_F(dev(torch, u), Fu)
        torch.cuda.synchronize()
        check_F(O, g, S, W, u, host(Fu).reshape(g.shape))


@pytest.mark.parametrize("dims", GRIDS)
def test_apply_F_viscosity(oracle_mod, R, torch_cuda, dims):
    O, torch = oracle_mod, torch_cuda
    v, g, S, W, ctx, dte = visc_setup(O, R, torch, dims)
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-13)
    Fu = torch.empty(3 * g.N, dtype=torch.float64, device="cuda")
    ctx.apply_F(dev(torch, v["v"]), Fu, ncomp=3)
    torch.cuda.synchronize()
    F = host(Fu).reshape((3,) + g.shape)
    for q in range(3):
        check_F(O, g, S, W, v["v"][q], F[q])


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("ratio", [1.0, 100.0, 1000.0])
def test_rkl2_superstep_conduction(oracle_mod, R, torch_cuda, dims, ratio):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = cond_setup(O, R, torch, dims)
    u = dev(torch, c["T"])
    s = ctx.rkl2_superstep(u, ratio * dte, dte)
    assert s == O.rkl2_stages(ratio)
    ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
    torch.cuda.synchronize()
    assert rel_l2(host(u).reshape(g.shape), ref) <= 1e-12


def test_rkl2_explicit_and_odd_stages(oracle_mod, R, torch_cuda):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = cond_setup(O, R, torch, (16, 12, 24), seed=2)
    for s_req, odd, ratio in ((2, False, 0.5), (7, False, 30.0), (0, True, 100.0)):
        u = dev(torch, c["T"])
        s = ctx.rkl2_superstep(u, ratio * dte, dte, s=s_req, force_odd=odd)
        expect_s = s_req if s_req else O.rkl2_stages(ratio, force_odd=True)
        assert s == expect_s and (not odd or s % 2 == 1)
        ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
        assert rel_l2(host(u).reshape(g.shape), ref) <= 1e-12


def test_rkl2_viscosity_three_components(oracle_mod, R, torch_cuda):
    O, torch = oracle_mod, torch_cuda
    v, g, S, W, ctx, dte = visc_setup(O, R, torch, (16, 12, 24))
    u = dev(torch, v["v"])
    s = ctx.rkl2_superstep(u, 500 * dte, dte, ncomp=3)
    out = host(u).reshape((3,) + g.shape)
    for q in range(3):
        ref = O.rkl2_superstep(g, S, W, v["v"][q], 500 * dte, s)
        assert rel_l2(out[q], ref) <= 1e-12


@pytest.mark.parametrize("pc,block", [(1, (8, 8, 8)), (2, (4, 6, 8)), (2, (4, 4, 4)), (2, (2, 3, 4)),
                                      (2, (16, 1, 1)), (2, (1, 1, 1))])
@pytest.mark.parametrize("ratio", [100.0, 10000.0])
def test_be_pcg_fixed_iterations(oracle_mod, R, torch_cuda, pc, block, ratio):
    """Same number of CG iterations on both sides (rtol <= 0 runs exactly maxit)."""
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = cond_setup(O, R, torch, (16, 12, 24))
    for k in (1, 7, 25):
        u = dev(torch, c["T"])
        code, its, rel = ctx.be_pcg_solve(u, ratio * dte, pc=pc, block=block, rtol=0.0, maxit=k)
        assert code == R.RKL_ENOTCONV and its == [k]
        x, it_o, rel_o, st = O.be_pcg(g, S, W, c["T"], ratio * dte, pc=pc, block=block, fixed_iters=k)
        assert rel_l2(host(u).reshape(g.shape), x) <= 1e-12
        assert rel[0] == pytest.approx(rel_o, rel=1e-6)


@pytest.mark.parametrize("dims,block", [((16, 12, 24), (4, 4, 4)), ((32, 32, 64), (8, 8, 8))])
@pytest.mark.parametrize("ratio", [100.0, 1000.0])
def test_be_pcg_converged(oracle_mod, R, torch_cuda, dims, block, ratio):
    O, torch = oracle_mod, torch_cuda
    c, g, S, W, ctx, dte = cond_setup(O, R, torch, dims)
    for pc in (1, 2):
        u = dev(torch, c["T"])
        code, its, rel = ctx.be_pcg_solve(u, ratio * dte, pc=pc, block=block, rtol=1e-10, maxit=5000)
        x, it_o, rel_o, st = O.be_pcg(g, S, W, c["T"], ratio * dte, pc=pc, block=block, rtol=1e-10, maxit=5000)
        assert code == R.RKL_OK and st == 0
        assert abs(its[0] - it_o) <= 1
        assert rel[0] <= 1e-10 and rel_o <= 1e-10
        # true residual of the GPU solution under the oracle's operator:
        # W u - (W + dt S) x = W (u - x + dt F(x))
        xg = host(u).reshape(g.shape)
        Wg = W.reshape(g.shape)
        res = Wg * (c["T"] - xg + ratio * dte * O.apply_F(g, S, W, xg))
        assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(Wg * c["T"])


def test_be_pcg_viscosity_and_initial_guess(oracle_mod, R, torch_cuda):
    O, torch = oracle_mod, torch_cuda
    v, g, S, W, ctx, dte = visc_setup(O, R, torch, (16, 12, 24))
    for pc in (1, 2):
        u = dev(torch, v["v"])
        code, its, rel = ctx.be_pcg_solve(u, 500 * dte, pc=pc, block=(4, 4, 4), rtol=0.0, maxit=12, ncomp=3)
        out = host(u).reshape((3,) + g.shape)
        for q in range(3):
            x, *_ = O.be_pcg(g, S, W, v["v"][q], 500 * dte, pc=pc, block=(4, 4, 4), fixed_iters=12, pattern=7)
            assert rel_l2(out[q], x) <= 1e-12
    # an initial guess is honoured: start from the oracle's converged solution
    x_ref, *_ = O.be_pcg(g, S, W, v["v"][0], 500 * dte, rtol=1e-12, maxit=5000, pattern=7)
    u = dev(torch, v["v"][0])
    code, its, rel = ctx.be_pcg_solve(u, 500 * dte, pc=1, rtol=1e-10, maxit=100, x0=dev(torch, x_ref))
    assert code == R.RKL_OK and its[0] <= 1


def test_host_pointers_match_device(oracle_mod, R, torch_cuda):
    """The same calls with host (numpy) arrays: staged by the library, same results."""
    O, torch = oracle_mod, torch_cuda
    dims = (16, 12, 24)
    c = synth.conduction_case(*dims, seed=3)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], dims[1], dims[2])
    dte = ctx.set_conduction(c["T"], c["bhat"], c["n"])
    dte_o, _ = O.gershgorin_dt(g, S, W)
    assert dte == pytest.approx(dte_o, rel=1e-13)
    Fu = np.empty(g.N)
    ctx.apply_F(c["T"], Fu)
    check_F(O, g, S, W, c["T"], Fu.reshape(g.shape))
    u = c["T"].copy()
    s = ctx.rkl2_superstep(u, 300 * dte, dte)
    assert rel_l2(u, O.rkl2_superstep(g, S, W, c["T"], 300 * dte, s)) <= 1e-12
    u = c["T"].copy()
    code, its, rel = ctx.be_pcg_solve(u, 300 * dte, pc=2, block=(4, 4, 4), rtol=0.0, maxit=9)
    x, *_ = O.be_pcg(g, S, W, c["T"], 300 * dte, pc=2, block=(4, 4, 4), fixed_iters=9)
    assert rel_l2(u, x) <= 1e-12


def test_host_staging_grows_across_calls(oracle_mod, R, torch_cuda):
    """Host-pointer calls whose staging needs grow from call to call (N, then 5N for the
    coefficients, then 2N): every argument keeps a valid staged copy."""
    O = oracle_mod
    dims = (24, 16, 32)
    c = synth.conduction_case(*dims, seed=4)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dte_o, _ = O.gershgorin_dt(g, S, W)
    ctx = R.Context(c["rf"], dims[1], dims[2])
    with pytest.raises(R.RklError):
        ctx.rkl2_superstep(c["T"].copy(), 1.0, 1.0)  # before set_coeffs: state error
    dte = ctx.set_conduction(c["T"], c["bhat"], c["n"])
    assert dte == pytest.approx(dte_o, rel=1e-13)
    u = c["T"].copy()
    ctx.rkl2_superstep(u, 50 * dte, dte, s=12)
    assert rel_l2(u, O.rkl2_superstep(g, S, W, c["T"], 50 * dte, 12)) <= 1e-12
    dte = ctx.set_conduction(c["T"], c["bhat"], c["n"])
    Fu = np.empty(g.N)
    ctx.apply_F(c["T"], Fu)
    check_F(O, g, S, W, c["T"], Fu.reshape(g.shape))
    ctx.close()


def test_error_paths(R, torch_cuda):
    """Argument and state errors come back as codes; bad data is flagged, never trapped."""
    torch = torch_cuda
    c = synth.conduction_case(8, 6, 8, seed=1)
    ctx = R.Context(c["rf"], 6, 8)
    u = dev(torch, c["T"])
    with pytest.raises(R.RklError) as e:
        ctx.rkl2_superstep(u, 1.0, 1.0)
    assert e.value.code == R.RKL_ESTATE
    bad = c["T"].copy()
    bad[0, 0, 3] = np.nan
    with pytest.raises(R.RklError) as e:
        ctx.set_conduction(dev(torch, bad), dev(torch, c["bhat"]), dev(torch, c["n"]))
    assert e.value.code == R.RKL_ENONFINITE
    neg = c["n"].copy()
    neg[1, 2, 3] = -1.0
    with pytest.raises(R.RklError) as e:
        ctx.set_conduction(dev(torch, c["T"]), dev(torch, c["bhat"]), dev(torch, neg))
    assert e.value.code == R.RKL_ENONFINITE
    dte = ctx.set_conduction(dev(torch, c["T"]), dev(torch, c["bhat"]), dev(torch, c["n"]))
    for kw in ({"s": 1}, {"dt": -1.0}):
        with pytest.raises(R.RklError) as e:
            args = dict(dt=10 * dte, dt_exp=dte)
            args.update(kw)
            ctx.rkl2_superstep(u, **args)
        assert e.value.code == R.RKL_EINVAL
    with pytest.raises(R.RklError) as e:
        ctx.be_pcg_solve(u, 10 * dte, pc=2, block=(3, 3, 3))
    assert e.value.code == R.RKL_EINVAL
    code, its, rel = ctx.be_pcg_solve(u, 1e4 * dte, pc=1, rtol=1e-14, maxit=2)
    assert code == R.RKL_ENOTCONV and its == [2]
    nanu = dev(torch, bad)
    code, its, rel = ctx.be_pcg_solve(nanu, 10 * dte, pc=1, rtol=1e-10, maxit=50)
    assert code == R.RKL_EBREAKDOWN
    with pytest.raises(R.RklError) as e:
        R.Context(c["rf"][::-1].copy(), 6, 8)
    assert e.value.code == R.RKL_EINVAL
    assert R.rkl2_stage_count(100.0) == 20 and R.rkl2_stage_count(100.0, R.RKL_FORCE_ODD) == 21
    ctx.close()


def test_beta_tcut_operator(oracle_mod, R, torch_cuda):
    """RKL_BETA_TCUT: kappa0 T^{5/2} (T / 5e5 K)^{5/2} below 5e5 K (Sec. 4.1); the seeded
    case dips below 5e5 K near r = 1, so the factor is exercised."""
    O = oracle_mod
    dims = (64, 16, 32)
    c = synth.conduction_case(*dims, seed=3)
    assert (c["T"] < 5e5).sum() > 50
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True)
    ctx = R.Context(c["rf"], dims[1], dims[2])
    dev = lambda a: torch_cuda.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]), beta_tcut=True)
    assert dte == pytest.approx(O.gershgorin_dt(g, S, W)[0], rel=1e-13)
    u = synth.random_field(g.shape, 9)
    Fu = dev(np.zeros(g.N))
    ctx.apply_F(dev(u), Fu)
    F_o = O.apply_F(g, S, W, u)
    assert np.linalg.norm(Fu.cpu().numpy() - F_o.ravel()) <= 1e-12 * np.linalg.norm(F_o)
    ctx.close()


def test_superstep_graph_replay_and_invalidation(oracle_mod, R, torch_cuda):
    """Repeated super-steps replay a captured CUDA graph; a new dt, new coefficients, another
    field or a switch of operator form must not reuse stale launches."""
    O = oracle_mod
    dims = (16, 12, 24)
    c = synth.conduction_case(*dims, seed=5)
    g = O.Grid(c["rf"], dims[1], dims[2])
    dev = lambda a: torch_cuda.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    ctx = R.Context(c["rf"], dims[1], dims[2])
    T2 = c["T"] * (1.0 + 0.1 * synth.random_field(g.shape, 3, 0.0, 1.0))
    cases = [(c["T"], 100.0, False), (c["T"], 100.0, False), (c["T"], 300.0, False), (c["T"], 100.0, False),
             (T2, 100.0, False), (T2, 100.0, True), (c["T"], 100.0, False)]
    u = dev(c["T"])
    other = dev(c["T"])
    for q, (Tc, ratio, flux) in enumerate(cases):
        S, W = O.assemble_conduction(g, Tc, c["bhat"], c["n"], flux_form=flux)
        dte = ctx.set_conduction(dev(Tc), dev(c["bhat"]), dev(c["n"]), flux_form=flux)
        target = other if q == 3 else u  # q == 3: same call on another field
        target.copy_(dev(c["T"]))
        s = ctx.rkl2_superstep(target, ratio * dte, dte)
        ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
        assert np.linalg.norm(target.cpu().numpy() - ref.ravel()) <= 1e-12 * np.linalg.norm(ref), q
    n0 = ctx.kernel_launches
    u.copy_(dev(c["T"]))
    s = ctx.rkl2_superstep(u, 100.0 * dte, dte)
    assert ctx.kernel_launches - n0 == s  # first stage + s - 1 stages, counted on replay too
    ctx.close()


def test_graph_paths_in_a_fresh_process():
    """In a new process no kernel is loaded yet (lazy module loading): set_coeffs followed by
    super-steps and a BE solve must work through the graph paths from the start."""
    import subprocess
    import sys
    import textwrap

    code = textwrap.dedent("""
        import numpy as np, torch
        from paper_1610_01265_gb300 import rklpcg as R, synth
        c = synth.conduction_case(16, 12, 24, seed=1)
        dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64).ravel()).cuda()
        ctx = R.Context(c["rf"], 12, 24)
        dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]))
        outs = []
        for _ in range(3):
            u = dev(c["T"])
            ctx.rkl2_superstep(u, 100 * dte, dte)
            outs.append(u.cpu().numpy())
        assert all(np.array_equal(outs[0], o) for o in outs[1:])
        u = dev(c["T"])
        code, its, rel = ctx.be_pcg_solve(u, 100 * dte, pc=1, rtol=1e-10, maxit=5000)
        assert code == 0 and rel[0] <= 1e-10
        print("fresh ok")
    """)
    import os

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stderr[-2000:]


def test_graphs_interleaved_and_teardown(oracle_mod, R, torch_cuda):
    """Super-steps and graph-driven PCG solves interleaved on one context (each re-capture
    replaces only its own graph), then a new context after closing it."""
    O = oracle_mod
    dims = (16, 12, 24)
    c = synth.conduction_case(*dims, seed=7)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    dev = lambda a: torch_cuda.from_numpy(np.array(a, dtype=np.float64)).cuda().view(-1)  # noqa: E731
    for _ in range(2):
        ctx = R.Context(c["rf"], dims[1], dims[2])
        dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]))
        for kind, ratio in (("rkl", 100.0), ("rkl", 1000.0), ("pcg", 100.0), ("rkl", 100.0), ("pcg", 100.0),
                            ("rkl", 10000.0), ("pcg", 300.0)):
            u = dev(c["T"])
            if kind == "rkl":
                s = ctx.rkl2_superstep(u, ratio * dte, dte)
                ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte, s)
                assert np.linalg.norm(u.cpu().numpy() - ref.ravel()) <= 1e-12 * np.linalg.norm(ref)
            else:
                code, its, rel = ctx.be_pcg_solve(u, ratio * dte, pc=1, rtol=1e-10, maxit=5000)
                x_o, it_o, _, st = O.be_pcg(g, S, W, c["T"], ratio * dte, pc=1, rtol=1e-10)
                assert code == R.RKL_OK and abs(its[0] - it_o) <= 1
        ctx.close()


def test_rsun_cm_scales_the_operator(R, torch_cuda):
    """rkl_grid.rsun_cm is the length unit of the radial faces: doubling it scales areas by
    4, spacings by 2 and volumes by 8, so S by 2, W by 8, F = -W^-1 S u by 1/4 and the
    Gershgorin dt_exp (App. B) by 4."""
    torch = torch_cuda
    c = synth.conduction_case(8, 6, 8, seed=2)
    T, b, n = dev(torch, c["T"]), dev(torch, c["bhat"]), dev(torch, c["n"])
    u = dev(torch, synth.random_field((8, 6, 8), 4))
    out = []
    for rs in (0.0, 2 * 6.96e10):
        with R.Context(c["rf"], 6, 8, rsun_cm=rs) as ctx:
            dte = ctx.set_conduction(T, b, n)
            Fu = torch.empty_like(u)
            ctx.apply_F(u, Fu)
            out.append((dte, host(Fu)))
    assert out[1][0] == pytest.approx(4 * out[0][0], rel=1e-13)
    assert rel_l2(4 * out[1][1], out[0][1]) <= 1e-13
    with pytest.raises(R.RklError) as e:
        R.Context(c["rf"], 6, 8, rsun_cm=-1.0)
    assert e.value.code == R.RKL_EINVAL
