"""Sec. 6 on the GPU: the damping variants of the super-step against the oracle, and the
amplification factors of Fig. 6 measured with the CUDA path.

Fig. 6 analyses the 1-D constant-coefficient diffusion equation.  With bhat = phi-hat and
uniform coefficients every (r, theta) ring of the grid is exactly that problem: cos(m phi)
and (-1)^k are eigenvectors, so one large step multiplies them by the method's
amplification factor, which the tests compare with e^{lam dt} (exact), 1/(1 - lam dt)
(BE), R_s(lam dt) (RKL2) and 1 + lam dt (explicit Euler)."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg

    B.build()
    return rklpcg


def dev(a):
    import torch

    return torch.from_numpy(np.array(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("scheme,cycles,extra,fe,odd", [
    (0, 1, 0, 0.0, False), (0, 4, 0, 0.0, False), (0, 1, 2, 0.0, False), (0, 10, 0, 0.0, True),
    (0, 1, 0, 0.25, False), (1, 1, 0, 0.0, False), (1, 2, 3, 0.0, False), (1, 3, 1, 0.1, False)])
def test_sts_variants_match_oracle(oracle_mod, R, scheme, cycles, extra, fe, odd):
    O = oracle_mod
    dims = (16, 12, 24)
    c = synth.conduction_case(*dims, seed=5)
    g = O.Grid(c["rf"], dims[1], dims[2])
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"])
    ctx = R.Context(c["rf"], dims[1], dims[2])
    dte = ctx.set_conduction(dev(c["T"]), dev(c["bhat"]), dev(c["n"]))
    dt = 201.37 * dte
    u = dev(c["T"])
    used = ctx.sts_advance(u, dt, dte, scheme=scheme, cycles=cycles, extra_stages=extra, euler_fraction=fe,
                           force_odd=odd)
    # the same composition from oracle steps
    x = c["T"].copy()
    te = fe * dt
    ne = math.ceil(te / dte) if te > 0 else 0
    for _ in range(ne):
        x = O.euler_step(g, S, W, x, te / ne)
    tau = (dt - te) / cycles
    if scheme == 0:
        s = O.rkl2_stages(tau / dte) + extra
        if odd and s % 2 == 0:
            s += 1
        step = O.rkl2_superstep
    else:
        s = O.rkl1_stages(tau / dte) + extra
        step = O.rkl1_superstep
    for _ in range(cycles):
        x = step(g, S, W, x, tau, s)
    assert used == ne + cycles * s
    assert _rel(u.cpu().numpy().reshape(g.shape), x) <= 1e-12
    ctx.close()


def ring_problem(R, nph=64):
    nr, nth = 2, 4
    rf = synth.r_faces(nr)
    one = np.ones((nph, nth, nr))
    ctx = R.Context(rf, nth, nph)
    dte = ctx.set_conduction(dev(1e6 * one), dev(np.stack([0 * one, 0 * one, one])), dev(1e8 * one))
    phi = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    return ctx, dte, phi, one


def factors(ctx, dte, u0, ratio, R, torch):
    """(lam, G_rkl2, G_be) per ring for the eigenvector u0 (shape (nph, nth, nr))."""
    x = dev(u0)
    Fu = torch.empty_like(x)
    ctx.apply_F(x, Fu)
    uu = (u0 * u0).sum(axis=0)
    lam = (Fu.cpu().numpy() * u0).sum(axis=0) / uu
    a = dev(u0)
    s = ctx.rkl2_superstep(a, ratio * dte, dte)
    g_rkl = (a.cpu().numpy() * u0).sum(axis=0) / uu
    b = dev(u0)
    code, its, rel = ctx.be_pcg_solve(b, ratio * dte, pc=R.RKL_PC_JACOBI, rtol=1e-14, maxit=5000)
    assert code == R.RKL_OK
    g_be = (b.cpu().numpy() * u0).sum(axis=0) / uu
    return lam, s, g_rkl, g_be


@pytest.mark.parametrize("ratio", [0.2, 5.0, 50.0, 500.0])
def test_fig6_amplification_factors(R, ratio):
    import torch

    ctx, dte, phi, one = ring_problem(R)
    nph = len(phi)
    w = {}
    for m in list(range(1, nph // 2)) + [nph // 2]:
        u0 = (np.cos(m * phi) if m < nph // 2 else (-1.0) ** np.arange(nph))[:, None, None] * one
        lam, s, g_rkl, g_be = factors(ctx, dte, u0, ratio, R, torch)
        z = lam * ratio * dte
        w1 = 4.0 / (s * s + s - 2)
        bs = (s * s + s - 2) / (2.0 * s * (s + 1))
        Rs = (1 - bs) + bs * eval_legendre(s, 1 + w1 * z)
        assert np.allclose(g_rkl, Rs, rtol=0, atol=1e-10)
        assert np.allclose(g_be, 1.0 / (1.0 - z), rtol=1e-9, atol=1e-12)
        w[m] = (z, g_rkl, g_be)
    exact = {m: np.exp(v[0]) for m, v in w.items()}
    if ratio < 1:
        # explicit Euler is stable below the limit, 1 + z in [-1, 1]
        assert all(np.all(np.abs(1 + v[0]) <= 1 + 1e-12) for v in w.values())
    # small wave modes (|z| < 0.05): second-order RKL2 is closer to exp(z) than BE
    for m, (z, gr, gb) in w.items():
        sel = np.abs(z) < 0.05
        assert np.all(np.abs(gr - exact[m])[sel] <= np.abs(gb - exact[m])[sel])
    if ratio >= 50:
        # BE (L-stable) nearly removes the highest mode; RKL2 keeps a large factor
        top = w[nph // 2]
        assert np.all(np.abs(top[1]) > 0.25) and np.all(np.abs(top[1]) > 2 * np.abs(top[2]))
        # mid-spectrum RKL2 amplification near a_s ~ 1/2, far above the exact factor
        mid = w[nph // 4]
        assert np.all(np.abs(mid[1] - 0.5) < 0.15) and np.all(exact[nph // 4] < 0.2 * mid[1])
    ctx.close()


def test_sec6_remedies_damp_the_highest_mode(R):
    """Sub-cycling RKL2 (10 cycles) or an explicit-Euler prefix over a quarter of the step
    damp the highest mode far more than one RKL2 super-step (Sec. 6); the measured factors
    equal the products of the closed forms (R_s per cycle, (1 + z h)^n per Euler step)."""
    import torch

    ctx, dte, phi, one = ring_problem(R)
    u0 = ((-1.0) ** np.arange(len(phi)))[:, None, None] * one
    uu = (u0 * u0).sum(axis=0)
    x = dev(u0)
    Fu = torch.empty_like(x)
    ctx.apply_F(x, Fu)
    lam = (Fu.cpu().numpy() * u0).sum(axis=0) / uu
    ratio = 500.5  # not a whole number of Euler limits: the last sub-step is shorter
    z = lam * ratio * dte

    def closed(s, zz):
        w1 = 4.0 / (s * s + s - 2)
        bs = (s * s + s - 2) / (2.0 * s * (s + 1))
        return (1 - bs) + bs * eval_legendre(s, 1 + w1 * zz)

    def measure(run):
        a = dev(u0)
        used = run(a)
        return (a.cpu().numpy() * u0).sum(axis=0) / uu, used

    g_one, s1 = measure(lambda a: ctx.rkl2_superstep(a, ratio * dte, dte))
    assert np.allclose(g_one, closed(s1, z), atol=1e-10, rtol=0)
    g_sub, n_sub = measure(lambda a: ctx.sts_advance(a, ratio * dte, dte, cycles=10))
    s10 = n_sub // 10
    assert np.allclose(g_sub, closed(s10, z / 10) ** 10, atol=1e-10, rtol=0)
    g_eul, n_eul = measure(lambda a: ctx.sts_advance(a, ratio * dte, dte, euler_fraction=0.25))
    ne = math.ceil(0.25 * ratio)
    se = n_eul - ne
    h = 0.25 * ratio * dte / ne
    assert np.allclose(g_eul, (1 + lam * h) ** ne * closed(se, 0.75 * z), atol=1e-10, rtol=0)
    assert np.abs(g_sub).max() < 0.05 * np.abs(g_one).max()
    assert np.abs(g_eul).max() < 0.2 * np.abs(g_one).max()
    ctx.close()
