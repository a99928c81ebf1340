"""The allocation-free super-step (for callers that cannot call cudaMalloc because another
component owns all device memory or because allocation would stall their time loop) gives
the same result as the context path rkl_create + set_coeffs + rkl2_superstep, and as the
CPU oracle, on calls in a row that share its static scratch: a call at the largest grid
the scratch holds, then a smaller ragged grid over the previous call's contents (with
beta_Tcut and a fixed stage count).  Kept in a file collected last."""
import numpy as np
import pytest

import oracle as O
from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

# (dims, seed, dt/dt_exp, beta_Tcut, s): the first two fill the whole scratch
# (65536 cells), the third is smaller and ragged (not a multiple of any tile) and runs
# 29 stages, more than the 24 that Eq. 5 gives for 150 dt_exp (stable up to 217)
CALLS = (((32, 32, 64), 1, 100.0, False, 0),
         ((32, 32, 64), 2, 1000.0, False, 0),
         ((12, 20, 40), 3, 150.0, True, 29))


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_noalloc_superstep_matches_context_path_and_oracle():
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    B.build()
    assert torch.cuda.is_available()
    for dims, seed, ratio, btc, s_fix in CALLS:
        nr, nth, nph = dims
        c = synth.conduction_case(nr, nth, nph, seed=seed)
        dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda()  # noqa: E731
        T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
        with R.Context(c["rf"], nth, nph) as ctx:
            dte = ctx.set_conduction(T, b, n, beta_tcut=btc)
            u_ref = T.clone()
            s_ref = ctx.rkl2_superstep(u_ref, ratio * dte, dte, s=s_fix)
            torch.cuda.synchronize()
        u = T.clone()
        s, dte2 = R.rkl2_superstep_noalloc(c["rf"], nth, nph, T, b, n, u, ratio * dte, beta_tcut=btc, s=s_fix)
        torch.cuda.synchronize()
        assert s == s_ref
        if s_fix:
            assert s == s_fix
        assert dte2 == pytest.approx(dte, rel=1e-13)
        got = u.cpu().numpy()
        assert _rel(got, u_ref.cpu().numpy()) <= 1e-12
        # directly against the oracle on the same inputs
        g = O.Grid(c["rf"], nth, nph)
        S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=btc)
        dte_o, _ = O.gershgorin_dt(g, S, W)
        assert dte2 == pytest.approx(dte_o, rel=1e-13)
        ref = O.rkl2_superstep(g, S, W, c["T"], ratio * dte2, s)
        assert _rel(got.reshape(ref.shape), ref) <= 1e-12


def test_noalloc_rejects_what_it_cannot_hold():
    import torch

    from paper_1610_01265_gb300 import rklpcg as R

    c = synth.conduction_case(4, 4, 8, seed=1)
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda()  # noqa: E731
    T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
    # a grid beyond the static scratch (64 x 64 x 32 = 131072 cells): refused up front
    big = torch.ones(3 * 64 * 64 * 32, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RklError) as e:
        R.rkl2_superstep_noalloc(synth.r_faces(64), 64, 32, big, big, big, big.clone(), 1.0)
    assert e.value.code == R.RKL_EINVAL
    # host arrays would need device staging buffers: refused
    with pytest.raises(R.RklError) as e:
        R.rkl2_superstep_noalloc(c["rf"], 4, 8, c["T"], c["bhat"], c["n"], c["T"].copy(), 1.0)
    assert e.value.code == R.RKL_EINVAL
    # a valid call still works after the refusals
    u = T.clone()
    s, dte = R.rkl2_superstep_noalloc(c["rf"], 4, 8, T, b, n, u, 1.0)
    torch.cuda.synchronize()
    assert s == R.rkl2_stage_count(1.0 / dte) and bool(torch.isfinite(u).all())
