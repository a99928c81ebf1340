"""The allocation-free super-step (for callers that cannot call cudaMalloc because another
component owns all device memory or because allocation would stall their time loop) gives
the same result as the context path rkl_create + set_coeffs + rkl2_superstep, on two calls
in a row that share its static scratch.  Kept in a file collected last."""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_noalloc_superstep_matches_context_path():
    import torch

    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg as R

    B.build()
    assert torch.cuda.is_available()
    dims = (32, 32, 64)
    # two calls in a row with different inputs: the second reuses the first's scratch
    for seed, ratio in ((1, 100.0), (2, 1000.0)):
        c = synth.conduction_case(*dims, seed=seed)
        dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda()  # noqa: E731
        T, b, n = dev(c["T"]), dev(c["bhat"]), dev(c["n"])
        with R.Context(c["rf"], dims[1], dims[2]) as ctx:
            dte = ctx.set_conduction(T, b, n)
            u_ref = T.clone()
            s_ref = ctx.rkl2_superstep(u_ref, ratio * dte, dte)
            torch.cuda.synchronize()
        u = T.clone()
        s, dte2 = R.rkl2_superstep_noalloc(c["rf"], dims[1], dims[2], T, b, n, u, ratio * dte)
        torch.cuda.synchronize()
        assert s == s_ref
        assert dte2 == pytest.approx(dte, rel=1e-13)
        assert _rel(u.cpu().numpy(), u_ref.cpu().numpy()) <= 1e-12


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
