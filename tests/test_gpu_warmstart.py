"""Parity of the learned initial guess (CUDA, BF16 tensor cores) with the oracle.

Both sides round to BF16 at the same points (features, weights, stored activations,
dy, back-propagated gradients), so they compute the same function; they differ only by
FP32 (GPU) versus FP64 (oracle) accumulation.  A sum of K = 864 products accumulated in
FP32 carries a relative error of about sqrt(K) 2^-24 ~ 2e-6; that moves a stored BF16
value to the neighbouring BF16 number (a change of 2^-8 relative) with a probability of
about 2e-6 / 2^-8 ~ 5e-4 per value.  Each flipped input perturbs an output by ~2^-8 /
sqrt(K) of its size, so the expected relative L2 difference after three rounded layers is
~1e-4.  The tests allow 2e-3 for the forward pass (a factor of about 20) and 1e-2 for the
parameter gradients, which pass through three more rounded tensors (dy, dz3, dz2, dz1)
and through sums over all cells that cancel.
"""
import numpy as np
import pytest

from paper_1610_01265_gb300 import synth

pytestmark = pytest.mark.gpu

FWD_TOL = 2e-3
GRAD_TOL = 1e-2


@pytest.fixture(scope="module")
def env():
    import torch

    from oracle import warmstart as OW
    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import warmstart as W

    B.build()
    return torch, OW, W


def _params(OW, seed):
    """He-uniform weights (oracle's SplitMix64) with random non-zero biases."""
    p = OW.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for (ci, co), (wo, bo) in zip(OW.LAYERS, OW.layer_offsets()):
        p[bo:bo + co] = rng.uniform(-0.1, 0.1, co).astype(np.float32)
    return p


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _feats_grid(OW, shape, seed, dt=37.0):
    nph, nth, nr = shape
    c = synth.conduction_case(nr, nth, nph, seed=seed)
    return c, OW.features(c["T"], c["bhat"], dt, rounding=False)


def test_initial_parameters_bitwise(env):
    torch, OW, W = env
    for seed in (0, 7, 2**40 + 3):
        net = W.Net(seed)
        assert np.array_equal(net.params(), OW.init_params(seed))
        net.close()


# shapes are (nph, nth, nr); r extents that are multiples of 128 run the 32-channel layers on
# the tcgen05 convolution (one 128-cell r line per UMMA tile: odd theta counts, a second r
# segment whose halo comes from the first, phi chunks and wrap), the others on mma.sync
@pytest.mark.parametrize("shape,nbox,periodic", [((10, 9, 37), 1, True), ((3, 5, 20), 3, False),
                                                 ((2, 4, 64), 2, True), ((1, 1, 1), 1, True),
                                                 ((6, 5, 128), 1, True), ((3, 3, 256), 2, False),
                                                 ((40, 2, 128), 1, True)])
def test_forward_parity(env, shape, nbox, periodic):
    torch, OW, W = env
    params = _params(OW, 3)
    feats = np.stack([_feats_grid(OW, shape, 10 + b)[1] for b in range(nbox)])  # (nbox, 5, ...)
    net = W.Net(0)
    net.set_params(params)
    f_dev = torch.from_numpy(np.ascontiguousarray(feats.transpose(1, 0, 2, 3, 4)).astype(np.float32)).cuda()
    y = torch.empty(f_dev[0].numel(), dtype=torch.float32, device="cuda")
    box = (shape[2], shape[1], shape[0])
    net.forward(box, f_dev.view(-1), y, nbox=nbox, periodic=periodic)
    net.check()
    y_o, _ = OW.forward(params, OW.bf16(feats.astype(np.float32)), periodic=periodic)
    y_g = y.cpu().numpy().reshape(y_o.shape)
    assert _rel(y_g, y_o.numpy()) <= FWD_TOL
    assert np.max(np.abs(y_g - y_o.numpy())) <= 10 * FWD_TOL * np.max(np.abs(y_o.numpy()))
    net.close()


@pytest.mark.parametrize("periodic,weighted,shape", [(True, False, (4, 6, 40)), (False, True, (4, 6, 40)),
                                                      (True, True, (5, 3, 128))])
def test_loss_gradient_parity(env, periodic, weighted, shape):
    torch, OW, W = env
    nbox = 2
    params = _params(OW, 5)
    feats = np.stack([_feats_grid(OW, shape, 20 + b)[1] for b in range(nbox)])
    target = synth.random_field((nbox,) + shape, 31).astype(np.float32)
    weight = synth.random_field((nbox,) + shape, 32, 0.0, 1.0).astype(np.float32) if weighted else None
    net = W.Net(0)
    net.set_params(params)
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda().view(-1)  # noqa: E731
    f_dev = dev(feats.transpose(1, 0, 2, 3, 4).astype(np.float32))
    loss = net.loss_grad((shape[2], shape[1], shape[0]), f_dev, dev(target), dev(weight), nbox=nbox,
                         periodic=periodic)
    g = net.grads()
    loss_o, g_o = OW.loss_grad(params, OW.bf16(feats.astype(np.float32)), target, weight, periodic=periodic)
    assert loss == pytest.approx(loss_o, rel=FWD_TOL)
    for (ci, co), (wo, bo) in zip(OW.LAYERS, OW.layer_offsets()):
        assert _rel(g[wo:bo], g_o[wo:bo]) <= GRAD_TOL, ("weights", ci, co)
        assert _rel(g[bo:bo + co], g_o[bo:bo + co]) <= GRAD_TOL, ("bias", ci, co)
    # the reductions run in a fixed order: a second pass is bitwise identical
    net.loss_grad((shape[2], shape[1], shape[0]), f_dev, dev(target), dev(weight), nbox=nbox, periodic=periodic)
    assert np.array_equal(net.grads(), g)
    net.close()


def test_adam_parity(env):
    torch, OW, W = env
    p0 = _params(OW, 9)
    rng = np.random.default_rng(41)
    net = W.Net(0)
    net.set_params(p0)
    p_o = p0.astype(np.float64)
    m = np.zeros_like(p_o)
    v = np.zeros_like(p_o)
    lr = 3e-3
    for step in range(1, 4):
        g = (rng.standard_normal(p0.size) * 10.0 ** rng.uniform(-4, 0, p0.size)).astype(np.float32)
        net.set_grads(g)
        net.adam(lr)
        p_o, m, v = OW.adam(p_o, g, m, v, step, lr)
        p_g = net.params().astype(np.float64)
        assert np.max(np.abs(p_g - p_o)) <= 1e-5 * lr + 2e-7 * np.max(np.abs(p_o))
    net.close()


def test_features_and_guess_parity(env):
    torch, OW, W = env
    shape = (12, 10, 24)
    c = synth.conduction_case(shape[2], shape[1], shape[0], seed=4)
    dt = 123.4
    params = _params(OW, 11)
    net = W.Net(0)
    net.set_params(params)
    T = torch.from_numpy(c["T"].ravel()).cuda()
    b = torch.from_numpy(c["bhat"].ravel()).cuda()
    N = T.numel()
    feat = torch.empty(5 * N, dtype=torch.float32, device="cuda")
    net.features(shape, T, b, dt, feat)
    f_o = OW.features(c["T"], c["bhat"], dt, rounding=False)
    f_g = feat.cpu().numpy().reshape(f_o.shape).astype(np.float64)
    assert np.array_equal(f_g[:4], f_o[:4])
    assert np.max(np.abs(f_g[4] - f_o[4])) <= 2.0**-22 * abs(f_o[4].flat[0])
    x0 = torch.empty_like(T)
    scale = 2.5e3
    net.guess(shape, T, b, dt, scale, x0)
    net.check()
    y_o, _ = OW.forward(params, OW.features(c["T"], c["bhat"], dt), periodic=True)
    x_o = c["T"] + scale * y_o[0].numpy()
    dx = x0.cpu().numpy().reshape(shape) - c["T"]
    assert _rel(dx, x_o - c["T"]) <= FWD_TOL
    net.close()


def test_training_reduces_the_loss(env):
    torch, OW, W = env
    shape = (6, 8, 32)
    feats = _feats_grid(OW, shape, 50)[1]
    # a smooth target the net can represent: a fixed linear map of the features
    target = (0.3 * feats[0] - 0.2 * feats[1] + 0.1).astype(np.float32)
    net = W.Net(1)
    f_dev = torch.from_numpy(feats.astype(np.float32).ravel()).cuda()
    t_dev = torch.from_numpy(target.ravel()).cuda()
    box = (shape[2], shape[1], shape[0])
    l0 = net.loss_grad(box, f_dev, t_dev)
    for _ in range(60):
        net.loss_grad(box, f_dev, t_dev, want_loss=False)
        net.adam(3e-3)
    l1 = net.loss_grad(box, f_dev, t_dev)
    assert l1 < 0.2 * l0
    net.close()


def test_fullsize_guess_sampled(env):
    """The guess at 128 x 192 x 384 (the size the benchmark runs) at sampled cells,
    each recomputed by the oracle from its own 9^3 window of inputs."""
    torch, OW, W = env
    nph, nth, nr = 384, 192, 128
    c = synth.conduction_case(nr, nth, nph, seed=1)
    params = _params(OW, 13)
    net = W.Net(0)
    net.set_params(params)
    T = torch.from_numpy(c["T"].ravel()).cuda()
    b = torch.from_numpy(c["bhat"].ravel()).cuda()
    x0 = torch.empty_like(T)
    dt, scale = 55.0, 1e4
    net.guess((nph, nth, nr), T, b, dt, scale, x0)
    net.check()
    x = x0.cpu().numpy().reshape(nph, nth, nr)
    feats = OW.features(c["T"], c["bhat"], dt)
    rng = np.random.default_rng(3)
    cells = [(0, 0, 0), (nph - 1, nth - 1, nr - 1), (0, nth // 2, 31), (nph - 1, 0, 32), (191, 1, nr - 2)]
    cells += [tuple(int(v) for v in (rng.integers(nph), rng.integers(nth), rng.integers(nr))) for _ in range(40)]
    y_o = OW.forward_at(params, feats, cells, periodic=True)
    y_g = np.array([(x[k, j, i] - c["T"][k, j, i]) / scale for k, j, i in cells])
    assert _rel(y_g, y_o) <= FWD_TOL
    net.close()


def test_study_small(env):
    """The learned-guess study on a small grid: every solve converges from every guess to
    the same solution, and the report carries iterations and times for each guess."""
    import bench

    out = bench.warmstart_study(seed=2, dims=(16, 24, 48), n_steps=8, n_train=4, epochs=2, pcs=(1, 2))
    assert out["solution_spread_rel"] <= 1e-6
    for pc in ("jacobi", "bilu0-8x8x8"):
        t = out["test"][pc]
        assert set(t) == set(bench.WS_GUESSES)
        for g, r in t.items():
            assert r["iters_mean"] > 0 and r["ms_mean"] > 0
        assert t["no_change"]["init_err_mean"] < t["zero"]["init_err_mean"]
    assert out["train"]["optimizer_steps"] == 8
