"""Pins of the learned-initial-guess oracle against facts fixed outside it: published
SplitMix64 outputs, hand-worked BF16 roundings and PyTorch's own BF16 conversion, a
brute-force convolution loop, autograd and finite differences for the gradient, closed
forms of Adam, translation equivariance in phi and the receptive field of four layers."""
import itertools

import numpy as np
import pytest
import torch

from oracle import warmstart as WS


def test_splitmix64_published_vector():
    # the first outputs of SplitMix64 started from state 0
    z = WS.splitmix64(0, [0, 1, 2])
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_bf16_rounding_cases_and_library():
    one = 1.0
    cases = {
        one: one,
        one + 2.0**-8: one,  # halfway, ties to the even neighbour 1.0
        one + 3 * 2.0**-8: one + 2.0**-6,  # halfway between odd 1+2^-7 and even 1+2^-6
        one + 2.0**-7: one + 2.0**-7,  # exactly representable
        one + 2.0**-8 + 2.0**-20: one + 2.0**-7,  # just above halfway
        -(3.0 + 2.0**-7): -(3.0),  # 3 + 2^-7 is halfway at exponent 1, even is 3
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert WS.bf16(np.array([x]))[0] == want, x
    x = np.random.default_rng(3).standard_normal(20000) * 10.0 ** np.random.default_rng(4).uniform(-20, 20, 20000)
    lib = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(WS.bf16(x), lib)


def _conv_loop(x, w, b, periodic):
    """Brute-force direct definition: out[co,k,j,i] = b + sum w[co,ci,dk+1,dj+1,di+1] x[ci,k+dk,j+dj,i+di]."""
    B, ci_n, nph, nth, nr = x.shape
    co_n = w.shape[0]
    out = np.zeros((B, co_n, nph, nth, nr))
    for bb, co, k, j, i in itertools.product(range(B), range(co_n), range(nph), range(nth), range(nr)):
        s = b[co] if b is not None else 0.0
        for ci, dk, dj, di in itertools.product(range(ci_n), (-1, 0, 1), (-1, 0, 1), (-1, 0, 1)):
            kk, jj, ii = k + dk, j + dj, i + di
            if not (0 <= jj < nth and 0 <= ii < nr):
                continue
            if not 0 <= kk < nph:
                if not periodic:
                    continue
                kk %= nph
            s += w[co, ci, dk + 1, dj + 1, di + 1] * x[bb, ci, kk, jj, ii]
        out[bb, co, k, j, i] = s
    return out


@pytest.mark.parametrize("periodic", [True, False])
def test_conv_matches_direct_loop(periodic):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 3, 4, 3, 5))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    got = WS.conv(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), periodic).numpy()
    assert np.allclose(got, _conv_loop(x, w, b, periodic), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("periodic", [True, False])
def test_adjoint_and_weight_grad_against_loop(periodic):
    rng = np.random.default_rng(6)
    x = rng.standard_normal((1, 2, 3, 4, 5))
    d = rng.standard_normal((1, 3, 3, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    # <conv(x), d> = <x, conv^T(d)> with conv^T from the loop applied to unit vectors
    Ax = _conv_loop(x, w, None, periodic)
    ATd = WS.conv_adjoint(torch.from_numpy(d), torch.from_numpy(w), periodic).numpy()
    assert np.sum(Ax * d) == pytest.approx(np.sum(x * ATd), rel=1e-12)
    # weight gradient of <conv(x; w), d> by perturbing single weights in the loop
    g = WS.conv_weight_grad(torch.from_numpy(d), torch.from_numpy(x), periodic).numpy()
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 0, 2, 2, 2), (0, 1, 1, 1, 1)]:
        e = np.zeros_like(w)
        e[idx] = 1.0
        assert g[idx] == pytest.approx(np.sum(_conv_loop(x, e, None, periodic) * d), rel=1e-12, abs=1e-12)


def _small_case(seed, shape=(6, 5, 7), nbox=1):
    rng = np.random.default_rng(seed)
    feats = rng.uniform(-1, 1, (nbox, 5) + shape)
    target = rng.standard_normal((nbox,) + shape)
    params = WS.init_params(seed)
    return params, feats, target


@pytest.mark.parametrize("periodic", [True, False])
def test_gradient_matches_autograd(periodic):
    params, feats, target = _small_case(7, nbox=2)
    weight = np.random.default_rng(8).uniform(0, 1, target.shape)
    loss, g = WS.loss_grad(params, feats, target, weight, periodic=periodic, rounding=False)
    # autograd through the plain net
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.from_numpy(feats)
    off = WS.layer_offsets()
    a = x
    for l, ((ci, co), (wo, bo)) in enumerate(zip(WS.LAYERS, off)):
        w = p[wo:bo].view(co, ci, 3, 3, 3)
        b = p[bo:bo + co]
        a = WS.conv(a, w, b, periodic)
        if l < 3:
            a = torch.relu(a)
    wt = torch.from_numpy(weight)
    L = (wt * (a[:, 0] - torch.from_numpy(target)) ** 2).sum() / wt.sum()
    L.backward()
    assert loss == pytest.approx(float(L.detach()), rel=1e-13)
    assert np.allclose(g, p.grad.numpy(), rtol=1e-10, atol=1e-14 * np.max(np.abs(g)))


def test_gradient_matches_finite_differences():
    params, feats, target = _small_case(9)
    _, g = WS.loss_grad(params, feats, target, rounding=False)
    p64 = params.astype(np.float64)
    rng = np.random.default_rng(10)
    off = WS.layer_offsets()
    picks = [off[3][1], off[0][1] + 3, off[2][0] + 100] + list(rng.integers(0, WS.num_params(), 5))
    for q in picks:
        h = 1e-6 * max(1.0, abs(p64[q]))
        lp = WS.loss_grad(_perturb(p64, q, h), feats, target, rounding=False)[0]
        lm = WS.loss_grad(_perturb(p64, q, -h), feats, target, rounding=False)[0]
        fd = (lp - lm) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.max(np.abs(g)))


def _perturb(p, q, h):
    out = p.copy()
    out[q] += h
    return out


def test_adam_closed_forms():
    rng = np.random.default_rng(11)
    p = rng.standard_normal(50)
    g = np.where(rng.uniform(size=50) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-1, 3, 50)  # |g| >> eps
    m = np.zeros(50)
    v = np.zeros(50)
    lr = 1e-3
    # a constant gradient moves every parameter by lr * sign(g) on every step
    q = p.copy()
    for step in range(1, 6):
        q, m, v = WS.adam(q, g, m, v, step, lr)
        assert np.allclose(q, p - step * lr * np.sign(g), rtol=0, atol=1e-9 * step)
    # a zero gradient with zero moments leaves the parameters where they are
    q2, _, _ = WS.adam(p, np.zeros(50), np.zeros(50), np.zeros(50), 1, lr)
    assert np.array_equal(q2, p)


def test_init_params_distribution():
    p = WS.init_params(123)
    assert p.dtype == np.float32 and p.size == WS.num_params() == 5 * 32 * 27 + 32 + 2 * (32 * 32 * 27 + 32) + 32 * 27 + 1
    for (ci, co), (wo, bo) in zip(WS.LAYERS, WS.layer_offsets()):
        w = p[wo:bo].astype(np.float64)
        a = np.sqrt(6.0 / (27 * ci))
        assert np.all(np.abs(w) <= a) and np.all(p[bo:bo + co] == 0)
        if w.size > 1000:
            assert abs(w.mean()) < 0.05 * a
            assert np.var(w) == pytest.approx(a * a / 3, rel=0.06)
    assert np.array_equal(p, WS.init_params(123))
    assert not np.array_equal(p, WS.init_params(124))


def test_features_values():
    T = np.array([[[1e6, 2e6, 5e5]]])
    b = np.zeros((3,) + T.shape)
    b[0] = 1.0
    f = WS.features(T, b, 10.0)
    assert f.shape == (5,) + T.shape
    assert np.array_equal(f[0].ravel(), [0.0, 1.0, -0.5])
    assert np.all(f[1] == 1.0) and np.all(f[2] == 0.0) and np.all(f[4] == 1.0)


def test_constant_net_guess():
    # all weights zero, output bias c: y = c everywhere, x0 = T + scale c
    p = np.zeros(WS.num_params(), dtype=np.float32)
    p[WS.layer_offsets()[3][1]] = 0.25
    T = 1e6 * (1 + np.random.default_rng(12).uniform(0, 1, (4, 3, 5)))
    b = np.random.default_rng(13).standard_normal((3, 4, 3, 5))
    x0 = WS.guess(p, T, b, 3.0, scale=8.0)
    assert np.array_equal(x0, T + 2.0)


def test_phi_roll_equivariance_and_receptive_field():
    params, feats, _ = _small_case(14, shape=(12, 11, 10))
    y, _ = WS.forward(params, feats[0], periodic=True)
    y_roll, _ = WS.forward(params, np.roll(feats[0], 3, axis=1), periodic=True)
    assert np.allclose(np.roll(y.numpy(), 3, axis=1), y_roll.numpy(), rtol=1e-13, atol=1e-13)
    # a change at one cell reaches exactly the cells within 4 in every index
    f2 = feats[0].copy()
    f2[:, 6, 5, 5] += 0.5
    y2, _ = WS.forward(params, f2, periodic=True)
    diff = np.abs(y2.numpy()[0] - y.numpy()[0]) > 0
    k, j, i = np.nonzero(diff)
    assert k.min() >= 2 and k.max() <= 10 and j.min() >= 1 and j.max() <= 9 and i.min() >= 1 and i.max() <= 9
    assert diff[6, 5, 5]


@pytest.mark.parametrize("periodic", [True, False])
def test_windowed_evaluation_matches_full(periodic):
    params, feats, _ = _small_case(15, shape=(9, 7, 12))
    y, _ = WS.forward(params, feats[0], periodic=periodic)
    cells = [(0, 0, 0), (8, 6, 11), (4, 3, 6), (1, 6, 0), (7, 0, 10)]
    got = WS.forward_at(params, feats[0], cells, periodic=periodic)
    want = np.array([y[0, k, j, i].item() for k, j, i in cells])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
