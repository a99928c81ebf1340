"""FP64 CPU oracle of the learned initial guess for the backward-Euler + PCG solve.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  Plain PyTorch CPU float64;
``torch.nn.functional.conv3d`` serves as the convolution primitive, everything else is
written out here.

The paper's solvers take any initial guess x0 (the PCG of Fig. 1 starts from it); this
module defines the map that supplies one: a 4-layer 3-D convolutional net

    a1 = relu(conv(a0; W1, b1))    5 -> 32 channels
    a2 = relu(conv(a1; W2, b2))   32 -> 32
    a3 = relu(conv(a2; W3, b3))   32 -> 32
    y  =      conv(a3; W4, b4)    32 -> 1

with 3x3x3 kernels (cross-correlation, taps ordered (dphi, dtheta, dr) with dr fastest),
zero outside the grid in r and theta and periodic in phi on a whole grid ("periodic"),
zero outside on every face for a detached box.  Input channels a0: (T - 1e6 K)/1e6 K,
bhat_r, bhat_theta, bhat_phi, log10(dt / 1 s); the output y is Delta T in units chosen by
the caller, and the guess is x0 = T + scale * y.

The net runs with BF16 weights and activations and FP32 accumulation.  The oracle
rounds at the same points (``rounding=True``) so that it computes the same function:
features, weights, the stored activations a1..a3, the output gradient dy and the
back-propagated gradients dz1..dz3 are rounded to BF16 (round to nearest, ties to
even); biases, the output y and the parameter gradients stay in full precision.  ``rounding=False`` gives the
plain FP64 net (used to pin the gradient code against autograd and finite
differences).

Parameters are one float32 vector: for each layer W (Cout, Cin, 3, 3, 3) flattened in
that order, then b (Cout).  Initial weights are He-uniform, (2u - 1) sqrt(6/(27 Cin)),
with u = SplitMix64(seed, counter) >> 11 times 2^-53 and counter = the weight's index in
the parameter vector (Steele, Lea & Flood 2014); biases start at zero.  The optimiser is
Adam (Kingma & Ba 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and bias correction.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

LAYERS = ((5, 32), (32, 32), (32, 32), (32, 1))
NTAP = 27
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8
T_REF = 1e6
RECEPTIVE_RADIUS = len(LAYERS)  # each 3x3x3 layer widens the dependence by one cell


def num_params() -> int:
    return sum(co * ci * NTAP + co for ci, co in LAYERS)


def layer_offsets():
    """(weight offset, bias offset) of every layer in the parameter vector."""
    out, off = [], 0
    for ci, co in LAYERS:
        out.append((off, off + co * ci * NTAP))
        off += co * ci * NTAP + co
    return out


# ---------------------------------------------------------------- random numbers
_GOLDEN = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def splitmix64(seed: int, counters) -> np.ndarray:
    """SplitMix64 output for state seed + (counter + 1) * golden (one step per counter)."""
    out = []
    for c in counters:
        z = (seed + _GOLDEN * (int(c) + 1)) & _MASK
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return np.array(out, dtype=np.uint64)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights from SplitMix64, zero biases, as float32."""
    p = np.zeros(num_params(), dtype=np.float32)
    for (ci, co), (wo, _) in zip(LAYERS, layer_offsets()):
        nw = co * ci * NTAP
        z = splitmix64(seed, range(wo, wo + nw))
        u = (z >> np.uint64(11)).astype(np.float64) * 2.0**-53
        p[wo:wo + nw] = ((2.0 * u - 1.0) * np.sqrt(6.0 / (ci * NTAP))).astype(np.float32)
    return p


# ---------------------------------------------------------------- rounding
def fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via FP32 as the hardware path does."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    bits = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64).reshape(np.shape(x))


def _bf16_t(t: torch.Tensor, on: bool) -> torch.Tensor:
    return torch.from_numpy(bf16(t.numpy())) if on else t


# ---------------------------------------------------------------- the net
def unpack(params, rounding: bool = True):
    """[(W (co, ci, 3, 3, 3), b (co,))] as float64 tensors; W rounded to BF16 if asked."""
    p = np.asarray(params).astype(np.float64)  # float32 parameters convert exactly
    out = []
    for (ci, co), (wo, bo) in zip(LAYERS, layer_offsets()):
        w = p[wo:bo].reshape(co, ci, 3, 3, 3)
        out.append((torch.from_numpy(bf16(w) if rounding else w.copy()), torch.from_numpy(p[bo:bo + co].copy())))
    return out


def features(T, bhat, dt, rounding: bool = True) -> np.ndarray:
    """Input channels (5, nph, nth, nr) of one grid."""
    T = np.asarray(T, dtype=np.float64)
    f = np.empty((5,) + T.shape)
    f[0] = fp32((T - T_REF) * (1.0 / T_REF))
    f[1:4] = fp32(bhat)
    f[4] = fp32(np.log10(dt))
    return bf16(f) if rounding else f


def _pad(x: torch.Tensor, periodic: bool) -> torch.Tensor:
    """One ghost layer on every side of (B, C, nph, nth, nr): phi wraps when periodic."""
    if periodic:
        x = torch.cat([x[:, :, -1:], x, x[:, :, :1]], dim=2)
        return F.pad(x, (1, 1, 1, 1, 0, 0))
    return F.pad(x, (1, 1, 1, 1, 1, 1))


def conv(x: torch.Tensor, w: torch.Tensor, b, periodic: bool) -> torch.Tensor:
    """out[co, x] = b[co] + sum_ci sum_taps w[co, ci, tap] in[ci, x + offset(tap)]."""
    return F.conv3d(_pad(x, periodic), w, b)


def conv_adjoint(d: torch.Tensor, w: torch.Tensor, periodic: bool) -> torch.Tensor:
    """Transpose of conv(., w, 0): the same padding with w[co, ci] reflected in every axis."""
    wt = torch.flip(w, dims=(2, 3, 4)).transpose(0, 1).contiguous()
    return F.conv3d(_pad(d, periodic), wt, None)


def conv_weight_grad(d: torch.Tensor, a: torch.Tensor, periodic: bool) -> torch.Tensor:
    """dW[co, ci, tap] = sum_{box, x} d[co, x] a[ci, x + offset(tap)]."""
    ap = _pad(a, periodic)
    nph, nth, nr = d.shape[2:]
    g = torch.zeros(d.shape[1], a.shape[1], 3, 3, 3, dtype=torch.float64)
    for kp in range(3):
        for kt in range(3):
            for kr in range(3):
                sh = ap[:, :, kp:kp + nph, kt:kt + nth, kr:kr + nr]
                g[:, :, kp, kt, kr] = torch.einsum("bopqr,bipqr->oi", d, sh)
    return g


def forward(params, feats, periodic: bool = True, rounding: bool = True):
    """Net output y (B, nph, nth, nr) and the activations [a0, a1, a2, a3] of (B, 5, ...) input."""
    layers = unpack(params, rounding)
    a = torch.from_numpy(np.asarray(feats, dtype=np.float64))
    if a.dim() == 4:
        a = a.unsqueeze(0)
    acts = [a]
    for l, (w, b) in enumerate(layers):
        z = conv(acts[-1], w, b, periodic)
        if l < len(layers) - 1:
            acts.append(_bf16_t(torch.relu(z), rounding))
        else:
            y = z[:, 0]
    return y, acts


def loss_grad(params, feats, target, weight=None, periodic: bool = True, rounding: bool = True):
    """Weighted mean squared error L = sum w (y - t)^2 / sum w and its gradient (float64)."""
    layers = unpack(params, rounding)
    y, acts = forward(params, feats, periodic, rounding)
    t = torch.from_numpy(np.asarray(target, dtype=np.float64).reshape(y.shape))
    w = torch.ones_like(y) if weight is None else torch.from_numpy(np.asarray(weight, dtype=np.float64).reshape(y.shape))
    wsum = float(w.sum())
    e = y - t
    loss = float((w * e * e).sum()) / wsum
    d = _bf16_t((2.0 / wsum) * w * e, rounding)
    d = d.unsqueeze(1)  # (B, 1, ...): gradient of L with respect to the pre-activation of layer 4
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        w_l = layers[l][0]
        grads[l] = (conv_weight_grad(d, acts[l], periodic), d.sum(dim=(0, 2, 3, 4)))
        if l > 0:
            g = conv_adjoint(d, w_l, periodic) * (acts[l] > 0)
            d = _bf16_t(g, rounding)
    flat = np.concatenate([np.concatenate([gw.numpy().ravel(), gb.numpy().ravel()]) for gw, gb in grads])
    return loss, flat


def adam(params, grads, m, v, step: int, lr: float):
    """One Adam step (step = 1, 2, ...): returns (params, m, v) in float64."""
    p = np.asarray(params, dtype=np.float64)
    g = np.asarray(grads, dtype=np.float64)
    m = ADAM_B1 * np.asarray(m, dtype=np.float64) + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * np.asarray(v, dtype=np.float64) + (1.0 - ADAM_B2) * g * g
    mhat = m / (1.0 - ADAM_B1**step)
    vhat = v / (1.0 - ADAM_B2**step)
    return p - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def guess(params, T, bhat, dt, scale, periodic: bool = True):
    """Initial guess x0 = T + scale * y on one grid."""
    y, _ = forward(params, features(T, bhat, dt), periodic)
    return np.asarray(T, dtype=np.float64) + scale * y[0].numpy()


def forward_at(params, feats, cells, periodic: bool = True):
    """y at selected cells (k, j, i) of one grid, each from its own window of radius 4.

    Hidden activations outside the grid are zero in the full evaluation, so a window that
    reaches past the r or theta ends masks them back to zero after every layer."""
    feats = np.asarray(feats, dtype=np.float64)
    nph, nth, nr = feats.shape[1:]
    layers = unpack(params, True)
    R = RECEPTIVE_RADIUS
    out = []
    for k, j, i in cells:
        kk = np.arange(k - R, k + R + 1)
        jj = np.arange(j - R, j + R + 1)
        ii = np.arange(i - R, i + R + 1)
        inside_k = np.ones(kk.size, bool) if periodic else (kk >= 0) & (kk < nph)
        inside = inside_k[:, None, None] & ((jj >= 0) & (jj < nth))[None, :, None] & ((ii >= 0) & (ii < nr))[None, None, :]
        win = feats[:, np.mod(kk, nph)[:, None, None], np.clip(jj, 0, nth - 1)[None, :, None],
                    np.clip(ii, 0, nr - 1)[None, None, :]] * inside
        a = torch.from_numpy(win).unsqueeze(0)
        mask = torch.from_numpy(inside.astype(np.float64))
        for l, (w, b) in enumerate(layers):
            z = F.conv3d(F.pad(a, (1, 1, 1, 1, 1, 1)), w, b)
            if l < len(layers) - 1:
                a = _bf16_t(torch.relu(z), True) * mask
            else:
                a = z
        out.append(float(a[0, 0, R, R, R]))
    return np.array(out)
