"""Training objective of the learned predictor in float64 (NumPy): loss,
gradient by backpropagation, and one Adam step.  The learned predictor is an
extension of the method (the paper has none).  Test infrastructure: only the
tests, the smoke check and the benchmark's CPU baseline use this module.

Network (same as the C oracle's inference): x = prev * 2^-23 (channels u, v),
a1 = conv(x, w1) + b1, h1 = relu(a1), a2 = conv(h1, w2) + b2, h2 = relu(a2),
y = conv(h2, w3) + b3, every conv 3x3 'same' with zero padding:
    conv(x, w)[co][i][j] = sum over (ci, ky, kx) of w[co][ci][ky][kx] * x[ci][i+ky-1][j+kx-1].
Objective over n pairs (prev, next): d = clamp((next - prev) * 2^-23, -2, 2),
loss = mean over (pair, component, i, j) of (y - d)^2.
The codec and the GPU trainer run the network at the parameters rounded to
bfloat16; net_gradients() does the same and differentiates through the
rounding as through the identity.
"""
from __future__ import annotations

import numpy as np

C = 32
# (cout, cin) of the three layers; layout w1 b1 w2 b2 w3 b3, w[co][ci][ky][kx]
LAYERS = [(C, 2), (C, C), (2, C)]
N_PARAMS = sum(co * ci * 9 + co for co, ci in LAYERS)


def bf16_round(p):
    """float32 values rounded to bfloat16 (round to nearest even), as float64."""
    b = np.asarray(p, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta):
    """Parameter vector -> [(w, b)] per layer (views into theta)."""
    out, o = [], 0
    for co, ci in LAYERS:
        w = theta[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    return out


def _pad(x):
    n, c, H, W = x.shape
    xp = np.zeros((n, c, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    return xp


def conv(x, w, b=None):
    """x [n][cin][H][W] -> [n][cout][H][W]."""
    n, _, H, W = x.shape
    xp = _pad(x)
    out = np.zeros((n, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv_input_grad(g, w):
    """d(sum g * conv(x, w)) / dx: gx[n][ci][i][j] = sum over (co, ky, kx) of
    w[co][ci][ky][kx] * g[n][co][i-ky+1][j-kx+1] (zero outside)."""
    n, _, H, W = g.shape
    gp = _pad(g)
    out = np.zeros((n, w.shape[1], H, W))
    for ky in range(3):
        for kx in range(3):
            # g[i - ky + 1] sits at padded row i - ky + 2
            out += np.einsum("oc,nohw->nchw", w[:, :, ky, kx], gp[:, :, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W])
    return out


def conv_weight_grad(g, x):
    """d(sum g * conv(x, w)) / dw and / db."""
    _, _, H, W = x.shape
    xp = _pad(x)
    gw = np.zeros((g.shape[1], x.shape[1], 3, 3))
    for ky in range(3):
        for kx in range(3):
            gw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", g, xp[:, :, ky:ky + H, kx:kx + W])
    return gw, g.sum(axis=(0, 2, 3))


def inputs(prev, nxt):
    """(x, d) [n][2][H][W] float64 from int32 pairs [n][H][W][2]."""
    p = np.asarray(prev, np.int64)
    q = np.asarray(nxt, np.int64)
    if p.ndim == 3:
        p, q = p[None], q[None]
    x = np.moveaxis(p.astype(np.float64) * 2.0 ** -23, 3, 1)
    d = np.clip(np.moveaxis((q - p).astype(np.float64) * 2.0 ** -23, 3, 1), -2.0, 2.0)
    return x, d


def loss_and_grad(theta, x, d):
    """float64 loss and gradient at the parameter vector theta (no rounding)."""
    (w1, b1), (w2, b2), (w3, b3) = unpack(np.asarray(theta, np.float64))
    h1 = np.maximum(conv(x, w1, b1), 0.0)
    h2 = np.maximum(conv(h1, w2, b2), 0.0)
    y = conv(h2, w3, b3)
    m = y.size
    e = y - d
    loss = float((e * e).sum() / m)
    gy = 2.0 * e / m
    gw3, gb3 = conv_weight_grad(gy, h2)
    gh2 = conv_input_grad(gy, w3) * (h2 > 0)
    gw2, gb2 = conv_weight_grad(gh2, h1)
    gh1 = conv_input_grad(gh2, w2) * (h1 > 0)
    gw1, gb1 = conv_weight_grad(gh1, x)
    g = np.concatenate([gw1.ravel(), gb1, gw2.ravel(), gb2, gw3.ravel(), gb3])
    return loss, g


def forward(theta, x):
    (w1, b1), (w2, b2), (w3, b3) = unpack(np.asarray(theta, np.float64))
    return conv(np.maximum(conv(np.maximum(conv(x, w1, b1), 0.0), w2, b2), 0.0), w3, b3)


def net_gradients(params, prev, nxt):
    """(loss, gradient) at float32 params rounded to bfloat16, over the int32
    pairs prev -> nxt [n][H][W][2]."""
    x, d = inputs(prev, nxt)
    return loss_and_grad(bf16_round(params), x, d)


def adam_step(P, m, v, g, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t counts from 1); returns (P, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return P - lr * mh / (np.sqrt(vh) + eps), m, v
