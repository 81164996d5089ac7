"""Pins of the training oracle of the learned predictor (an extension: the
paper has no learned predictor): the backpropagated gradient against central
finite differences, the convolution adjoints by the dot-product identity, the
zero-last-layer closed form, the first Adam step's closed form, bfloat16
rounding on hand-picked values, and the float64 forward pass against the C
oracle's float32 inference."""
import numpy as np

import oracle
from oracle import net_train as nt


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, nt.N_PARAMS)


def _pairs(seed, n=2, H=5, W=6):
    rng = np.random.default_rng(seed)
    prev = rng.integers(-(1 << 23), 1 << 23, (n, H, W, 2)).astype(np.int32)
    nxt = (prev + rng.integers(-(1 << 20), 1 << 20, prev.shape)).astype(np.int32)
    return prev, nxt


def test_param_count_and_layout():
    assert nt.N_PARAMS == oracle.net_params() == 10434
    th = np.arange(nt.N_PARAMS, dtype=np.float64)
    (w1, b1), (w2, b2), (w3, b3) = nt.unpack(th)
    assert w1.shape == (32, 2, 3, 3) and w1[0, 1, 2, 0] == 1 * 9 + 2 * 3
    assert b1[0] == 576 and w2[0, 0, 0, 0] == 608 and b3[-1] == nt.N_PARAMS - 1
    assert w3.shape == (2, 32, 3, 3)


def test_gradient_matches_central_differences():
    prev, nxt = _pairs(1)
    x, d = nt.inputs(prev, nxt)
    th = _theta(2)
    loss, g = nt.loss_and_grad(th, x, d)
    rng = np.random.default_rng(3)
    # indices in every parameter group (w1 b1 w2 b2 w3 b3)
    bounds = np.cumsum([0, 576, 32, 9216, 32, 576, 2])
    idx = np.concatenate([rng.integers(bounds[k], bounds[k + 1], 8) for k in range(6)])
    h = 1e-6
    scale = np.abs(g).max()
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (nt.loss_and_grad(tp, x, d)[0] - nt.loss_and_grad(tm, x, d)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * scale + 1e-6 * abs(g[k]), (k, fd, g[k])


def test_conv_adjoints():
    """<conv(x, w), g> = <x, conv_input_grad(g, w)> = <w, conv_weight_grad(g, x)>."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 3, 7, 5))
    w = rng.normal(size=(4, 3, 3, 3))
    g = rng.normal(size=(2, 4, 7, 5))
    lhs = (nt.conv(x, w) * g).sum()
    assert np.isclose(lhs, (x * nt.conv_input_grad(g, w)).sum(), rtol=1e-12)
    gw, gb = nt.conv_weight_grad(g, x)
    assert np.isclose(lhs, (w * gw).sum(), rtol=1e-12)
    assert np.allclose(gb, g.sum(axis=(0, 2, 3)))
    # a single tap moves the input by one cell: w = delta at (ky, kx) = (0, 2)
    wd = np.zeros((1, 1, 3, 3))
    wd[0, 0, 0, 2] = 1.0
    xs = rng.normal(size=(1, 1, 6, 6))
    out = nt.conv(xs, wd)
    assert np.allclose(out[0, 0, 1:, :-1], xs[0, 0, :-1, 1:])
    assert np.allclose(out[0, 0, 0, :], 0) and np.allclose(out[0, 0, :, -1], 0)


def test_zero_last_layer_closed_form():
    prev, nxt = _pairs(5)
    x, d = nt.inputs(prev, nxt)
    th = _theta(6)
    th[-(2 * 32 * 9 + 2):] = 0.0
    loss, g = nt.loss_and_grad(th, x, d)
    assert np.isclose(loss, (d * d).mean(), rtol=1e-14)
    assert not g[:576 + 32 + 9216 + 32].any()
    m = d.size
    assert np.allclose(g[-2:], -2.0 * d.sum(axis=(0, 2, 3)) / m, rtol=1e-12)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(7)
    P = rng.normal(size=50)
    g = rng.normal(size=50)
    z = np.zeros(50)
    P1, m1, v1 = nt.adam_step(P, z, z, g, 1e-3, 1)
    assert np.allclose(P1, P - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_bf16_round_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -20],
                 np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 1.0 + 2.0 ** -7])
    assert np.array_equal(nt.bf16_round(v), want)


def test_forward_matches_c_oracle_inference():
    """The float64 forward pass at bfloat16 parameters against the C oracle's
    float32 fixed-order inference (float32 rounding apart)."""
    rng = np.random.default_rng(8)
    P = rng.normal(0.0, 0.2, nt.N_PARAMS).astype(np.float32)
    bits = (nt.bf16_round(P).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    prev = rng.integers(-(1 << 23), 1 << 23, (9, 11, 2)).astype(np.int32)
    x, _ = nt.inputs(prev, prev)
    y64 = nt.forward(nt.bf16_round(P), x)[0]
    y32 = oracle.net_forward(bits, prev)
    assert np.allclose(y32, y64, rtol=1e-5, atol=1e-5 * np.abs(y64).max())
