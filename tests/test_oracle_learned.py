"""Oracle pins for the learned predictor (an extension of the method: the
paper has no learned predictor).  The C oracle's net is checked against an
independent NumPy float64 restatement of the same network, against the zero
network (prediction = previous reconstruction), against its 7 x 7 receptive
field with zero padding, and by the compress/decompress round trip."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import synth

C = 32


def bf16_bits(x):
    """float32 -> bfloat16 bits, round to nearest even (the storage of the weights)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def bf16_val(h):
    return (np.asarray(h, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def split(model):
    m = bf16_val(model)
    sizes = [C * 2 * 9, C, C * C * 9, C, 2 * C * 9, 2]
    parts, o = [], 0
    for n in sizes:
        parts.append(m[o:o + n])
        o += n
    w1, b1, w2, b2, w3, b3 = parts
    return w1.reshape(C, 2, 3, 3), b1, w2.reshape(C, C, 3, 3), b2, w3.reshape(2, C, 3, 3), b3


def conv_ref(x, w, b, relu):
    """float64 'same' 3x3 convolution with zero padding: x [Cin][H][W]."""
    cin, H, W = x.shape
    xp = np.zeros((cin, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], xp[:, ky:ky + H, kx:kx + W])
    out += b[:, None, None]
    return np.maximum(out, 0) if relu else out


def net_ref(model, prev):
    w1, b1, w2, b2, w3, b3 = split(model)
    x = np.moveaxis(prev.astype(np.float64), 2, 0) * 2.0 ** -23
    return conv_ref(conv_ref(conv_ref(x, w1, b1, True), w2, b2, True), w3, b3, False)


def random_model(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    n = oracle.net_params()
    return bf16_bits(rng.normal(0, scale, n).astype(np.float32))


def test_param_count():
    assert oracle.net_params() == 2 * C * 9 + C + C * C * 9 + C + 2 * C * 9 + 2 == 10434


def test_forward_matches_float64_restatement():
    rng = np.random.default_rng(5)
    prev = rng.integers(-(1 << 22), 1 << 22, (13, 11, 2)).astype(np.int32)
    model = random_model(1)
    y = oracle.net_forward(model, prev).astype(np.float64)
    ref = net_ref(model, prev)
    # float32 accumulation of up to 289 terms against float64: relative 1e-4 of the magnitudes
    scale = np.abs(ref).max() + 1e-6
    assert np.abs(y - ref).max() <= 1e-4 * scale


def test_zero_net_predicts_previous_slice():
    prev = np.random.default_rng(2).integers(-(1 << 23), 1 << 23, (9, 7, 2)).astype(np.int32)
    model = np.zeros(oracle.net_params(), np.uint16)
    assert (oracle.net_predict(model, prev) == prev).all()


def test_receptive_field_and_zero_padding():
    # zero biases, positive weights: a single input impulse reaches exactly the
    # 7 x 7 neighbourhood (three 3 x 3 layers), clipped by the field boundary
    n = oracle.net_params()
    model = bf16_bits(np.full(n, 0.01, np.float32))
    w1, b1, w2, b2, w3, b3 = [np.zeros(0)] * 6
    m = bf16_val(model).astype(np.float32)
    sizes = np.cumsum([0, C * 2 * 9, C, C * C * 9, C, 2 * C * 9, 2])
    for a, b in ((sizes[1], sizes[2]), (sizes[3], sizes[4]), (sizes[5], sizes[6])):
        m[a:b] = 0.0  # biases
    model = bf16_bits(m)
    for (pi, pj) in ((0, 0), (6, 5), (11, 12)):
        prev = np.zeros((12, 13, 2), np.int32)
        prev[pi, pj, 0] = 1 << 22
        y = oracle.net_forward(model, prev)
        nz = np.argwhere(np.abs(y[0]) > 0)
        ii, jj = np.meshgrid(np.arange(12), np.arange(13), indexing="ij")
        want = (np.abs(ii - pi) <= 3) & (np.abs(jj - pj) <= 3)
        got = np.zeros((12, 13), bool)
        got[nz[:, 0], nz[:, 1]] = True
        assert (got == want).all()


def test_prediction_rounding_and_clamp():
    # a network whose output is its bias: y = b3 exactly (other parameters 0)
    n = oracle.net_params()
    m = np.zeros(n, np.float32)
    m[-2], m[-1] = 0.5, -3.0          # u: +0.5 * 2^23; v: clamped to -2 * 2^23
    prev = np.full((4, 5, 2), 1000, np.int32)
    p = oracle.net_predict(bf16_bits(m), prev)
    assert (p[..., 0] == 1000 + (1 << 22)).all()
    assert (p[..., 1] == 1000 - (1 << 24)).all()


@pytest.mark.parametrize("scale", [0.0, 0.05])
def test_learned_roundtrip_and_invariants(scale):
    uv = synth.vortex_sum(20, 24, 5, seed=9, n_vortex=3)
    model = random_model(3, scale) if scale else np.zeros(oracle.net_params(), np.uint16)
    r = oracle.compress(uv, 1e-2, pred="learned", model=model)
    qhat, uvh, k = oracle.decompress(r["bytes"])
    assert (qhat == r["qhat"]).all()
    eps = r["stats"]["eps"]
    assert np.abs(uvh.astype(np.float64) - uv).max() <= max(eps, 0.5 * 2.0 ** -k)
    mask_h = oracle.face_masks(qhat) if hasattr(oracle, "face_masks") else None
    if mask_h is not None:
        assert (mask_h == r["mask"]).all()


def test_learned_needs_a_model():
    uv = synth.vortex_sum(8, 8, 2, seed=1, n_vortex=1)
    with pytest.raises(RuntimeError):
        oracle.compress(uv, 1e-2, pred="learned")


# ---------------------------------------------------------------------------
# the learned mixture: per block (Sec. VI's selection) 3DL or the net
# ---------------------------------------------------------------------------
def _lorenzo(Q, t, i, j, c):
    """3DL from the reconstruction (zero outside the field), Eq. of Sec. V-B."""
    def at(tt, ii, jj):
        return int(Q[tt, ii, jj, c]) if tt >= 0 and ii >= 0 and jj >= 0 else 0
    return (at(t, i - 1, j) + at(t, i, j - 1) + at(t - 1, i, j) - at(t, i - 1, j - 1) - at(t - 1, i - 1, j)
            - at(t - 1, i, j - 1) + at(t - 1, i - 1, j - 1))


def test_learned_mop_codes_follow_block_modes():
    """Every predicted vertex is quantised against the prediction its block's
    mode names: the net's (mode 1) or 3DL's (mode 0).  The zero net
    (prediction = previous slice) on a slowly drifting field wins some
    blocks and loses others."""
    uv = synth.vortex_sum(24, 20, 4, seed=12, n_vortex=3, drift=0.1)
    model = np.zeros(oracle.net_params(), np.uint16)
    model[:576] = random_model(5, 0.02)[:576]  # hidden layers do not reach the output
    B = 8
    r = oracle.compress(uv, 3e-3, pred="learned_mop", model=model, block=B)
    qh, q, qxi, qd, modes = r["qhat"], r["q"], r["qxi"], r["qd"], r["modes"]
    T, H, W, _ = q.shape
    assert modes[1:].any() and not modes[1:].all()
    for t in range(1, T):
        npred = oracle.net_predict(model, qh[t - 1])
        for i in range(H):
            for j in range(W):
                code = int(qxi[t, i, j])
                if code == 0:
                    continue
                for c in range(2):
                    p = int(npred[i, j, c]) if modes[t, i // B, j // B] else _lorenzo(qh, t, i, j, c)
                    sym, rec = oracle.quantize(int(q[t, i, j, c]), p, 1 << (code - 1))
                    assert sym == qd[t, i, j, c] and rec == qh[t, i, j, c]


def test_learned_mop_with_useless_net_is_lorenzo():
    """A net whose predictions are noise of large amplitude loses every
    block: the codes are plain 3DL's."""
    uv = synth.vortex_sum(20, 24, 5, seed=13, n_vortex=3)
    r = oracle.compress(uv, 1e-2, pred="learned_mop", model=random_model(15, 0.5))
    l = oracle.compress(uv, 1e-2, pred="lorenzo")
    assert not r["modes"].any()
    assert (r["qd"] == l["qd"]).all() and (r["qhat"] == l["qhat"]).all() and (r["qxi"] == l["qxi"]).all()


def test_learned_mop_roundtrip():
    uv = synth.vortex_sum(33, 30, 5, seed=14, n_vortex=4)
    r = oracle.compress(uv, 5e-3, pred="learned_mop", model=random_model(6, 0.02))
    qhat, uvh, k = oracle.decompress(r["bytes"])
    assert (qhat == r["qhat"]).all()
    assert np.abs(uvh.astype(np.float64) - uv).max() <= r["stats"]["eps"]
    assert (oracle.face_masks(qhat) == r["mask"]).all()
