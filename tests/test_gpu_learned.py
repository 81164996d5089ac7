"""GPU parity of the learned predictor (an extension: the paper has none):
inference bit-exact against the oracle, compression and decompression
bit-exact with the learned and the learned-mixture predictors, gradients of
the GPU trainer against the float64 oracle, the first Adam step, and what
the trained network gains over the method without it."""
import numpy as np
import pytest

import oracle
from oracle import net_train as nt
from paper_2510_25143_gb300 import cpt, synth
from test_gpu_parity import _dev, compare

pytestmark = pytest.mark.gpu

MODEL_BYTES = 4 + 4 * ((nt.N_PARAMS + 1) // 2)  # the model's section of a stream


def bits_of(P):
    return (nt.bf16_round(P).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def random_model(seed, scale):
    return bits_of(np.random.default_rng(seed).normal(0.0, scale, nt.N_PARAMS))


def fixed(uv):
    return oracle.to_fixed(uv, oracle.scale_exponent(float(np.abs(uv).max())))


@pytest.mark.parametrize("shape", [(64, 64), (37, 45), (5, 3), (1, 9)])
def test_net_predict_matches_oracle(shape):
    H, W = shape
    q = fixed(synth.vortex_sum(max(H, 2), max(W, 2), 2, seed=20 + H, n_vortex=3))[1, :H, :W]
    for seed, scale in ((1, 0.2), (2, 0.05)):
        m = random_model(seed, scale)
        assert np.array_equal(cpt.net_predict(m, q), oracle.net_predict(m, q))


@pytest.mark.parametrize("pred", ["learned", "learned_mop"])
@pytest.mark.parametrize("case", ["vortex64", "ragged", "block8"])
def test_learned_compress_matches_oracle(pred, case):
    model = random_model(3, 0.03)
    if case == "vortex64":
        uv, eb = synth.workload("vortex64")
        compare(uv, eb, pred, model=model)
    elif case == "ragged":
        compare(synth.vortex_sum(37, 45, 5, seed=21, n_vortex=3), 5e-3, pred, model=model)
    else:
        compare(synth.vortex_sum(50, 61, 5, seed=22, drift=0.1), 3e-3, pred, block=8, model=model)


@pytest.mark.parametrize("pred", ["learned", "learned_mop"])
def test_learned_decompress_matches_oracle(pred):
    uv = synth.vortex_sum(40, 52, 6, seed=23, drift=0.1)
    model = random_model(4, 0.03)
    blob, st, g = cpt.compress(_dev(uv), 3e-3, pred=pred, model=model, block=8, debug=True)
    out, qh, _ = cpt.decompress(blob, want_q=True)
    oq, ouv, _ = oracle.decompress(blob)
    assert (qh == oq).all() and (qh == g["qhat"]).all()
    assert np.array_equal(out.view(np.uint32), ouv.view(np.uint32))
    assert np.abs(out.astype(np.float64) - uv).max() <= st["eps"]


def _pairs(n=2, H=20, W=24):
    q = fixed(synth.vortex_sum(H, W, n + 1, seed=24, n_vortex=4, drift=0.7))
    return q[:-1], q[1:]


def test_gradients_match_oracle():
    prev, nxt = _pairs()
    P = np.random.default_rng(5).normal(0.0, 0.1, nt.N_PARAMS).astype(np.float32)
    loss, g = cpt.net_gradients(P, prev, nxt)
    lref, gref = nt.net_gradients(P, prev, nxt)
    assert abs(loss - lref) <= 1e-5 * lref
    bounds = np.cumsum([0, 576, 32, 9216, 32, 576, 2])
    for k in range(6):
        a, b = g[bounds[k]:bounds[k + 1]], gref[bounds[k]:bounds[k + 1]]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, k
    # float32 against float64: besides rounding, a pre-activation within
    # rounding of 0 may take the other side of a ReLU, which moves a single
    # position's share of a gradient; the norm-wise error stays small
    assert np.linalg.norm(g - gref) <= 1e-3 * np.linalg.norm(gref)


def test_training_forward_is_the_inference():
    """The trainer's loss at bfloat16 parameters is the loss of the codec's
    own float32 outputs (the oracle's fixed-order inference)."""
    prev, nxt = _pairs(n=1, H=33, W=29)
    m = random_model(6, 0.1)
    P = (m.astype(np.uint32) << 16).view(np.float32)
    loss, _ = cpt.net_gradients(P, prev, nxt)
    y = oracle.net_forward(m, prev[0])
    diff = (nxt[0].astype(np.int64) - prev[0]).astype(np.float32) * np.float32(2.0 ** -23)
    d = np.clip(np.moveaxis(diff, 2, 0), np.float32(-2), np.float32(2))
    e = (y - d).astype(np.float32).astype(np.float64)
    assert abs(loss - float((e * e).mean())) <= 1e-6 * loss


def test_first_adam_step():
    prev, nxt = _pairs()
    m0 = random_model(7, 0.1)
    P0 = (m0.astype(np.uint32) << 16).view(np.float32)
    m1, losses = cpt.train_predictor(prev, nxt, steps=1, lr=1e-3, init=m0)
    l0, g = nt.net_gradients(P0, prev, nxt)
    assert abs(losses[0] - l0) <= 1e-5 * l0
    want = bits_of(P0.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8))
    # where the gradient is clearly away from 0 the step is -lr * sign(g),
    # so the float32 and float64 gradients give the same bfloat16 result
    sure = np.abs(g) > 1e-3 * np.abs(g).max()
    assert sure.mean() > 0.3
    assert np.array_equal(m1[sure], want[sure])
    dead = g == 0  # units that never fire: no step
    assert np.array_equal(m1[dead], m0[dead])


def test_trained_net_gains():
    """Trained on the decompressed slices of one field (plain MoP), the net
    cuts the training loss and improves the compression ratio of the field
    over the untrained net (which predicts the previous slice) and over the
    plain predictors (on this drifting field by about 3.5 %, model section
    excluded)."""
    uv = synth.vortex_sum(128, 128, 12, seed=25, n_vortex=8, drift=0.5)
    eb = 1e-3
    d = _dev(uv)
    blob, st, _ = cpt.compress(d, eb, pred="mop")
    _, qh, _ = cpt.decompress(blob, want_q=True)
    model, losses = cpt.train_predictor(qh[:-1], qh[1:], steps=400, lr=1e-3, seed=1)
    untrained, l0 = cpt.train_predictor(qh[:1], qh[1:2], steps=1, lr=1e-30, seed=1)
    assert losses[-1] < 0.25 * losses[0]
    raw = uv.nbytes
    ratios = {}
    for name, pred, m in (("plain lorenzo", "lorenzo", None), ("plain mop", "mop", None),
                          ("untrained", "learned", untrained), ("learned", "learned", model),
                          ("learned mixture", "learned_mop", model)):
        b, s, _ = cpt.compress(d, eb, pred=pred, model=m)
        assert s["verify_mismatch_slice"] == 0 and s["verify_mismatch_slab"] == 0
        ratios[name] = raw / (len(b) - (MODEL_BYTES if m is not None else 0))
    print("ratios without the model section:", {k: round(v, 3) for k, v in ratios.items()})
    assert ratios["learned"] > 1.2 * ratios["untrained"]
    # over the method without it: both plain predictors at the same bound
    assert ratios["learned"] > 1.02 * max(ratios["plain lorenzo"], ratios["plain mop"])
    assert ratios["learned mixture"] > 1.02 * max(ratios["plain lorenzo"], ratios["plain mop"])
