"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.  Integer work (fixed point,
face predicates, bounds, codes, reconstruction, bytes) must be bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth

pytestmark = pytest.mark.gpu


def _dev(uv):
    import torch
    return torch.from_numpy(np.ascontiguousarray(uv)).to("cuda:0")


def compare(uv, eb, pred="lorenzo", eb_mode="rel", block=16, stride=2, dx=1.0, dy=1.0, dt=1.0,
            host_input=False, model=None):
    src = uv if host_input else _dev(uv)
    blob, st, g = cpt.compress(src, eb, eb_mode=eb_mode, pred=pred, block=block, stride=stride,
                               dx=dx, dy=dy, dt=dt, debug=True, model=model)
    r = oracle.compress(uv, eb, eb_mode=eb_mode, pred=pred, block=block, stride=stride, dx=dx, dy=dy, dt=dt,
                        model=model)
    assert st["scale_log2"] == r["stats"]["k"] and st["eps_int"] == r["stats"]["eps_int"]
    assert (g["q"] == r["q"]).all()
    assert (g["mask"] == r["mask"]).all()
    assert (g["xi"] == r["xi"]).all()
    assert (g["qxi"] == r["qxi"]).all()
    nz = r["qxi"] > 0
    assert (g["sym"][nz] == r["qd"][nz]).all()
    if pred in ("mop", "learned_mop"):
        assert (g["modes"] == r["modes"]).all()
    assert (g["qhat"] == r["qhat"]).all()
    assert blob == r["bytes"]
    assert st["verify_mismatch_slice"] == 0 and st["verify_mismatch_slab"] == 0
    assert st["linf"] <= st["eps"] or st["eps_int"] == 0
    # the verification's L-inf error: the largest exact |x_hat - x|, rounded
    # once to double (a double difference of two floats is that rounding)
    err = np.abs(np.ldexp(r["qhat"].astype(np.float64), -r["stats"]["k"]) - np.asarray(uv, np.float64))
    assert st["linf"] == (err.max() if err.size else 0.0)
    assert st["crossed_faces"] == r["stats"]["crossed_faces"]
    assert st["n_ld"] == r["stats"]["n_ld"] and st["n_qd"] == r["stats"]["n_qd"]
    return blob, st, g, r


@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
def test_vortex64(pred):
    uv, eb = synth.workload("vortex64")
    compare(uv, eb, pred)


@pytest.mark.parametrize("shape", [(37, 45, 5), (33, 70, 3), (100, 40, 4), (2, 2, 3), (5, 3, 1)])
@pytest.mark.parametrize("pred", ["lorenzo", "mop"])
def test_ragged_shapes(shape, pred):
    H, W, T = shape
    uv = synth.vortex_sum(H, W, T, seed=7 + H, n_vortex=3)
    compare(uv, 5e-3, pred)


def test_stream_without_copy_matches_bytes():
    """The zero-copy stream object holds the same bytes; its buffer goes back
    to the library and is reused by the next call."""
    uv, eb = synth.workload("vortex64")
    d = _dev(uv)
    ref, _, _ = cpt.compress(d, eb, pred="mop")
    for _ in range(3):
        blob, st, _ = cpt.compress(d, eb, pred="mop", copy=False)
        assert len(blob) == len(ref) == st["out_bytes"]
        assert bytes(blob) == ref
        assert blob.numpy().tobytes() == ref
        del blob


def test_sl_nonunit_spacing_and_host_input():
    uv = synth.vortex_sum(48, 40, 6, seed=3, drift=2.5)
    compare(uv, 2e-2, "sl", dx=0.5, dy=2.0, dt=3.0, host_input=True)


@pytest.mark.parametrize("spacing", [(0.5, 0.25, 1.0), (0.125, 0.125, 1.0), (1.0, 1.0, 2.0)])
def test_sl_power_of_two_spacing(spacing):
    """Other spacings of the semi-Lagrangian back-trace: CFL numbers that
    are powers of two other than 2^-k, and large ones that make the
    back-trace take Euler substeps."""
    dx, dy, dt = spacing
    uv = synth.vortex_sum(40, 52, 5, seed=9, drift=1.5)
    compare(uv, 1e-2, "sl", dx=dx, dy=dy, dt=dt)
    compare(uv, 1e-2, "mop", dx=dx, dy=dy, dt=dt, block=8)


def test_mop_block8_stride3():
    uv = synth.vortex_sum(50, 61, 5, seed=4)
    compare(uv, 1e-2, "mop", block=8, stride=3)


@pytest.mark.parametrize("seed", range(3))
def test_small_integer_fields_degenerate_sos(seed):
    rng = np.random.default_rng(100 + seed)
    uv = rng.integers(-2, 3, (4, 9, 11, 2)).astype(np.float32)
    compare(uv, 0.4, "lorenzo", eb_mode="abs")
    compare(uv, 0.4, "mop", eb_mode="abs", block=4)


@pytest.mark.parametrize("pred", ["lorenzo", "mop"])
def test_rough_field_interior_items(pred):
    """Integers in -2..2 on a field with interior work items: most vertices
    need the exact face test, so the interior items' queues fill and the
    rest of each item is tested vertex by vertex; masks, codes and bytes
    stay identical to the oracle's."""
    rng = np.random.default_rng(30)
    uv = rng.integers(-2, 3, (3, 70, 130, 2)).astype(np.float32)
    compare(uv, 0.4, pred, eb_mode="abs", block=8)


@pytest.mark.parametrize("shift,noise", [(1.0, 0.0), (1.0, 2e-4), (0.0, 2e-4)])
def test_mop_carried_and_static_patterns(shift, noise):
    """Fields on which the MoP choice is fixed by the predictors' exactness
    (SL in every interior block of a pattern the flow carries, 3DL on a static
    one); small noise breaks the degenerate faces that make the noiseless
    carried field lossless, so the codes and both predictors run."""
    from test_oracle_pins import _pattern_field
    uv = _pattern_field(5, 70, 90, shift=shift)
    uv = uv + np.random.default_rng(12).normal(0.0, noise, uv.shape).astype(np.float32)
    _, st, g, r = compare(uv, 1e-3, "mop")
    if shift:
        assert (g["modes"][1:, 1:-1, 1:-1] == 1).all()
    else:
        assert st["sl_blocks"] < st["blocks"] // 10


def test_invalid_arguments_are_rejected():
    """Inputs outside the method's domain come back as status codes, with no
    stream, and the library stays usable."""
    good = synth.vortex_sum(9, 10, 2, seed=13)
    nan, inf = good.copy(), good.copy()
    nan[1, 4, 5, 0] = np.nan
    inf[0, 0, 0, 1] = -np.inf
    cases = [
        (np.zeros((2, 1, 5, 2), np.float32), 1e-2, {}, cpt.ERR_ARG),      # H < 2
        (np.zeros((2, 5, 1, 2), np.float32), 1e-2, {}, cpt.ERR_ARG),      # W < 2
        (np.zeros((0, 5, 5, 2), np.float32), 1e-2, {}, cpt.ERR_ARG),      # no slice
        (good, -1e-3, {}, cpt.ERR_ARG),                                     # negative bound
        (good, float("inf"), {}, cpt.ERR_ARG),
        (good, float("nan"), {}, cpt.ERR_ARG),
        (nan, 1e-2, {}, cpt.ERR_ARG),                                       # non-finite data
        (inf, 1e-2, {"pred": "sl"}, cpt.ERR_ARG),
        (good, 1e-2, {"block": 40}, cpt.ERR_ARG),                          # block side
        (good, 1e-2, {"pred": "mop", "block": 6}, cpt.ERR_UNSUPPORTED),   # MoP blocks must tile 32
        (good, 1e-2, {"pred": "learned"}, cpt.ERR_ARG),                    # no model
    ]
    for uv, eb, kw, want in cases:
        with pytest.raises(cpt.CptError) as e:
            cpt.compress(_dev(uv), eb, **kw)
        assert e.value.status == want, (uv.shape, eb, kw)
    compare(good, 1e-2, "mop")


def test_zero_and_constant_fields():
    compare(np.zeros((3, 6, 7, 2), np.float32), 1e-2, "mop")
    c = np.ones((3, 6, 7, 2), np.float32) * 0.25
    compare(c, 0.01, "sl", eb_mode="abs")


def test_zero_error_bound_is_lossless():
    uv = synth.vortex_sum(20, 24, 3, seed=5)
    blob, st, g, r = compare(uv, 0.0, "lorenzo", eb_mode="abs")
    assert (g["qhat"] == g["q"]).all() and st["lossless_vertices"] == 20 * 24 * 3


def test_large_bound():
    uv = synth.vortex_sum(30, 30, 4, seed=6)
    compare(uv, 10.0, "lorenzo", eb_mode="abs")


def test_exact_zero_determinants():
    """Small-integer fields make exact zero determinants (M = 0 in Alg. 2) common
    on faces through reconstructed vertices; every such vertex must still be
    encoded exactly as the oracle does."""
    rng = np.random.default_rng(77)
    for _ in range(4):
        uv = rng.integers(-2, 3, (5, 12, 13, 2)).astype(np.float32)
        compare(uv, 0.6, "lorenzo", eb_mode="abs")
        compare(uv, 0.6, "mop", eb_mode="abs", block=4)


# ---------------------------------------------------------------------------
# decompression (the inverse raster loop) through the C ABI
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
@pytest.mark.parametrize("shape", [(64, 64, 8), (37, 45, 5), (2, 2, 3)])
def test_decompress_matches_oracle(pred, shape):
    H, W, T = shape
    uv = synth.vortex_sum(H, W, T, seed=11 + H + W, n_vortex=3)
    blob, st, g = cpt.compress(_dev(uv), 5e-3, pred=pred, debug=True)
    out, qh, dims = cpt.decompress(blob, want_q=True)
    oq, ouv, k = oracle.decompress(blob)
    assert dims == (H, W, T)
    assert (qh == oq).all() and (qh == g["qhat"]).all()
    assert np.array_equal(out.view(np.uint32), ouv.view(np.uint32))
    assert np.abs(out.astype(np.float64) - uv.astype(np.float64)).max() <= st["eps"]


def test_decompress_to_device_tensor():
    import torch
    uv, eb = synth.workload("vortex64")
    blob, _, _ = cpt.compress(_dev(uv), eb, pred="mop")
    dst = torch.empty(uv.shape, dtype=torch.float32, device="cuda:0")
    cpt.decompress(blob, out=dst)
    _, ouv, _ = oracle.decompress(blob)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), ouv.view(np.uint32))


def test_decompress_rejects_malformed_streams():
    uv, eb = synth.workload("vortex64")
    blob, _, _ = cpt.compress(_dev(uv), eb, pred="lorenzo")
    for bad in (b"XXXX" + blob[4:], blob[:50], blob[: len(blob) // 2], blob[:-3]):
        with pytest.raises(cpt.CptError) as e:
            cpt.decompress(bad)
        assert e.value.status == cpt.ERR_CORRUPT
    # a moved sync point of the bound-code stream is caught by the decoder
    b = bytearray(blob)
    off = 96 + 16 + 4 * 25  # header, stream header, at most 25 used codes
    hdr_used = int.from_bytes(b[96 + 8:96 + 12], "little")
    off = 96 + 16 + 4 * hdr_used + 8  # second sync point
    v = int.from_bytes(b[off:off + 8], "little")
    b[off:off + 8] = (v + 1).to_bytes(8, "little")
    with pytest.raises(cpt.CptError) as e:
        cpt.decompress(bytes(b))
    assert e.value.status == cpt.ERR_CORRUPT
    # a verbatim-value count (header offset 80) that disagrees with the codes,
    # with the section resized to match, is caught after the tiled expansion
    n_ld = int.from_bytes(blob[80:88], "little")
    for delta in (-2, 2):
        b = bytearray(blob)
        b[80:88] = (n_ld + delta).to_bytes(8, "little")
        b = b[:len(blob) - 8] if delta < 0 else b + bytes(8)
        with pytest.raises(cpt.CptError) as e:
            cpt.decompress(bytes(b))
        assert e.value.status == cpt.ERR_CORRUPT


def test_oracle_stream_decodes_on_gpu():
    """Bytes written by the oracle decode on the GPU to the oracle's values."""
    uv = synth.vortex_sum(40, 52, 6, seed=8)
    r = oracle.compress(uv, 1e-2, pred="mop", block=8)
    _, qh, _ = cpt.decompress(r["bytes"], want_q=True)
    assert (qh == r["qhat"]).all()


# ---------------------------------------------------------------------------
# trajectories (Sec. III-D, Thm. 2) through the C ABI
# ---------------------------------------------------------------------------
def _oracle_trajs(uv, k=None):
    if k is None:
        k = oracle.scale_exponent(float(np.abs(uv).max()))
    return oracle.trajectories(oracle.to_fixed(uv, k))


def _same_trajs(a, b):
    ta, pa, ba = a
    tb, pb, bb = b
    assert ba == bb == 0
    assert len(ta) == len(tb)
    for x, y in zip(ta, tb):
        assert np.array_equal(x, y)
    for x, y in zip(pa, pb):
        assert np.allclose(x, y, rtol=0, atol=1e-12)


@pytest.mark.parametrize("case", ["vortex64", "ragged", "ints", "linear", "birth", "centre"])
def test_trajectories_match_oracle(case):
    if case == "vortex64":
        uv = synth.vortex_sum()
    elif case == "ragged":
        uv = synth.vortex_sum(37, 45, 5, seed=9, n_vortex=4)
    elif case == "ints":
        uv = np.random.default_rng(3).integers(-2, 3, (4, 9, 11, 2)).astype(np.float32)
    elif case == "linear":
        uv = synth.linear_field(24, 32, 8, 6.3, 1.7, 5.6, 1.45)
    elif case == "birth":
        uv = synth.birth_field(16, 32, 6, 15.5, 7.5, 6.0, 2)
    else:
        uv = synth.centre_field(20, 20, 5, 9.4, 10.7)
    _same_trajs(cpt.extract_trajectories(_dev(uv)), _oracle_trajs(uv))


def test_trajectories_preserved_by_roundtrip():
    """Thm. 2: the decompressed field has the same trajectories, face by face."""
    uv, eb = synth.workload("vortex64")
    blob, st, _ = cpt.compress(_dev(uv), eb, pred="mop")
    out, _, _ = cpt.decompress(blob)
    k = st["scale_log2"]
    t0 = cpt.extract_trajectories(_dev(uv), scale_log2=k)
    t1 = cpt.extract_trajectories(_dev(out), scale_log2=k)
    assert len(t0[0]) == len(t1[0]) > 0
    for x, y in zip(t0[0], t1[0]):
        assert np.array_equal(x, y)
