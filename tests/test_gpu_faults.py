"""Failure detection of the encoder pipeline's bounded waits, without a GPU
fault: a host-side injection makes one wave item never run, so the waits of
the items that depend on it run out; the kernel sets its status word and
stops, the call returns ERR_TIMEOUT, and the device stays usable."""
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth
from test_gpu_parity import _dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pred", ["lorenzo", "mop"])
def test_stalled_wave_times_out_and_the_library_recovers(pred):
    uv = synth.vortex_sum(64, 64, 6, seed=3)
    d = _dev(uv)
    cpt.inject_wave_stall(0, timeout_s=0.2)  # wave(0, 0): every other item depends on it
    with pytest.raises(cpt.CptError) as e:
        cpt.compress(d, 1e-2, pred=pred)
    assert e.value.status == cpt.ERR_TIMEOUT
    # the injection is consumed; the next call completes and matches the oracle
    blob, st, _ = cpt.compress(d, 1e-2, pred=pred)
    assert blob == oracle.compress(uv, 1e-2, pred=pred)["bytes"]
    assert st["verify_mismatch_slice"] == 0 and st["verify_mismatch_slab"] == 0


def test_stall_in_a_batch_fails_the_whole_call():
    fields = [synth.vortex_sum(40 + 8 * k, 48, 4, seed=30 + k, n_vortex=3) for k in range(3)]
    cpt.inject_wave_stall(1, timeout_s=0.2)
    blobs, _, b = cpt.compress_batch([_dev(f) for f in fields], 5e-3, pred="sl", check=False)
    assert b["status"] == cpt.ERR_TIMEOUT and all(x is None for x in blobs)
    ok, _, _ = cpt.compress_batch([_dev(f) for f in fields], 5e-3, pred="sl")
    assert ok == [cpt.compress(_dev(f), 5e-3, pred="sl")[0] for f in fields]


def test_injection_arguments():
    with pytest.raises(cpt.CptError):
        cpt.inject_wave_stall(0, timeout_s=100.0)
    cpt.inject_wave_stall(None)  # clears; nothing pending
    uv = synth.vortex_sum(32, 32, 3, seed=4)
    blob, _, _ = cpt.compress(_dev(uv), 1e-2)
    assert blob == oracle.compress(uv, 1e-2)["bytes"]


def test_verification_catches_a_corrupted_reconstruction():
    """The verification is not vacuous: one reconstructed value pushed past
    the bound, or moved across a crossed face, is reported."""
    import numpy as np
    uv = synth.vortex_sum(48, 56, 5, seed=6)
    d = _dev(uv)
    blob, st, g = cpt.compress(d, 1e-2, pred="mop", debug=True)
    assert st["verify_mismatch_slice"] == 0 and st["verify_mismatch_slab"] == 0
    T, H, W, _ = uv.shape
    # (1) far past the pointwise bound at an interior vertex
    v = (2 * H + H // 2) * W + W // 2
    cpt.inject_verify_fault(v, 1 << 20)
    b2, s2, _ = cpt.compress(d, 1e-2, pred="mop", check=False)
    assert s2["status"] == cpt.ERR_VERIFY and s2["linf"] > s2["eps"]
    assert b2 == blob  # the stream does not change
    # (2) a vertex of a crossed face flipped to the other side of the origin
    crossed = np.flatnonzero(g["mask"].reshape(-1))
    v = int(crossed[len(crossed) // 2])
    qv = int(g["qhat"].reshape(-1, 2)[v, 0])
    cpt.inject_verify_fault(v, -2 * qv if qv != 0 else 1 << 10)
    _, s3, _ = cpt.compress(d, 1e-2, pred="mop", check=False)
    assert s3["status"] == cpt.ERR_VERIFY
    assert s3["verify_mismatch_slice"] + s3["verify_mismatch_slab"] > 0 or s3["linf"] > s3["eps"]
    # nothing pending afterwards
    _, s4, _ = cpt.compress(d, 1e-2, pred="mop")
    assert s4["verify_mismatch_slice"] == 0 and s4["linf"] <= s4["eps"]


def _expected_force(r0, uv, v, delta, eps):
    """The vertices a repair must store losslessly, from the oracle alone: the
    oracle's reconstruction with the injected change at vertex v, the faces
    whose predicate that changes (their three vertices each) and the vertices
    past the pointwise bound."""
    import numpy as np
    T, H, W, _ = uv.shape
    qh = r0["qhat"].copy()
    qh.reshape(-1, 2)[v, 0] += delta
    diff = oracle.face_masks(qh) ^ r0["mask"]
    faces = oracle.face_table()  # [type][vertex][(dt, di, dj)]
    force = np.zeros((T, H, W), bool)
    for t, i, j in np.argwhere(diff != 0):
        d = int(diff[t, i, j])
        for ty in range(12):
            if (d >> ty) & 1:
                for dt, di, dj in faces[ty]:
                    force[t + dt, i + di, j + dj] = True
    k = r0["stats"]["k"]
    bound = max(eps, np.ldexp(0.5, -k))
    err = np.abs(np.ldexp(qh.astype(np.float64), -k) - uv.astype(np.float64)).max(axis=3)
    force |= err > bound
    return force


@pytest.mark.parametrize("case", ["crossed_face", "past_bound"])
def test_repair_after_a_failed_verification(case):
    """Reading R14's repair: an injected fault makes the first verification
    fail; the vertices of the changed faces (and those past the bound) are
    stored losslessly and the field is encoded again.  The stream returned
    equals the oracle's with the same vertices forced (computed from the
    oracle), verifies, and decodes identically on both sides."""
    import numpy as np
    uv = synth.vortex_sum(48, 56, 5, seed=6)
    d = _dev(uv)
    eb = 1e-2
    r0 = oracle.compress(uv, eb, pred="mop")
    T, H, W, _ = uv.shape
    if case == "crossed_face":
        crossed = np.flatnonzero(r0["mask"].reshape(-1))
        v = int(crossed[len(crossed) // 2])
        qv = int(r0["qhat"].reshape(-1, 2)[v, 0])
        delta = -2 * qv if qv != 0 else 1 << 10
    else:
        v = (2 * H + H // 2) * W + W // 2
        delta = 1 << 20
    force = _expected_force(r0, uv, v, delta, r0["stats"]["eps"])
    assert force.any()
    cpt.inject_verify_fault(v, delta)
    blob, st, _ = cpt.compress(d, eb, pred="mop", repair=True)
    assert st["status"] == cpt.OK and st["repair_rounds"] == 1
    assert st["forced_vertices"] == int(force.sum())
    assert st["verify_mismatch_slice"] == 0 and st["verify_mismatch_slab"] == 0 and st["linf"] <= st["eps"]
    ref = oracle.compress(uv, eb, pred="mop", force=force)
    assert blob == ref["bytes"]
    qo, xo, _ = oracle.decompress(blob)
    out, qg, _ = cpt.decompress(blob, want_q=True)
    assert (qg == qo).all() and np.array_equal(out.view(np.uint32), xo.view(np.uint32))
    assert (oracle.face_masks(qo) == r0["mask"]).all()
    # without repair the same fault is reported, and nothing stays pending
    cpt.inject_verify_fault(v, delta)
    _, s2, _ = cpt.compress(d, eb, pred="mop", check=False)
    assert s2["status"] == cpt.ERR_VERIFY
    b3, s3, _ = cpt.compress(d, eb, pred="mop", repair=True)
    assert s3["repair_rounds"] == 0 and b3 == r0["bytes"]


def test_verification_counts_on_a_rough_field():
    """On a field where most vertices take the exact face test (integers in
    -2..2), the per-warp queue of the interior items fills and the rest of
    such an item is tested vertex by vertex.  A corrupted reconstruction is
    counted exactly there: slice and slab mismatches equal the popcounts of
    the oracle's mask difference."""
    import numpy as np
    rng = np.random.default_rng(31)
    uv = rng.integers(-2, 3, (3, 70, 130, 2)).astype(np.float32)
    d = _dev(uv)
    r0 = oracle.compress(uv, 0.4, eb_mode="abs", pred="lorenzo")
    T, H, W, _ = uv.shape
    for (t, i, j) in ((1, 55, 70), (0, 60, 100), (1, 20, 10)):
        v = (t * H + i) * W + j
        qv = int(r0["qhat"].reshape(-1, 2)[v, 0])
        delta = -2 * qv if qv != 0 else 3
        qh = r0["qhat"].copy()
        qh.reshape(-1, 2)[v, 0] += delta
        diff = (oracle.face_masks(qh) ^ r0["mask"]).astype(np.uint32)
        bits = np.unpackbits(diff.view(np.uint8).reshape(-1, 4), axis=1, bitorder="little")
        want_slice = int(bits[:, 0:2].sum())
        want_slab = int(bits[:, 2:12].sum())
        assert want_slice + want_slab > 0
        cpt.inject_verify_fault(v, delta)
        _, s, _ = cpt.compress(d, 0.4, eb_mode="abs", pred="lorenzo", check=False)
        assert s["status"] == cpt.ERR_VERIFY
        assert s["verify_mismatch_slice"] == want_slice and s["verify_mismatch_slab"] == want_slab
    _, s, _ = cpt.compress(d, 0.4, eb_mode="abs", pred="lorenzo")
    assert s["verify_mismatch_slice"] == 0 and s["verify_mismatch_slab"] == 0
