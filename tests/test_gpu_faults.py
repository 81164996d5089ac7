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
