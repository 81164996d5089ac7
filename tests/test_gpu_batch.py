"""GPU tests of batched compression: many fields of uneven size and length in
one call, the encoder pipeline of all of them in one persistent launch.  Each
field's stream must be byte for byte the stream of a single-field call (and,
for the small fields, the oracle's); the pipeline's schedule, the autotuner
and the grouping under a memory budget must not change any byte."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth
from test_gpu_parity import _dev

pytestmark = pytest.mark.gpu

# uneven sizes and lengths, ragged against the 32-row strips, the 16-column
# sub-chunks and the MoP blocks; one single-slice field, one 2 x 2 field
SHAPES = [(37, 45, 5), (64, 64, 8), (50, 61, 3), (20, 33, 1), (96, 40, 7), (33, 70, 6), (2, 2, 3), (65, 17, 4)]


def _fields(seed=40, drift=0.7):
    return [synth.vortex_sum(H, W, T, seed=seed + k, n_vortex=3, drift=drift) for k, (H, W, T) in enumerate(SHAPES)]


def _singles(fields, eb, pred, **kw):
    return [cpt.compress(_dev(uv), eb, pred=pred, **kw)[0] for uv in fields]


def _random_model(seed=3, scale=0.03):
    from oracle import net_train as nt
    P = np.random.default_rng(seed).normal(0.0, scale, nt.N_PARAMS)
    return (nt.bf16_round(P).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop", "learned_mop"])
def test_batch_matches_single_and_oracle(pred):
    fields = _fields()
    eb = 5e-3
    model = _random_model() if pred.startswith("learned") else None
    blobs, stats, b = cpt.compress_batch([_dev(uv) for uv in fields], eb, pred=pred, model=model)
    assert b["groups"] == 1 and b["status"] == 0
    singles = _singles(fields, eb, pred, model=model)
    for k, uv in enumerate(fields):
        assert blobs[k] == singles[k], f"field {k} {SHAPES[k]}: batch stream differs from its single-field stream"
        st = stats[k]
        assert st["verify_mismatch_slice"] == 0 and st["verify_mismatch_slab"] == 0
        assert st["linf"] <= st["eps"] or st["eps_int"] == 0
    # the oracle on a few of them
    for k in (0, 3, 5, 6):
        assert blobs[k] == oracle.compress(fields[k], eb, pred=pred, model=model)["bytes"], k
    assert b["in_bytes"] == sum(uv.nbytes for uv in fields)
    assert b["out_bytes"] == sum(len(x) for x in blobs)


def test_batch_host_inputs_and_round_trip():
    fields = _fields(seed=60)
    blobs, stats, _ = cpt.compress_batch(fields, 3e-3, pred="mop")  # numpy inputs: copied inside the call
    for k, uv in enumerate(fields):
        out, _, _ = cpt.decompress(blobs[k])
        assert np.abs(out.astype(np.float64) - uv).max() <= stats[k]["eps"]


@pytest.mark.parametrize("pred,schedules", [
    ("lorenzo", [(0, 0, 1, 0, 4), (0, 0, 8, 0, 0)]),
    ("sl", [(30, 16, 0, 0, 2), (70, 8, 0, 0, 0)]),
    ("mop", [(30, 0, 0, 32, 3), (60, 0, 0, 128, 0)]),
])
def test_schedule_does_not_change_bytes(pred, schedules):
    fields = _fields(seed=80, drift=1.3)
    ref, _, _ = cpt.compress_batch([_dev(uv) for uv in fields], 4e-3, pred=pred)
    for sch in schedules:
        blobs, _, b = cpt.compress_batch([_dev(uv) for uv in fields], 4e-3, pred=pred, schedule=sch)
        assert blobs == ref, sch
        assert b["schedule"][:len(sch)] == tuple(sch)
    one, _, _ = cpt.compress(_dev(fields[1]), 4e-3, pred=pred, schedule=schedules[-1])
    assert one == ref[1]


def test_autotune_keeps_bytes():
    fields = _fields(seed=90)
    ref, _, _ = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="mop")
    tuned, _, b = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="mop", tune=True)
    assert tuned == ref
    # one of the MoP candidates: prediction-warp share 35..80 %, slack 64 or 128
    assert 35 <= b["schedule"][0] <= 80 and b["schedule"][3] in (64, 128)
    again, _, b2 = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="mop", tune=True)
    assert again == ref and b2["ms_tune"] == 0.0 and b2["schedule"] == b["schedule"]  # cached


def test_budget_groups_fields():
    fields = _fields(seed=100)
    ref, _, b1 = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="sl")
    blobs, _, b = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="sl", device_budget=1)
    assert b1["groups"] == 1 and b["groups"] == len(fields)  # every group holds one field
    assert blobs == ref


def test_batch_rejects_bad_field_and_returns_nothing():
    fields = _fields(seed=110)
    fields[4] = fields[4].copy()
    fields[4][2, 3, 4, 1] = np.nan
    blobs, _, b = cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="lorenzo", check=False)
    assert b["status"] == cpt.ERR_ARG
    assert all(x is None for x in blobs)
    with pytest.raises(cpt.CptError):
        cpt.compress_batch([_dev(uv) for uv in fields], 5e-3, pred="lorenzo")
    # the library stays usable
    ok, _, _ = cpt.compress_batch([_dev(uv) for uv in fields[:3]], 5e-3, pred="lorenzo")
    assert ok == _singles(fields[:3], 5e-3, "lorenzo")
