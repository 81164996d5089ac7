"""Slab-by-slab compression (cpt_params.device_budget below the field's
working set): the stream is byte for byte the in-memory call's, for every
predictor, from device or host input, with slabs of one slice up to many."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth
from test_gpu_parity import _dev

pytestmark = pytest.mark.gpu

FIXED = 160 << 20    # the slab compressor's fixed device buffers
PER_VS = 72          # window bytes per vertex of one window slice


def budget_for(H, W, S):
    """A device budget that gives slabs of S slices."""
    return FIXED + (S + 2) * PER_VS * H * W + (1 << 20)


def _same(blob, st, ref, st0):
    assert blob == ref
    for f in ("crossed_faces", "n_ld", "n_qd", "lossless_vertices", "unpredictable", "sl_blocks",
              "verify_mismatch_slice", "verify_mismatch_slab", "scale_log2", "eps_int"):
        assert st[f] == st0[f], f
    assert st["linf"] == st0["linf"]


@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
def test_street512_slabs_match_in_memory(pred):
    uv, eb = synth.workload("street512")
    d = _dev(uv)
    ref, st0, _ = cpt.compress(d, eb, pred=pred)
    blob, st, _ = cpt.compress(d, eb, pred=pred, device_budget=budget_for(512, 512, 12))
    _same(blob, st, ref, st0)


@pytest.mark.parametrize("S", [1, 2, 5])
def test_slab_sizes_and_host_input(S):
    """Slabs of 1, 2 and 5 slices over 12 slices of the vortex street (MoP):
    equal to the in-memory stream and to the oracle's, from host input too."""
    uv, eb = synth.workload("street512")
    uv = np.ascontiguousarray(uv[:12])
    ref, st0, _ = cpt.compress(_dev(uv), eb, pred="mop")
    blob, st, _ = cpt.compress(_dev(uv), eb, pred="mop", device_budget=budget_for(512, 512, S))
    _same(blob, st, ref, st0)
    hb, hs, _ = cpt.compress(uv, eb, pred="mop", device_budget=budget_for(512, 512, S))
    assert hb == ref
    if S == 1:
        assert blob == oracle.compress(uv, eb, pred="mop", debug=False)["bytes"]


def test_learned_mixture_slabs_match_in_memory():
    uv, eb = synth.workload("street512")
    uv = np.ascontiguousarray(uv[:10])
    P = np.random.default_rng(5).normal(0.0, 0.03, cpt.NET_PARAMS).astype(np.float32)
    model = (P.view(np.uint32) >> 16).astype(np.uint16)
    ref, st0, _ = cpt.compress(_dev(uv), eb, pred="learned_mop", model=model)
    blob, st, _ = cpt.compress(_dev(uv), eb, pred="learned_mop", model=model, device_budget=budget_for(512, 512, 3))
    _same(blob, st, ref, st0)


def test_budget_errors():
    uv, eb = synth.workload("street512")
    d = _dev(np.ascontiguousarray(uv[:10]))
    with pytest.raises(cpt.CptError) as e:
        cpt.compress(d, eb, pred="mop", device_budget=1 << 20)
    assert e.value.status == cpt.ERR_OOM
    with pytest.raises(cpt.CptError) as e:
        cpt.compress(d, eb, pred="mop", device_budget=budget_for(512, 512, 2), debug=True)
    assert e.value.status == cpt.ERR_UNSUPPORTED
    # a budget the field fits in: the in-memory call
    ref, _, _ = cpt.compress(d, eb, pred="mop")
    blob, _, _ = cpt.compress(d, eb, pred="mop", device_budget=64 << 30)
    assert blob == ref
