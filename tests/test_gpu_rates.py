"""GPU parity of the rate diagnostics: the histograms of the bound codes and
the residual symbols and the zero-code run lengths computed by the CUDA path,
against the oracle's streams (bit-exact: the streams are identical)."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth
from test_gpu_parity import _dev

pytestmark = pytest.mark.gpu


def _check(uv, eb, pred):
    _, st, g = cpt.compress(_dev(uv), eb, pred=pred, rates=True)
    r = oracle.compress(uv, eb, pred=pred)
    qd = oracle.qd_stream(r)
    assert (g["qxi_hist"] == np.bincount(r["qxi"].reshape(-1), minlength=33)).all()
    assert (g["qd_hist"] == np.bincount(qd, minlength=65536)).all()
    assert (g["zero_runs"] == oracle.zero_runs(qd)).all()
    return g, qd


@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
def test_vortex64(pred):
    uv, eb = synth.workload("vortex64")
    _check(uv, eb, pred)


def test_many_chunks():
    """About 2 M symbols: runs cross the 65536-symbol chunks of the kernel."""
    uv = synth.vortex_street(512, 512, 4, seed=1001)
    g, qd = _check(uv, 1e-3, "mop")
    assert qd.size > 20 * 65536


def test_runs_longer_than_a_chunk():
    """A field the Lorenzo predictor reproduces except near its critical
    point: zero codes in runs far longer than a chunk and the bin limit."""
    uv = synth.linear_field(256, 256, 3, a=100.3, b=0.3, c=120.7, d=0.2)
    g, qd = _check(uv, 1e-3, "lorenzo")
    assert g["zero_runs"][cpt.RUN_MAX + 1] > 0 and g["zero_runs"][0] > 65536
