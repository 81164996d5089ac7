"""Pins of the oracle's rate diagnostics (the zero-code runs behind the
compression ratios, Sec. VII-E): hand-built streams, a brute-force run
counter, the conservation of zero codes, and the Q_d stream of a compression
against the stream's own counts."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import synth

Z = oracle.QRADIUS


def brute(stream, run_max):
    bins = np.zeros(run_max + 2, np.uint64)
    L = 0
    for x in list(stream) + [None]:
        if x == Z:
            L += 1
            continue
        if L:
            if L <= run_max:
                bins[L] += 1
            else:
                bins[run_max + 1] += 1
                bins[0] += L
        L = 0
    return bins


def test_hand_built_streams():
    b = oracle.zero_runs([Z, Z, 5, Z, 7, 7, Z, Z, Z])
    assert b[2] == 1 and b[1] == 1 and b[3] == 1 and b.sum() == 3
    assert oracle.zero_runs([]).sum() == 0
    assert oracle.zero_runs([1, 2, 3]).sum() == 0
    b = oracle.zero_runs([Z] * 10, run_max=4)
    assert b[5] == 1 and b[0] == 10 and b[1:5].sum() == 0
    b = oracle.zero_runs([Z] * 4, run_max=4)
    assert b[4] == 1 and b[5] == 0 and b[0] == 0


@pytest.mark.parametrize("p", [0.0, 0.3, 0.8, 0.97, 1.0])
def test_against_brute_force_and_conservation(p):
    rng = np.random.default_rng(int(p * 100))
    for n in (1, 2, 31, 33, 500):
        s = np.where(rng.random(n) < p, Z, rng.integers(0, 2 * Z, n))
        b = oracle.zero_runs(s, run_max=16)
        assert (b == brute(s, 16)).all()
        L = np.arange(17, dtype=np.uint64)
        assert int((L[1:] * b[1:17]).sum() + b[0]) == int((s == Z).sum())


def test_qd_stream_of_a_compression():
    uv = synth.vortex_sum(24, 30, 4, seed=5, n_vortex=3)
    r = oracle.compress(uv, 5e-3, pred="mop")
    qd = oracle.qd_stream(r)
    assert qd.size == r["stats"]["n_qd"]
    # the stream holds both components of every vertex with a bound, in raster order
    xs = r["qxi"].reshape(-1) > 0
    assert qd.size == 2 * int(xs.sum())
    assert (qd[0::2] == r["qd"].reshape(-1, 2)[xs, 0]).all()
    assert (qd[1::2] == r["qd"].reshape(-1, 2)[xs, 1]).all()
    b = oracle.zero_runs(qd)
    L = np.arange(b.size - 1, dtype=np.uint64)
    assert int((L[1:] * b[1:-1]).sum() + b[0]) == int((qd == Z).sum())
