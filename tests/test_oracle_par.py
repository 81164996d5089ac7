"""The all-core harness of the oracle's parallel stages (crossed-face masks
and verification, run slab by slab on host threads) gives exactly what the
single-threaded oracle gives; it only serves the CPU timing of the
benchmark."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import synth


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_par_masks_equal_oracle(threads):
    for uv in (synth.vortex_sum(37, 45, 6, seed=5, n_vortex=4),
               np.random.default_rng(2).integers(-2, 3, (5, 9, 11, 2)).astype(np.float32),
               synth.vortex_sum(20, 24, 1, seed=6)):
        q = oracle.to_fixed(uv, oracle.scale_exponent(float(np.abs(uv).max())))
        assert np.array_equal(oracle.face_masks_par(q, threads), oracle.face_masks(q))


def test_par_verify_counts_changes():
    uv = synth.vortex_sum(40, 44, 5, seed=9, n_vortex=4)
    r = oracle.compress(uv, 1e-2, pred="mop")
    k = r["stats"]["k"]
    a, b, linf = oracle.verify_par(r["qhat"], r["mask"], uv, k, 4)
    assert a == 0 and b == 0 and 0 < linf <= r["stats"]["eps"]
    # a reconstruction whose predicates differ: the original with one vertex
    # moved across the origin of a crossed face is counted, face by face
    q = r["q"].copy()
    t, i, j = np.argwhere(r["mask"][:, 1:-1, 1:-1] != 0)[0] + (0, 1, 1)
    q[t, i, j] = -q[t, i, j] * 3 + 7
    m_new = oracle.face_masks(q)
    diff = np.bitwise_xor(m_new, r["mask"]).astype(np.uint32)
    want_slice = int(sum(bin(int(x) & 3).count("1") for x in diff.ravel()))
    want_slab = int(sum(bin(int(x) & ~3 & 0xFFF).count("1") for x in diff.ravel()))
    assert want_slice + want_slab > 0
    a, b, linf = oracle.verify_par(q, r["mask"], uv, k, 3)
    assert (a, b) == (want_slice, want_slab)
    want_linf = np.abs(np.ldexp(q.astype(np.float64), -k) - uv.astype(np.float64)).max()
    assert linf == want_linf
