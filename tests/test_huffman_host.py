"""The library's code-length construction (host code of the entropy stage,
no GPU) against the oracle's: the same lengths, bit for bit, on random,
skewed and degenerate frequency tables, with and without the length limit
binding.  Equal lengths give equal canonical codes, so the two produce the
same stream bits for the same symbols."""
import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt


def _tables():
    rng = np.random.default_rng(21)
    yield np.zeros(40, np.uint64)                        # nothing used
    f = np.zeros(33, np.uint64); f[7] = 5; yield f       # one used symbol
    f = np.zeros(33, np.uint64); f[[0, 32]] = [1, 10**12]; yield f
    yield np.ones(1000, np.uint64)                       # ties everywhere
    for n in (2, 3, 33, 300, 5000, 65536):
        yield rng.integers(0, 1000, n).astype(np.uint64)
        g = np.zeros(n, np.uint64)                       # geometric: the limit binds
        used = rng.choice(n, min(n, 60), replace=False)
        g[used] = (2 ** np.arange(len(used))).astype(np.uint64)
        yield g
        yield (rng.pareto(1.2, n) * 100).astype(np.uint64)
    # a quantisation-code histogram: a sharp peak at the zero code
    x = np.rint(np.random.default_rng(22).laplace(0, 3.0, 200000)).astype(np.int64) + 32768
    yield np.bincount(x, minlength=65536).astype(np.uint64)


@pytest.mark.parametrize("maxlen", [24, 12, 8])
def test_lengths_match_the_oracle(maxlen):
    for f in _tables():
        if int((f > 0).sum()) > 2 ** maxlen:
            with pytest.raises(cpt.CptError):
                cpt.huffman_lengths(f, maxlen)
            continue
        got = cpt.huffman_lengths(f, maxlen)
        want = oracle.huff_lengths(f, maxlen)
        assert (got == want).all(), (f.size, maxlen)
        used = f > 0
        assert (got[~used] == 0).all() and got.max(initial=0) <= maxlen
        if used.sum() > 1:  # complete: Kraft sum exactly 1
            assert sum(2.0 ** -int(l) for l in got[used]) == 1.0


def test_arguments():
    with pytest.raises(cpt.CptError):
        cpt.huffman_lengths(np.ones(4, np.uint64), 0)
    with pytest.raises(cpt.CptError):
        cpt.huffman_lengths(np.ones(4, np.uint64), 33)
    assert cpt.huffman_lengths(np.zeros(0, np.uint64)).size == 0
