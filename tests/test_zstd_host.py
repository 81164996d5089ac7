"""The optional ZSTD container of a stream (the lossless stage after the
Huffman coder, Alg. 3 lossless_comp), host side, no GPU needed: the stream
inside is the stream byte for byte, the decompressor reads containers
(a dimensions query touches no device), malformed containers are rejected."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth

CORRUPT, ARG, UNSUPPORTED = -4, -1, -7


def _wrap_or_skip(blob, level=3):
    try:
        return cpt.zstd_wrap(blob, level)
    except cpt.CptError as e:
        if e.status == UNSUPPORTED:
            pytest.skip("libzstd.so.1 is not available on this machine")
        raise


def _query(blob):
    buf = np.frombuffer(bytes(blob), np.uint8)
    d = cpt.Dims()
    rc = cpt.lib().cpt_decompress(buf.ctypes.data, buf.size, None, None, C.byref(d), None)
    return rc, d


@pytest.mark.parametrize("level", [1, 3, 19])
def test_container_round_trip(level):
    uv = synth.vortex_sum(40, 44, 6, seed=3)
    raw = oracle.compress(uv, 1e-2, pred="mop", debug=False)["bytes"]
    z = _wrap_or_skip(raw, level)
    assert z[:4] == b"CPTZ" and int.from_bytes(z[8:16], "little") == len(raw)
    assert cpt.zstd_unwrap(z) == raw
    rc, d = _query(z)
    assert rc == 0 and (d.H, d.W, d.T) == (40, 44, 6)


def test_container_shrinks_a_redundant_stream():
    uv = np.zeros((4, 32, 32, 2), np.float32)  # a field of zeros: long runs of one code
    raw = oracle.compress(uv, 1e-2, pred="lorenzo", debug=False)["bytes"]
    z = _wrap_or_skip(raw)
    assert len(z) < len(raw) and cpt.zstd_unwrap(z) == raw


def test_malformed_containers_are_rejected():
    raw = oracle.compress(synth.vortex_sum(10, 12, 2, seed=8), 1e-2, debug=False)["bytes"]
    z = bytearray(_wrap_or_skip(raw))
    for bad in (z[:10], z[:-5], z[:16] + bytes(len(z) - 16)):
        with pytest.raises(cpt.CptError) as e:
            cpt.zstd_unwrap(bytes(bad))
        assert e.value.status == CORRUPT
        assert _query(bad)[0] == CORRUPT
    wrong_size = bytearray(z)
    wrong_size[8:16] = (len(raw) + 1).to_bytes(8, "little")
    with pytest.raises(cpt.CptError) as e:
        cpt.zstd_unwrap(bytes(wrong_size))
    assert e.value.status == CORRUPT
    with pytest.raises(cpt.CptError) as e:
        cpt.zstd_unwrap(raw)  # a plain stream is not a container
    assert e.value.status == CORRUPT
    for level in (0, 1000):
        with pytest.raises(cpt.CptError) as e:
            cpt.zstd_wrap(raw, level)
        assert e.value.status == ARG
