"""Host-side behaviour of the C ABI that needs no GPU: the stream header
written by the oracle parses to the same grid in the library (a dimensions
query touches no device), malformed headers and null arguments are rejected
with their status codes, and on a machine without a GPU every compute call
fails with CPT_ERR_CUDA instead of falling back to the host."""
import ctypes as C
import struct

import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import cpt, synth

ARG, CUDA, CORRUPT = -1, -2, -4


def _query(blob):
    L = cpt.lib()
    buf = np.frombuffer(bytes(blob), np.uint8)
    d = cpt.Dims()
    rc = L.cpt_decompress(buf.ctypes.data if buf.size else None, buf.size, None, None, C.byref(d), None)
    return rc, d


@pytest.mark.parametrize("shape,pred,spacing", [((3, 9, 11), "lorenzo", (1.0, 1.0, 1.0)),
                                                ((2, 20, 17), "sl", (0.5, 2.0, 0.25)),
                                                ((4, 16, 32), "mop", (1.0, 1.0, 1.0))])
def test_header_of_oracle_stream(shape, pred, spacing):
    T, H, W = shape
    uv = synth.vortex_sum(H, W, T, seed=7)
    dx, dy, dt = spacing
    blob = oracle.compress(uv, 1e-2, pred=pred, dx=dx, dy=dy, dt=dt, debug=False)["bytes"]
    rc, d = _query(blob)
    assert rc == 0
    assert (d.H, d.W, d.T, d.dx, d.dy, d.dt) == (H, W, T, dx, dy, dt)


def _blob():
    return bytearray(oracle.compress(synth.vortex_sum(10, 12, 2, seed=8), 1e-2, debug=False)["bytes"])


def test_malformed_headers_are_rejected():
    good = _blob()
    assert _query(good)[0] == 0
    cases = []
    b = bytearray(good); b[0:4] = b"XPT1"; cases.append(b)           # magic
    b = bytearray(good); b[4:8] = struct.pack("<I", 99); cases.append(b)  # format version
    b = bytearray(good); b[8:12] = struct.pack("<I", 1); cases.append(b)  # H < 2
    b = bytearray(good); b[28:32] = struct.pack("<I", 7); cases.append(b)  # unknown predictor
    cases.append(good[:40])                                           # truncated header
    cases.append(bytearray(b"CPT"))                                   # shorter than the magic
    for b in cases:
        assert _query(b)[0] == CORRUPT
    assert _query(good)[0] == 0  # the original still parses


def test_null_arguments():
    L = cpt.lib()
    d = cpt.Dims(4, 4, 1, 1.0, 1.0, 1.0)
    p = cpt.Params()
    out = C.POINTER(C.c_uint8)()
    n = C.c_size_t(0)
    assert L.cpt_compress(None, C.byref(d), C.byref(p), C.byref(out), C.byref(n), None) == ARG
    assert L.cpt_decompress(None, 0, None, None, C.byref(d), None) == ARG
    tr = C.POINTER(cpt.Trajs)()
    assert L.cpt_extract_trajectories(None, C.byref(d), 0, C.byref(tr), None) == ARG
    assert L.cpt_compress_batch(None, C.byref(d), 1, C.byref(p), 0, C.byref(out), C.byref(n), None, None) == ARG
    assert b"null" in L.cpt_last_error()


def test_no_gpu_means_an_error_not_a_host_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU tests cover these calls")
    L = cpt.lib()
    uv = np.ascontiguousarray(synth.vortex_sum(8, 8, 2, seed=9))
    d = cpt.Dims(8, 8, 2, 1.0, 1.0, 1.0)
    p = cpt.Params()
    p.mode, p.eb, p.pred, p.block, p.stride, p.verify = 1, 1e-2, 0, 16, 2, 1
    out = C.POINTER(C.c_uint8)()
    n = C.c_size_t(0)
    assert L.cpt_compress(uv.ctypes.data, C.byref(d), C.byref(p), C.byref(out), C.byref(n), None) == CUDA
    assert not out and n.value == 0
    blob = np.frombuffer(bytes(_blob()), np.uint8)
    dest = np.zeros((2, 10, 12, 2), np.float32)
    assert L.cpt_decompress(blob.ctypes.data, blob.size, dest.ctypes.data, None, None, None) == CUDA
    assert not dest.any()
    tr = C.POINTER(cpt.Trajs)()
    assert L.cpt_extract_trajectories(uv.ctypes.data, C.byref(d), -2**31, C.byref(tr), None) == CUDA
