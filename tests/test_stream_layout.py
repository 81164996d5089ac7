"""The stream layout, read by a decoder written here from its documented
format (reading R12), independently of both encoders: the 96-byte header,
the block-mode bits, the model section of the learned predictors, two
canonical Huffman streams (code book in symbol order, a bit offset every
16384 symbols, 32-bit words filled most significant bit first) and the
verbatim values L_d.  Decoding an oracle stream must give back exactly the
oracle's bound codes, residual symbols and verbatim values, with no byte
left over.  (The GPU's streams are byte-identical to the oracle's in the GPU
parity tests, so this covers them too.)"""
import struct

import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import synth


class _Reader:
    def __init__(self, b):
        self.b, self.p = b, 0

    def take(self, fmt):
        v = struct.unpack_from("<" + fmt, self.b, self.p)
        self.p += struct.calcsize("<" + fmt)
        return v if len(v) > 1 else v[0]

    def raw(self, n):
        v = self.b[self.p:self.p + n]
        self.p += n
        return v


def _canonical(lengths):
    """Canonical prefix code from code lengths (the construction of RFC 1951,
    Sec. 3.2.2): codes of one length are consecutive in symbol order, and
    shorter codes come first."""
    maxlen = max(lengths.values())
    count = [0] * (maxlen + 1)
    for l in lengths.values():
        count[l] += 1
    nxt, code = [0] * (maxlen + 2), 0
    for l in range(1, maxlen + 1):
        code = (code + count[l - 1]) << 1
        nxt[l] = code
    codes = {}
    for s in sorted(lengths):
        l = lengths[s]
        codes[s] = (nxt[l], l)
        nxt[l] += 1
    return codes


def _huffman(r):
    nsym, nused, chunk = r.take("QII")
    assert chunk == 16384
    table = [r.take("I") for _ in range(nused)]
    syms = [e >> 8 for e in table]
    assert syms == sorted(syms) and len(set(syms)) == nused
    lengths = {e >> 8: e & 0xFF for e in table}
    offs = [r.take("Q") for _ in range((nsym + chunk - 1) // chunk)]
    nwords = r.take("Q")
    words = np.frombuffer(r.raw(4 * nwords), "<u4")
    if nsym == 0:
        return np.zeros(0, np.int64)
    if nused == 1:  # one symbol: length-1 code
        assert list(lengths.values()) == [1]
    by_code = {c: s for s, c in _canonical(lengths).items()}
    bits = np.unpackbits(words.astype(">u4").view(np.uint8))  # most significant bit first
    out, pos, code, l = [], 0, 0, 0
    for x in range(nsym):
        if x % chunk == 0:
            assert offs[x // chunk] == pos
        code, l = 0, 0
        while (code, l) not in by_code:
            code = (code << 1) | int(bits[pos])
            pos += 1
            l += 1
            assert l <= 24
        out.append(by_code[(code, l)])
    assert nwords == (pos + 31) // 32 and not bits[pos:].any()  # zero padding
    return np.array(out, np.int64)


def _decode(blob):
    r = _Reader(blob)
    assert r.raw(4) == b"CPT1"
    ver, H, W, T, k, epsq, pred, B, n, radius, zero = r.take("IIIIiIIIIII")
    dx, dy, dt, eps = r.take("dddd")
    n_ld, mode_bytes = r.take("QQ")
    assert ver == 1 and radius == 32768 and zero == 0
    modes = np.unpackbits(np.frombuffer(r.raw(mode_bytes), np.uint8), bitorder="little")
    model = None
    if pred in (3, 4):
        npar = r.take("I")
        words = np.frombuffer(r.raw(4 * ((npar + 1) // 2)), "<u4")
        model = np.stack([words & 0xFFFF, words >> 16], 1).reshape(-1)[:npar].astype(np.uint16)
    qxi = _huffman(r)
    qd = _huffman(r)
    ld = np.frombuffer(r.raw(4 * n_ld), "<i4")
    assert r.p == len(blob)
    return dict(H=H, W=W, T=T, k=k, eps_int=epsq, pred=pred, B=B, n=n, dx=dx, dy=dy, dt=dt, eps=eps,
                modes=modes, model=model, qxi=qxi, qd=qd, ld=ld)


def _check(uv, eb, pred, model=None, **kw):
    res = oracle.compress(uv, eb, pred=pred, model=model, **kw)
    d = _decode(res["bytes"])
    T, H, W, _ = uv.shape
    st = res["stats"]
    assert (d["H"], d["W"], d["T"], d["k"], d["eps_int"]) == (H, W, T, st["k"], st["eps_int"])
    assert d["eps"] == st["eps"]
    assert (d["qxi"] == res["qxi"].reshape(-1)).all()
    present = res["qd"].reshape(-1) != 0xFFFFFFFF
    assert (d["qd"] == res["qd"].reshape(-1)[present]).all()
    # L_d: both values of a lossless vertex, the value of an unpredictable component
    q, qxi, qd = res["q"].reshape(-1, 2), res["qxi"].reshape(-1), res["qd"].reshape(-1, 2)
    want = []
    for v in range(q.shape[0]):
        for c in range(2):
            if qxi[v] == 0 or qd[v, c] == 0:
                want.append(int(q[v, c]))
    assert d["ld"].tolist() == want
    if pred in ("mop", "learned_mop"):
        m = res["modes"].reshape(-1)
        assert (d["modes"][:m.size] == m).all() and not d["modes"][m.size:].any()
    else:
        assert d["modes"].size == 0
    if model is not None:
        assert (d["model"] == model).all()
    return d


@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
def test_oracle_streams_follow_the_documented_layout(pred):
    uv, eb = synth.workload("vortex64")  # 32768 vertices: several sync points in both streams
    d = _check(uv, eb, pred)
    assert d["qxi"].size > 16384 and d["qd"].size > 2 * 16384


def test_layout_of_edge_cases():
    _check(np.zeros((2, 5, 6, 2), np.float32), 1e-2, "lorenzo")          # all zero: one symbol
    _check(synth.vortex_sum(9, 7, 3, seed=4), 0.0, "sl", eb_mode="abs")  # lossless: no Q_d symbol
    _check(synth.vortex_sum(20, 24, 3, seed=6), 1e-6, "mop", dx=0.5, dt=2.0)


def test_layout_with_a_model():
    from oracle import net_train as nt
    P = np.random.default_rng(3).normal(0.0, 0.03, nt.N_PARAMS)
    model = (nt.bf16_round(P).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    _check(synth.vortex_sum(24, 20, 3, seed=7), 5e-3, "learned_mop", model=model)
