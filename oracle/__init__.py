"""ctypes binding of the CPU oracle (``oracle/cpt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow, single-threaded
restatement of the compressor of "Time-Varying Vector Field Compression with
Preserved Critical Point Trajectories" (Alg. 1-4, Sec. VI).  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  The CUDA library never links or calls it.

The stream's byte layout is not fixed by the paper (reading R12); the tests
pin the writer to R12's description with a decoder written from it alone.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

QRADIUS = 32768


class Stats(C.Structure):
    _fields_ = [
        ("k", C.c_int32), ("eps_int", C.c_int32),
        ("eps", C.c_double), ("vmin", C.c_double), ("vmax", C.c_double),
        ("crossed_faces", C.c_uint64), ("lossless_vertices", C.c_uint64),
        ("unpredictable", C.c_uint64), ("sl_blocks", C.c_uint64), ("blocks", C.c_uint64),
        ("n_ld", C.c_uint64), ("n_qd", C.c_uint64),
        ("substep_vertices", C.c_uint64), ("substeps_total", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_PAR_SRC = os.path.join(_HERE, "cpt_oracle_par.c")
_PAR_LIB_PATH = os.path.join(_BUILD, "liboracle_par.so")
_lib_par = None


def build_par(force: bool = False) -> str:
    """Compiles the all-core harness of the oracle's parallel stages (the
    oracle's source included unchanged, run on slabs by host threads)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_PAR_SRC))
    if force or not os.path.exists(_PAR_LIB_PATH) or os.path.getmtime(_PAR_LIB_PATH) < newest:
        tmp = _PAR_LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-pthread",
                               "-fPIC", "-shared", "-I", _HERE, "-o", tmp, _PAR_SRC, "-lm"])
        os.replace(tmp, _PAR_LIB_PATH)
    return _PAR_LIB_PATH


def lib_par():
    global _lib_par
    with _lock:
        if _lib_par is None:
            L = C.CDLL(build_par())
            P = C.POINTER
            L.o_face_masks_par.argtypes = [P(C.c_int32), C.c_int, C.c_int, C.c_int, P(C.c_uint16), C.c_int]
            L.o_verify_par.argtypes = [P(C.c_int32), P(C.c_uint16), P(C.c_float), C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_int, P(C.c_uint64), P(C.c_uint64), P(C.c_double)]
            _lib_par = L
    return _lib_par


def face_masks_par(q, nthreads):
    """face_masks(q) computed slab by slab on nthreads host threads."""
    q = np.ascontiguousarray(q, np.int32)
    T, H, W, _ = q.shape
    m = np.zeros((T, H, W), np.uint16)
    rc = lib_par().o_face_masks_par(_p(q, C.c_int32), H, W, T, _p(m, C.c_uint16), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle face masks failed: {rc}")
    return m


def verify_par(qhat, mask, uv, k, nthreads):
    """Verification of a reconstruction qhat (exponent k) against the
    original's masks and values on nthreads host threads: (mismatching slice
    faces, mismatching slab faces, max |x_hat - x|)."""
    qhat = np.ascontiguousarray(qhat, np.int32)
    mask = np.ascontiguousarray(mask, np.uint16)
    uv = np.ascontiguousarray(uv, np.float32)
    T, H, W, _ = qhat.shape
    a, b, l = C.c_uint64(), C.c_uint64(), C.c_double()
    rc = lib_par().o_verify_par(_p(qhat, C.c_int32), _p(mask, C.c_uint16), _p(uv, C.c_float), H, W, T, int(k),
                                int(nthreads), C.byref(a), C.byref(b), C.byref(l))
    if rc != 0:
        raise RuntimeError(f"oracle verification failed: {rc}")
    return a.value, b.value, l.value


def lib():
    """The oracle library; CPT_ORACLE_LIB names another build of it (the
    mutation tests load deliberately broken copies this way)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(os.environ.get("CPT_ORACLE_LIB") or build())
            _declare(_lib)
            assert _lib.o_stats_size() == C.sizeof(Stats)
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _declare(L):
    i64, u64, i32, dbl = C.c_int64, C.c_uint64, C.c_int32, C.c_double
    P = C.POINTER
    L.o_incident_face_count.restype = C.c_int
    L.o_face_count.restype = i64
    L.o_face_count.argtypes = [C.c_int] * 3
    L.o_scale_exponent.restype = C.c_int
    L.o_scale_exponent.argtypes = [dbl]
    L.o_eps_int.restype = i32
    L.o_eps_int.argtypes = [dbl, C.c_int]
    L.o_range.argtypes = [P(C.c_float), i64, P(dbl), P(dbl), P(dbl)]
    L.o_to_fixed.argtypes = [P(C.c_float), i64, C.c_int, P(i32)]
    L.o_sos_det2.argtypes = [i64] * 4
    L.o_face_crossed_batch.argtypes = [P(i64), i64, P(C.c_uint8)]
    L.o_face_masks.argtypes = [P(i32), C.c_int, C.c_int, C.c_int, P(C.c_uint16)]
    L.o_alg2.restype = i64
    L.o_alg2.argtypes = [i64] * 6
    L.o_xi_code.argtypes = [i64]
    L.o_quantize.argtypes = [i64, i64, i64, P(i64)]
    L.o_lorenzo.restype = i64
    L.o_lorenzo.argtypes = [P(i32)] + [C.c_int] * 6
    L.o_sl_predict.argtypes = [P(i32), C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, P(i64), P(i64)]
    L.o_cfl.restype = C.c_float
    L.o_cfl.argtypes = [dbl, dbl, C.c_int]
    L.o_ilog2_q32.restype = u64
    L.o_ilog2_q32.argtypes = [C.c_uint32]
    L.o_score_q32.restype = i64
    L.o_score_q32.argtypes = [P(C.c_uint32), C.c_uint32, C.c_uint32, C.c_int]
    L.o_huff_lengths.argtypes = [P(u64), C.c_uint32, C.c_int, P(C.c_uint8)]
    L.o_compress.argtypes = [P(C.c_float), C.c_int, C.c_int, C.c_int, dbl, dbl, dbl, C.c_int, dbl,
                             C.c_int, C.c_int, C.c_int, C.c_int, P(P(C.c_uint8)), P(C.c_size_t),
                             P(i32), P(i32), P(i64), P(C.c_uint8), P(C.c_uint8), P(C.c_uint16),
                             P(C.c_uint32), P(Stats)]
    L.o_compress2.argtypes = [P(C.c_float), C.c_int, C.c_int, C.c_int, dbl, dbl, dbl, C.c_int, dbl,
                              C.c_int, C.c_int, C.c_int, C.c_int, P(C.c_uint16), P(P(C.c_uint8)),
                              P(C.c_size_t), P(i32), P(i32), P(i64), P(C.c_uint8), P(C.c_uint8),
                              P(C.c_uint16), P(C.c_uint32), P(Stats), P(C.c_uint8)]
    L.o_net_params.argtypes = []
    L.o_net_forward.argtypes = [P(C.c_uint16), P(i32), C.c_int, C.c_int, P(C.c_float)]
    L.o_net_predict.argtypes = [P(C.c_uint16), P(i32), C.c_int, C.c_int, P(i32)]
    L.o_decompress.argtypes = [P(C.c_uint8), C.c_size_t, P(C.c_int), P(i32), P(C.c_float)]
    L.o_free.argtypes = [C.c_void_p]
    L.o_trajectories.argtypes = [P(i32), C.c_int, C.c_int, C.c_int, P(u64), P(u64), P(P(u64)),
                                 P(P(u64)), P(P(dbl)), P(u64)]
    L.o_face_table.argtypes = [P(C.c_int)]
    L.o_tet_table.argtypes = [P(C.c_int)]


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def face_table():
    a = np.zeros((12, 3, 3), np.int32)
    lib().o_face_table(_p(a, C.c_int))
    return a


def tet_table():
    a = np.zeros((6, 4, 4), np.int32)
    lib().o_tet_table(_p(a, C.c_int))
    return a


def incident_face_count(H, W, T, t, i, j):
    return lib().o_incident_face_count(H, W, T, t, i, j)


def face_count(H, W, T):
    return lib().o_face_count(H, W, T)


def value_range(uv):
    """(min, max, max |x|) over u and v pooled, in double (Alg. 3's range
    for the relative bound and the fixed-point scale)."""
    uv = np.ascontiguousarray(uv, np.float32)
    mn, mx, am = C.c_double(), C.c_double(), C.c_double()
    rc = lib().o_range(_p(uv, C.c_float), uv.size, C.byref(mn), C.byref(mx), C.byref(am))
    if rc != 0:
        raise ValueError("non-finite value in the field")
    return mn.value, mx.value, am.value


def scale_exponent(amax):
    return lib().o_scale_exponent(float(amax))


def eps_int(eps, k):
    return lib().o_eps_int(float(eps), int(k))


def to_fixed(uv, k):
    uv = np.ascontiguousarray(uv, np.float32)
    q = np.empty(uv.shape, np.int32)
    lib().o_to_fixed(_p(uv, C.c_float), uv.size, int(k), _p(q, C.c_int32))
    return q


def sos_det2(au, av, bu, bv):
    return lib().o_sos_det2(int(au), int(av), int(bu), int(bv))


def face_crossed_batch(p):
    p = np.ascontiguousarray(p, np.int64).reshape(-1, 6)
    out = np.zeros(len(p), np.uint8)
    lib().o_face_crossed_batch(_p(p, C.c_int64), len(p), _p(out, C.c_uint8))
    return out.astype(bool)


def face_masks(q):
    """q: int32 [T][H][W][2] -> uint16 [T][H][W] crossed-face masks."""
    q = np.ascontiguousarray(q, np.int32)
    T, H, W, _ = q.shape
    m = np.zeros((T, H, W), np.uint16)
    lib().o_face_masks(_p(q, C.c_int32), H, W, T, _p(m, C.c_uint16))
    return m


def alg2(u0, v0, u1, v1, u2, v2):
    return lib().o_alg2(*(int(x) for x in (u0, v0, u1, v1, u2, v2)))


def xi_code(xi):
    return lib().o_xi_code(int(xi))


def quantize(q, p, xiq):
    out = C.c_int64()
    sym = lib().o_quantize(int(q), int(p), int(xiq), C.byref(out))
    return sym, out.value


def lorenzo(Q, t, i, j, c):
    Q = np.ascontiguousarray(Q, np.int32)
    T, H, W, _ = Q.shape
    return lib().o_lorenzo(_p(Q, C.c_int32), H, W, t, i, j, c)


def sl_predict(P, i, j, cfl_x, cfl_y):
    """P: reconstructed slice t-1, int32 [H][W][2]; cfl_x, cfl_y are rounded
    to binary32, the precision of the back-trace."""
    P = np.ascontiguousarray(P, np.int32)
    H, W, _ = P.shape
    pu, pv = C.c_int64(), C.c_int64()
    mode = lib().o_sl_predict(_p(P, C.c_int32), H, W, i, j, float(cfl_x), float(cfl_y),
                              C.byref(pu), C.byref(pv))
    return pu.value, pv.value, mode


def cfl(dt, dx, k):
    return lib().o_cfl(float(dt), float(dx), int(k))


def ilog2_q32(x):
    return lib().o_ilog2_q32(int(x))


def score_q32(hist, n_valid, n_fail, B):
    h = np.ascontiguousarray(hist, np.uint32)
    assert h.size == 2 * QRADIUS
    return lib().o_score_q32(_p(h, C.c_uint32), int(n_valid), int(n_fail), int(B))


def huff_lengths(freq, maxlen=24):
    f = np.ascontiguousarray(freq, np.uint64)
    out = np.zeros(f.size, np.uint8)
    rc = lib().o_huff_lengths(_p(f, C.c_uint64), f.size, int(maxlen), _p(out, C.c_uint8))
    assert rc == 0
    return out


PRED = {"lorenzo": 0, "sl": 1, "mop": 2, "learned": 3, "learned_mop": 4}


def net_params():
    """Number of bfloat16 parameters of the learned predictor."""
    return int(lib().o_net_params())


def net_forward(model, prev):
    """Learned predictor output y float32 [2][H][W] for a reconstructed slice
    prev int32 [H][W][2] and bfloat16 parameters model (uint16 bits)."""
    prev = np.ascontiguousarray(prev, np.int32)
    model = np.ascontiguousarray(model, np.uint16)
    H, W, _ = prev.shape
    y = np.empty((2, H, W), np.float32)
    lib().o_net_forward(_p(model, C.c_uint16), _p(prev, C.c_int32), H, W, _p(y, C.c_float))
    return y


def net_predict(model, prev):
    """Learned predictions int32 [H][W][2] of a slice from prev int32 [H][W][2]."""
    prev = np.ascontiguousarray(prev, np.int32)
    model = np.ascontiguousarray(model, np.uint16)
    H, W, _ = prev.shape
    out = np.empty((H, W, 2), np.int32)
    lib().o_net_predict(_p(model, C.c_uint16), _p(prev, C.c_int32), H, W, _p(out, C.c_int32))
    return out


def compress(uv, eb, *, eb_mode="rel", pred="lorenzo", block=16, stride=2, dx=1.0, dy=1.0,
             dt=1.0, t_end=None, debug=True, model=None, force=None):
    """Runs the oracle compressor on uv float32 [T][H][W][2].

    Returns a dict with the stream bytes (when t_end is None) and, with debug,
    the fixed-point input q, the reconstruction qhat, per-vertex bounds xi,
    their codes qxi, block modes, crossed-face masks, per-vertex symbols qd
    and the run statistics.  pred="learned" needs model (bfloat16 bits).
    force: optional bool [T][H][W], vertices stored losslessly (the repair of
    a failed verification, reading R14)."""
    uv = np.ascontiguousarray(uv, np.float32)
    T, H, W, two = uv.shape
    assert two == 2
    nby, nbx = -(-H // block), -(-W // block)
    L = lib()
    out = C.POINTER(C.c_uint8)()
    nbytes = C.c_size_t(0)
    st = Stats()
    d = {}
    if debug:
        d = dict(q=np.empty((T, H, W, 2), np.int32), qhat=np.empty((T, H, W, 2), np.int32),
                 xi=np.empty((T, H, W), np.int64), qxi=np.empty((T, H, W), np.uint8),
                 modes=np.empty((T, nby, nbx), np.uint8), mask=np.empty((T, H, W), np.uint16),
                 qd=np.empty((T, H, W, 2), np.uint32))
    te = T if t_end is None else int(t_end)
    m = None if model is None else np.ascontiguousarray(model, np.uint16)
    fz = None if force is None else np.ascontiguousarray(force, np.uint8).reshape(-1)
    assert fz is None or fz.size == T * H * W
    rc = L.o_compress2(_p(uv, C.c_float), H, W, T, dx, dy, dt, 1 if eb_mode == "rel" else 0,
                      float(eb), PRED[pred], block, stride, te, _p(m, C.c_uint16),
                      C.byref(out) if t_end is None else None,
                      C.byref(nbytes) if t_end is None else None,
                      _p(d.get("q"), C.c_int32), _p(d.get("qhat"), C.c_int32),
                      _p(d.get("xi"), C.c_int64), _p(d.get("qxi"), C.c_uint8),
                      _p(d.get("modes"), C.c_uint8), _p(d.get("mask"), C.c_uint16),
                      _p(d.get("qd"), C.c_uint32), C.byref(st), _p(fz, C.c_uint8))
    if rc != 0:
        raise RuntimeError(f"oracle compress failed: {rc}")
    if t_end is None:
        d["bytes"] = C.string_at(out, nbytes.value)
        L.o_free(out)
    d["stats"] = {f: getattr(st, f) for f, _ in Stats._fields_}
    return d


def qd_stream(res):
    """The residual-symbol stream Q_d of an oracle compression (debug=True):
    the u and v symbols of every vertex with a nonzero bound code, in raster
    order (the order in which Alg. 3 emits them)."""
    return res["qd"][res["qxi"] > 0].reshape(-1)


def zero_runs(qd, zero_sym=QRADIUS, run_max=4096):
    """Rate diagnostics: the maximal runs of the zero quantisation code
    (symbol zero_sym) in a symbol stream.  bins[L] counts the runs of length
    L for 1 <= L <= run_max, bins[run_max + 1] the longer runs and bins[0]
    their total length (so sum(L * bins[L]) + bins[0] is the number of zero
    codes)."""
    z = np.concatenate([[False], np.asarray(qd) == zero_sym, [False]]).astype(np.int8)
    d = np.diff(z)
    lengths = np.flatnonzero(d == -1) - np.flatnonzero(d == 1)
    bins = np.zeros(run_max + 2, np.uint64)
    short = lengths[lengths <= run_max]
    np.add.at(bins, short, 1)
    long_ = lengths[lengths > run_max]
    bins[run_max + 1] = len(long_)
    bins[0] = int(long_.sum())
    return bins


def decompress(blob):
    """Returns (qhat int32 [T][H][W][2], uv float32 [T][H][W][2], k)."""
    buf = np.frombuffer(blob, np.uint8).copy()
    dims = (C.c_int * 4)()
    L = lib()
    rc = L.o_decompress(_p(buf, C.c_uint8), buf.size, dims, None, None)
    if rc != 0:
        raise RuntimeError(f"oracle decompress failed: {rc}")
    H, W, T, k = dims
    qhat = np.empty((T, H, W, 2), np.int32)
    uv = np.empty((T, H, W, 2), np.float32)
    rc = L.o_decompress(_p(buf, C.c_uint8), buf.size, dims, _p(qhat, C.c_int32), _p(uv, C.c_float))
    if rc != 0:
        raise RuntimeError(f"oracle decompress failed: {rc}")
    return qhat, uv, k


def trajectories(q):
    """Links crossed faces of int32 q [T][H][W][2] into trajectories.

    Returns (list of face-id arrays, list of xyt arrays, number of tets whose
    crossed-face count is not 0 or 2)."""
    q = np.ascontiguousarray(q, np.int32)
    T, H, W, _ = q.shape
    L = lib()
    nt, nf, bad = C.c_uint64(), C.c_uint64(), C.c_uint64()
    fp, op, xp = C.POINTER(C.c_uint64)(), C.POINTER(C.c_uint64)(), C.POINTER(C.c_double)()
    rc = L.o_trajectories(_p(q, C.c_int32), H, W, T, C.byref(nt), C.byref(nf), C.byref(fp),
                          C.byref(op), C.byref(xp), C.byref(bad))
    if rc != 0:
        raise RuntimeError(f"oracle trajectories failed: {rc}")
    n, m = nt.value, nf.value
    faces = np.ctypeslib.as_array(fp, shape=(max(m, 1),))[:m].copy()
    offs = np.ctypeslib.as_array(op, shape=(n + 1,)).copy()
    xyt = np.ctypeslib.as_array(xp, shape=(max(3 * m, 1),))[:3 * m].reshape(m, 3).copy()
    L.o_free(fp)
    L.o_free(op)
    L.o_free(xp)
    trajs = [faces[offs[a]:offs[a + 1]] for a in range(n)]
    pts = [xyt[offs[a]:offs[a + 1]] for a in range(n)]
    return trajs, pts, bad.value
