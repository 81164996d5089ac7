"""ctypes binding of the CUDA library ``_build/libcpt.so`` (C ABI of
``include/cpt.h``).  Argument marshalling only: every step of the
compressor runs in the library's kernels.  Raises if the library has not
been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcpt.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_CORRUPT, ERR_VERIFY, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
PRED = {"lorenzo": 0, "sl": 1, "mop": 2, "learned": 3, "learned_mop": 4}
NET_PARAMS = 10434
EB_MODE = {"abs": 0, "rel": 1}
STAGES = ["range_fixed", "face_masks", "mop_sl", "incident_bounds", "wavefront", "entropy", "verify", "host"]


class Dims(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("T", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double)]


class Params(C.Structure):
    _fields_ = [("mode", C.c_int), ("eb", C.c_double), ("pred", C.c_int), ("block", C.c_int32),
                ("stride", C.c_int32), ("verify", C.c_int32), ("cuda_stream", C.c_void_p),
                ("model", C.c_void_p), ("tune", C.c_int32), ("schedule", C.c_int32 * 6),
                ("zstd_level", C.c_int32), ("repair", C.c_int32), ("device_budget", C.c_uint64)]


class BatchStats(C.Structure):
    _fields_ = [("ms_total", C.c_double), ("ms_pipeline", C.c_double), ("ms_tune", C.c_double),
                ("groups", C.c_uint32), ("launches", C.c_uint32), ("schedule", C.c_int32 * 6),
                ("device_budget", C.c_uint64), ("in_bytes", C.c_uint64), ("out_bytes", C.c_uint64),
                ("ms_phase", C.c_double * 8)]


class Stats(C.Structure):
    _fields_ = [("ms_total", C.c_double), ("ms_stage", C.c_double * 8), ("launches", C.c_uint32 * 8),
                ("scale_log2", C.c_int32), ("eps_int", C.c_int32), ("eps", C.c_double),
                ("faces", C.c_uint64), ("crossed_faces", C.c_uint64), ("lossless_vertices", C.c_uint64),
                ("unpredictable", C.c_uint64), ("sl_blocks", C.c_uint64), ("blocks", C.c_uint64),
                ("n_ld", C.c_uint64), ("n_qd", C.c_uint64), ("verify_mismatch_slice", C.c_uint64),
                ("verify_mismatch_slab", C.c_uint64), ("linf", C.c_double), ("psnr", C.c_double),
                ("ratio", C.c_double), ("out_bytes", C.c_uint64), ("raw_bytes", C.c_uint64),
                ("forced_vertices", C.c_uint64), ("repair_rounds", C.c_int32), ("reserved0", C.c_int32)]


class Debug(C.Structure):
    _fields_ = [("q", C.c_void_p), ("qhat", C.c_void_p), ("xi", C.c_void_p), ("qxi", C.c_void_p),
                ("sym", C.c_void_p), ("mask", C.c_void_p), ("modes", C.c_void_p),
                ("qxi_hist", C.c_void_p), ("qd_hist", C.c_void_p), ("zero_runs", C.c_void_p)]

RUN_MAX = 4096  # zero_runs bins: [L] for 1 <= L <= RUN_MAX, [RUN_MAX + 1] longer runs, [0] their total length


class Trajs(C.Structure):
    _fields_ = [("n_traj", C.c_uint64), ("n_points", C.c_uint64), ("offsets", C.POINTER(C.c_uint64)),
                ("face_ids", C.POINTER(C.c_uint64)), ("xyt", C.POINTER(C.c_double)), ("bad_tets", C.c_uint64)]


class CptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cpt status {status}: {msg}")
        self.status = status


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            P = C.POINTER
            L.cpt_compress_ex.restype = C.c_int
            L.cpt_compress_ex.argtypes = [C.c_void_p, P(Dims), P(Params), P(P(C.c_uint8)), P(C.c_size_t),
                                          P(Stats), P(Debug)]
            L.cpt_compress.restype = C.c_int
            L.cpt_compress.argtypes = [C.c_void_p, P(Dims), P(Params), P(P(C.c_uint8)), P(C.c_size_t), P(Stats)]
            L.cpt_compress_batch.restype = C.c_int
            L.cpt_compress_batch.argtypes = [P(C.c_void_p), P(Dims), C.c_int32, P(Params), C.c_size_t,
                                             P(P(C.c_uint8)), P(C.c_size_t), P(Stats), P(BatchStats)]
            L.cpt_decompress.restype = C.c_int
            L.cpt_decompress.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, P(Dims), C.c_void_p]
            L.cpt_extract_trajectories.restype = C.c_int
            L.cpt_extract_trajectories.argtypes = [C.c_void_p, P(Dims), C.c_int32, P(P(Trajs)), C.c_void_p]
            L.cpt_free.argtypes = [C.c_void_p]
            L.cpt_zstd_wrap.argtypes = [C.c_void_p, C.c_size_t, C.c_int32, P(P(C.c_uint8)), P(C.c_size_t)]
            L.cpt_zstd_unwrap.argtypes = [C.c_void_p, C.c_size_t, P(P(C.c_uint8)), P(C.c_size_t)]
            L.cpt_free_trajs.argtypes = [P(Trajs)]
            L.cpt_error_string.restype = C.c_char_p
            L.cpt_error_string.argtypes = [C.c_int]
            L.cpt_last_error.restype = C.c_char_p
            L.cpt_version.restype = C.c_uint32
            L.cpt_inject_verify_fault.restype = C.c_int
            L.cpt_inject_verify_fault.argtypes = [C.c_int64, C.c_int32]
            L.cpt_inject_wave_stall.restype = C.c_int
            L.cpt_inject_wave_stall.argtypes = [C.c_int64, C.c_int64]
            L.cpt_fixed_point_noalloc.restype = C.c_int
            L.cpt_fixed_point_noalloc.argtypes = [C.c_void_p, P(Dims), C.c_void_p, C.c_void_p, C.c_void_p]
            vp, i32 = C.c_void_p, C.c_int32
            L.cpt_net_predict.restype = C.c_int
            L.cpt_net_predict.argtypes = [vp, vp, i32, i32, vp, vp]
            L.cpt_net_gradients.restype = C.c_int
            L.cpt_net_gradients.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp]
            L.cpt_train_predictor.restype = C.c_int
            L.cpt_train_predictor.argtypes = [vp, vp, i32, i32, i32, i32, C.c_float, C.c_uint32, vp, vp, vp, vp]
            L.cpt_huffman_lengths.restype = C.c_int
            L.cpt_huffman_lengths.argtypes = [vp, C.c_uint32, i32, vp]
            L.cpt_pipeline_order.restype = C.c_int
            L.cpt_pipeline_order.argtypes = [i32, vp, vp, vp, P(C.c_uint64)]
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        L = lib()
        raise CptError(rc, f"{L.cpt_error_string(rc).decode()}: {L.cpt_last_error().decode()}")


def _ptr_and_shape(uv):
    """(pointer, (T,H,W), keepalive, device_stream) of a float32 [T][H][W][2]
    numpy array or torch tensor."""
    if isinstance(uv, np.ndarray):
        a = np.ascontiguousarray(uv, np.float32)
        assert a.ndim == 4 and a.shape[3] == 2
        return a.ctypes.data, a.shape[:3], a, None
    import torch  # noqa: WPS433 - torch only for device memory and streams
    assert isinstance(uv, torch.Tensor) and uv.dtype == torch.float32 and uv.is_contiguous()
    assert uv.dim() == 4 and uv.shape[3] == 2
    stream = torch.cuda.current_stream(uv.device).cuda_stream if uv.is_cuda else None
    return uv.data_ptr(), tuple(uv.shape[:3]), uv, stream


def _stats_dict(st):
    d = {f: getattr(st, f) for f, _ in Stats._fields_ if f not in ("ms_stage", "launches")}
    d["ms_stage"] = {STAGES[k]: st.ms_stage[k] for k in range(8)}
    d["launches"] = {STAGES[k]: st.launches[k] for k in range(8)}
    return d


class Stream:
    """A compressed stream left in the library's buffer (no copy): supports
    len(), bytes(), memoryview() and numpy(); the buffer goes back to the
    library when the object is released."""

    def __init__(self, ptr, n):
        self._ptr, self._n = ptr, n
        self._arr = (C.c_uint8 * n).from_address(C.addressof(ptr.contents)) if n else (C.c_uint8 * 0)()

    def __len__(self):
        return self._n

    def __bytes__(self):
        return bytes(memoryview(self._arr))

    def memoryview(self):
        return memoryview(self._arr)

    def numpy(self):
        return np.frombuffer(self._arr, np.uint8)

    def __del__(self):
        if getattr(self, "_ptr", None):
            try:
                lib().cpt_free(self._ptr)
            except Exception:  # interpreter shutdown
                pass
            self._ptr = None


def _params(eb, eb_mode, pred, block, stride, verify, stream, mdl, tune, schedule, zstd=0, repair=False,
            device_budget=0):
    sch = (C.c_int32 * 6)(*(tuple(schedule or ()) + (0,) * 6)[:6])
    return Params(EB_MODE[eb_mode], float(eb), PRED[pred], block, stride, 1 if verify else 0, stream,
                  None if mdl is None else mdl.ctypes.data, 1 if tune else 0, sch, int(zstd), 1 if repair else 0,
                  int(device_budget))


def compress(uv, eb, *, eb_mode="rel", pred="lorenzo", block=16, stride=2, verify=True, stream=None,
             dx=1.0, dy=1.0, dt=1.0, debug=False, check=True, copy=True, model=None, tune=False,
             schedule=None, rates=False, zstd=0, repair=False, device_budget=0):
    """Compresses float32 uv [T][H][W][2] (numpy array or torch tensor, host
    or device).  Returns (bytes, stats dict, debug dict or None); with
    copy=False the stream comes back as a Stream over the library's buffer.
    pred="learned" and "learned_mop" need `model`: uint16 [NET_PARAMS]
    bfloat16 bits.  zstd=L > 0 returns the stream wrapped in a ZSTD frame
    (level L, host side).  repair=True stores the vertices of faces a failed
    verification reports losslessly and encodes again.  device_budget=B > 0
    compresses slab by slab when the field's working set exceeds B bytes of
    device memory (same stream).  tune=True lets the
    library pick the encoder pipeline's
    schedule; schedule=(prep_share, sl_unit, slice_weight, slack, warps_per_sm)
    fixes it (zeros: defaults).
    rates=True (or debug=True) returns the rate diagnostics in the debug
    dict: qxi_hist [33], qd_hist [65536] and zero_runs [RUN_MAX + 2]."""
    ptr, (T, H, W), keep, dev_stream = _ptr_and_shape(uv)
    if stream is None:
        stream = dev_stream
    dims = Dims(H, W, T, dx, dy, dt)
    mdl = None if model is None else _model_array(model)
    prm = _params(eb, eb_mode, pred, block, stride, verify, stream, mdl, tune, schedule, zstd, repair,
                  device_budget)
    out = C.POINTER(C.c_uint8)()
    n = C.c_size_t(0)
    st = Stats()
    dbg_arrays = None
    dbgp = None
    if debug or rates:
        dbg_arrays = dict(qxi_hist=np.zeros(33, np.uint32), qd_hist=np.zeros(65536, np.uint32),
                          zero_runs=np.zeros(RUN_MAX + 2, np.uint64))
    if debug:
        nby, nbx = -(-H // block), -(-W // block)
        dbg_arrays.update(q=np.zeros((T, H, W, 2), np.int32), qhat=np.zeros((T, H, W, 2), np.int32),
                          xi=np.zeros((T, H, W), np.int32), qxi=np.zeros((T, H, W), np.uint8),
                          sym=np.zeros((T, H, W, 2), np.uint16), mask=np.zeros((T, H, W), np.uint16),
                          modes=np.zeros((T, nby, nbx), np.uint8))
    if dbg_arrays is not None:
        dbgp = C.byref(Debug(*(dbg_arrays[f].ctypes.data if f in dbg_arrays else None for f, _ in Debug._fields_)))
    L = lib()
    rc = L.cpt_compress_ex(ptr, C.byref(dims), C.byref(prm), C.byref(out), C.byref(n), C.byref(st), dbgp)
    blob = None
    if out:
        if copy:
            blob = C.string_at(out, n.value)
            L.cpt_free(out)
        else:
            blob = Stream(out, n.value)
    if check:
        _check(rc)
    del keep, mdl
    s = _stats_dict(st)
    s["status"] = rc
    return blob, s, dbg_arrays


def compress_batch(fields, eb, *, eb_mode="rel", pred="lorenzo", block=16, stride=2, verify=True, stream=None,
                   dx=1.0, dy=1.0, dt=1.0, check=True, copy=True, model=None, tune=False, schedule=None,
                   device_budget=0):
    """Compresses a list of float32 fields [T][H][W][2] (numpy arrays or torch
    tensors, host or device) with one set of parameters in one batched call.
    Returns (list of streams, list of stats dicts, batch stats dict); each
    stream equals compress() of that field alone."""
    n = len(fields)
    ptrs, dims, keep = (C.c_void_p * n)(), (Dims * n)(), []
    dev_stream = None
    for f, uv in enumerate(fields):
        ptr, (T, H, W), kp, ds = _ptr_and_shape(uv)
        ptrs[f] = ptr
        dims[f] = Dims(H, W, T, dx, dy, dt)
        keep.append(kp)
        dev_stream = dev_stream or ds
    if stream is None:
        stream = dev_stream
    mdl = None if model is None else _model_array(model)
    prm = _params(eb, eb_mode, pred, block, stride, verify, stream, mdl, tune, schedule)
    outs = (C.POINTER(C.c_uint8) * n)()
    nb = (C.c_size_t * n)()
    sts = (Stats * n)()
    bst = BatchStats()
    L = lib()
    rc = L.cpt_compress_batch(ptrs, dims, n, C.byref(prm), int(device_budget), outs, nb, sts, C.byref(bst))
    blobs = []
    for f in range(n):
        if not outs[f]:
            blobs.append(None)
        elif copy:
            blobs.append(C.string_at(outs[f], nb[f]))
            L.cpt_free(outs[f])
        else:
            blobs.append(Stream(outs[f], nb[f]))
    if check:
        _check(rc)
    del keep, mdl
    b = {f: getattr(bst, f) for f, _ in BatchStats._fields_ if f not in ("schedule", "ms_phase")}
    b["schedule"] = tuple(bst.schedule)
    b["ms_phase"] = [round(x, 3) for x in bst.ms_phase]
    b["status"] = rc
    return blobs, [_stats_dict(sts[f]) for f in range(n)], b


def decompress(blob, out=None, *, stream=None, want_q=False):
    """Decompresses a stream into float32 [T][H][W][2]: `out` may be a torch
    tensor (host or device) or None (a new numpy array).  Returns
    (uv, qhat or None, dims)."""
    L = lib()
    buf = np.frombuffer(blob, np.uint8)
    dims = Dims()
    _check(L.cpt_decompress(buf.ctypes.data, buf.size, None, None, C.byref(dims), stream))
    T, H, W = dims.T, dims.H, dims.W
    if out is None:
        out = np.empty((T, H, W, 2), np.float32)
        optr = out.ctypes.data
    else:
        optr, _, _, dev_stream = _ptr_and_shape(out)
        if stream is None:
            stream = dev_stream
    q = np.empty((T, H, W, 2), np.int32) if want_q else None
    _check(L.cpt_decompress(buf.ctypes.data, buf.size, optr, q.ctypes.data if want_q else None,
                            C.byref(dims), stream))
    return out, q, (H, W, T)


def extract_trajectories(uv, scale_log2=None, stream=None):
    """Trajectories of float32 uv [T][H][W][2]: (list of face-id arrays, list
    of xyt arrays, number of tets violating the 0-or-2 crossing count)."""
    ptr, (T, H, W), keep, dev_stream = _ptr_and_shape(uv)
    if stream is None:
        stream = dev_stream
    dims = Dims(H, W, T, 1.0, 1.0, 1.0)
    k = -(2 ** 31) if scale_log2 is None else int(scale_log2)
    out = C.POINTER(Trajs)()
    L = lib()
    _check(L.cpt_extract_trajectories(ptr, C.byref(dims), k, C.byref(out), stream))
    t = out.contents
    n, m = t.n_traj, t.n_points
    offs = np.ctypeslib.as_array(t.offsets, shape=(n + 1,)).copy()
    faces = np.ctypeslib.as_array(t.face_ids, shape=(max(m, 1),))[:m].copy() if m else np.zeros(0, np.uint64)
    xyt = (np.ctypeslib.as_array(t.xyt, shape=(max(3 * m, 1),))[:3 * m].reshape(m, 3).copy()
           if m else np.zeros((0, 3)))
    bad = t.bad_tets
    L.cpt_free_trajs(out)
    del keep
    return ([faces[offs[a]:offs[a + 1]] for a in range(n)], [xyt[offs[a]:offs[a + 1]] for a in range(n)], bad)


def inject_wave_stall(ticket, timeout_s=0.2):
    """Failure injection for tests: the next compression on this thread skips
    the wave item with this ticket and limits every wait to timeout_s, so it
    returns ERR_TIMEOUT.  ticket=None clears a pending injection."""
    _check(lib().cpt_inject_wave_stall(-1 if ticket is None else int(ticket), int(timeout_s * 1e9)))


def huffman_lengths(freq, maxlen=24):
    """Code lengths of the library's entropy stage for symbol frequencies
    (host only): uint8 array like freq."""
    f = np.ascontiguousarray(freq, np.uint64)
    out = np.zeros(f.size, np.uint8)
    _check(lib().cpt_huffman_lengths(f.ctypes.data if f.size else None, f.size, int(maxlen),
                                     out.ctypes.data if f.size else None))
    return out


def pipeline_order(fields, schedule=None):
    """Ticket order of the encoder pipeline's wave items for fields given as
    (T, H, R, with_units) tuples (host only): int32 [n_items][3] rows
    (field, t, strip)."""
    f = np.ascontiguousarray(np.asarray(fields, np.int32).reshape(-1, 4))
    sch = None
    if schedule is not None:
        sch = np.zeros(6, np.int32)
        sch[:len(schedule)] = schedule
    n = C.c_uint64(0)
    L = lib()
    _check(L.cpt_pipeline_order(len(f), f.ctypes.data, None if sch is None else sch.ctypes.data, None, C.byref(n)))
    out = np.empty((n.value, 3), np.int32)
    _check(L.cpt_pipeline_order(len(f), f.ctypes.data, None if sch is None else sch.ctypes.data,
                                out.ctypes.data, C.byref(n)))
    return out


def inject_verify_fault(vertex, delta):
    """Failure injection for tests: the next compression on this thread adds
    delta to the u component of one reconstructed vertex before verifying.
    vertex=None clears a pending injection."""
    _check(lib().cpt_inject_verify_fault(-1 if vertex is None else int(vertex), int(delta)))


def zstd_wrap(blob, level=3):
    """The optional ZSTD container around a stream (host only): bytes."""
    src = bytes(blob)
    out, n = C.POINTER(C.c_uint8)(), C.c_size_t(0)
    _check(lib().cpt_zstd_wrap(src, len(src), int(level), C.byref(out), C.byref(n)))
    r = C.string_at(out, n.value)
    lib().cpt_free(out)
    return r


def zstd_unwrap(blob):
    """The stream inside a ZSTD container (host only): bytes."""
    src = bytes(blob)
    out, n = C.POINTER(C.c_uint8)(), C.c_size_t(0)
    _check(lib().cpt_zstd_unwrap(src, len(src), C.byref(out), C.byref(n)))
    r = C.string_at(out, n.value)
    lib().cpt_free(out)
    return r


def fixed_point_noalloc(uv, q, k, stream=None):
    """Allocation-free range reduction + fixed-point conversion on the device:
    uv float32 [T][H][W][2], q int32 of the same shape and k an int32 tensor of
    one element, all CUDA tensors supplied by the caller.  Returns the status
    (asynchronous on `stream`, default the current torch stream)."""
    import torch
    assert uv.is_cuda and q.is_cuda and k.is_cuda and uv.dtype == torch.float32 and q.dtype == torch.int32
    T, H, W, _ = uv.shape
    if stream is None:
        stream = torch.cuda.current_stream(uv.device).cuda_stream
    dims = Dims(H, W, T, 1.0, 1.0, 1.0)
    return lib().cpt_fixed_point_noalloc(uv.data_ptr(), C.byref(dims), q.data_ptr(), k.data_ptr(), stream)


# ---------------------------------------------------------------------------
# learned predictor (an extension of the method)
# ---------------------------------------------------------------------------
def _model_array(model):
    m = np.ascontiguousarray(model, np.uint16)
    if m.shape != (NET_PARAMS,):
        raise ValueError(f"model must hold {NET_PARAMS} bfloat16 values")
    return m


def _pairs(prev, nxt=None):
    p = np.ascontiguousarray(prev, np.int32)
    if p.ndim == 3:
        p = p[None]
    assert p.ndim == 4 and p.shape[3] == 2
    if nxt is None:
        return p, None
    q = np.ascontiguousarray(nxt, np.int32).reshape(p.shape)
    return p, q


def net_predict(model, prev, stream=None):
    """Learned predictions int32 [H][W][2] of a slice from the reconstructed
    previous slice prev int32 [H][W][2] (fixed point), on the GPU."""
    m = _model_array(model)
    p, _ = _pairs(prev)
    _, H, W, _ = p.shape
    out = np.empty((H, W, 2), np.int32)
    _check(lib().cpt_net_predict(m.ctypes.data, p.ctypes.data, H, W, out.ctypes.data, stream))
    return out


def net_gradients(params, prev, nxt, stream=None):
    """(loss, gradient float32 [NET_PARAMS]) of the training objective at the
    float32 parameters over the pairs prev -> nxt (int32 [n][H][W][2])."""
    P = np.ascontiguousarray(params, np.float32)
    assert P.shape == (NET_PARAMS,)
    p, q = _pairs(prev, nxt)
    n, H, W, _ = p.shape
    g = np.empty(NET_PARAMS, np.float32)
    loss = C.c_float(0.0)
    _check(lib().cpt_net_gradients(P.ctypes.data, p.ctypes.data, q.ctypes.data, n, H, W, g.ctypes.data,
                                   C.addressof(loss), stream))
    return float(loss.value), g


def train_predictor(prev, nxt, steps, lr=1e-3, seed=0, init=None, stream=None):
    """Trains the learned predictor on the GPU with Adam over the pairs
    prev -> nxt (int32 [n][H][W][2]).  Returns (bfloat16 model uint16
    [NET_PARAMS], loss before each step float32 [steps])."""
    p, q = _pairs(prev, nxt)
    n, H, W, _ = p.shape
    ini = None if init is None else _model_array(init)
    model = np.empty(NET_PARAMS, np.uint16)
    losses = np.empty(int(steps), np.float32)
    _check(lib().cpt_train_predictor(p.ctypes.data, q.ctypes.data, n, H, W, int(steps), float(lr), int(seed) & 0xFFFFFFFF,
                                     None if ini is None else ini.ctypes.data, model.ctypes.data,
                                     losses.ctypes.data, stream))
    return model, losses
