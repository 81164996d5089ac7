"""The allocation-free fixed-point entry point, for callers that cannot
allocate device memory when they call it (pre-reserved pools, allocators that
forbid foreign allocations).  Through the C ABI it must give exactly the
fixed-point field and scale that cpt_compress_ex computes as its first step,
on two calls in a row (the shared scratch array keeps the previous call's
contents).  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2510_25143_gb300 import cpt, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(64, 64, 8), (37, 45, 5), (3, 5, 1)])
def test_noalloc_matches_compress_two_calls(shape):
    import torch
    H, W, T = shape
    uv = synth.vortex_sum(H, W, T, seed=21 + H, n_vortex=3)
    d_uv = torch.from_numpy(uv).to("cuda:0")
    _, st, dbg = cpt.compress(d_uv, 1e-2, pred="lorenzo", debug=True)
    for call in range(2):
        q = torch.full((T, H, W, 2), -7, dtype=torch.int32, device="cuda:0")
        k = torch.full((1,), 12345, dtype=torch.int32, device="cuda:0")
        assert cpt.fixed_point_noalloc(d_uv, q, k) == cpt.OK
        torch.cuda.synchronize()
        assert int(k.item()) == st["scale_log2"], call
        assert np.array_equal(q.cpu().numpy(), dbg["q"]), call


def test_noalloc_rejects_oversized_and_misaligned():
    import torch
    import ctypes
    buf = torch.zeros(64, dtype=torch.float32, device="cuda:0")
    q = torch.zeros(64, dtype=torch.int32, device="cuda:0")
    k = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    L = cpt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    big = cpt.Dims(16384, 16384, 1, 1.0, 1.0, 1.0)   # 2*H*W*T above the 16384*16384 limit
    assert L.cpt_fixed_point_noalloc(buf.data_ptr(), ctypes.byref(big), q.data_ptr(), k.data_ptr(), stream) == cpt.ERR_ARG
    # products that wrap around 64 bits are rejected, not run on a wrapped count
    for H, W, T in ((1 << 21, 1 << 21, 1 << 22), (1 << 30, 1 << 30, 1 << 30), (1 << 28, 2, 1)):
        huge = cpt.Dims(H, W, T, 1.0, 1.0, 1.0)
        assert L.cpt_fixed_point_noalloc(buf.data_ptr(), ctypes.byref(huge), q.data_ptr(), k.data_ptr(),
                                         stream) == cpt.ERR_ARG
    small = cpt.Dims(2, 2, 1, 1.0, 1.0, 1.0)
    assert L.cpt_fixed_point_noalloc(buf.data_ptr() + 4, ctypes.byref(small), q.data_ptr(), k.data_ptr(),
                                     stream) == cpt.ERR_ARG


@pytest.mark.parametrize("shape,nan_at,inf_tail", [((3, 5, 1), None, True), ((130, 130, 2), (1, 129, 100, 1), True),
                                                   ((130, 130, 2), (0, 70, 3, 0), False)])
def test_noalloc_non_finite_input(shape, nan_at, inf_tail):
    """A NaN in a late block or an infinity among the values after the last
    whole float4 group gives k = INT32_MIN and leaves q untouched; the next
    call on a finite field is not affected by what the shared scratch array
    kept."""
    import torch
    H, W, T = shape
    uv = synth.vortex_sum(H, W, T, seed=31 + H, n_vortex=3)
    bad = uv.copy()
    if nan_at is not None:
        bad[nan_at] = np.nan
    if inf_tail:
        # 2*H*W*T values; when that is not a multiple of 4 the last two are the tail
        bad.reshape(-1)[-1] = np.inf
    d_bad = torch.from_numpy(bad).to("cuda:0")
    q = torch.full((T, H, W, 2), -7, dtype=torch.int32, device="cuda:0")
    k = torch.full((1,), 12345, dtype=torch.int32, device="cuda:0")
    assert cpt.fixed_point_noalloc(d_bad, q, k) == cpt.OK
    torch.cuda.synchronize()
    assert int(k.item()) == np.iinfo(np.int32).min
    assert bool((q == -7).all())
    # a finite field next: the scratch array's stale contents leave no trace
    d_uv = torch.from_numpy(uv).to("cuda:0")
    _, st, dbg = cpt.compress(d_uv, 1e-2, pred="lorenzo", debug=True)
    assert cpt.fixed_point_noalloc(d_uv, q, k) == cpt.OK
    torch.cuda.synchronize()
    assert int(k.item()) == st["scale_log2"]
    assert np.array_equal(q.cpu().numpy(), dbg["q"])
