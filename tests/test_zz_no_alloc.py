"""The allocation-free index build, against the ordinary one.

trd_index_build_noalloc is for callers that cannot allocate device memory
where they build an index (a framework whose pool owns all device memory, a
real-time loop that must not call cudaMalloc).  It keeps its scratch in a
fixed array inside the library and writes the index into buffers the caller
already owns.  This test calls it twice in a row through the C ABI, each time
on a different timeframe, and checks every output against trd_index_build:
identical bucket offsets, identical bucket membership, records that carry
exactly their tracklet's values, and the same rejected count.  The second
call's records start 16 bytes past a 32-byte boundary (the entry point asks
for 16-byte alignment only; the scatter stores whole 32-byte records where
the buffer allows it), and its offsets 4 bytes past a 16-byte boundary (the
scan writes four offsets per 16-byte store where the buffer allows it).  The file is named to be collected last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from synth import make_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_TRACKLETS = 1 << 20


def _noalloc_fn():
    from paper_2003_03174_b300 import trd
    L = trd.lib()
    fn = L.trd_index_build_noalloc
    fn.argtypes = [C.POINTER(trd.Tracklets), C.c_float, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    return fn


def _with_invalid(trk, k):
    """Append k tracklets the index must reject (bad chamber, NaN, negative variance)."""
    bad = {key: v[:k].copy() for key, v in trk.items()}
    bad["chamber"][: k // 3] = 600
    bad["y"][k // 3: 2 * k // 3] = np.nan
    bad["vzz"][2 * k // 3:] = -1.0
    return {key: np.concatenate([trk[key], bad[key]]) for key in trk}


def _check_one(ctx, trk_np, w, stream, shift=0, off_shift=0):
    from paper_2003_03174_b300 import trd
    fn = _noalloc_fn()
    dev = trd.to_device(trk_np)
    n = int(trk_np["chamber"].shape[0])
    nb = int(math.ceil(np.float32(132.0) / np.float32(w)))
    n_buckets = 540 * 18 * nb
    # caller-owned outputs (the test allocates them; the entry point does not)
    off_buf = torch.full((n_buckets + 1 + off_shift,), -7, dtype=torch.int32, device="cuda")
    offsets = off_buf[off_shift:]
    assert offsets.data_ptr() % 16 == 4 * off_shift % 16
    # shift floats past the allocation's start (torch aligns it to 512 bytes)
    buf = torch.full((max(n, 1) * 8 + shift,), float("nan"), dtype=torch.float32, device="cuda")
    records = buf[shift:].view(-1, 8)
    assert records.data_ptr() % 32 == 4 * shift % 32
    stats = torch.full((4,), 12345, dtype=torch.int32, device="cuda")
    ts = trd.tracklets_struct(dev)
    # the fills and copies above ran on torch's current stream; the call runs
    # on its own (non-blocking) stream, so it must wait for them
    stream.wait_stream(torch.cuda.current_stream())
    rc = fn(C.byref(ts), float(w), C.c_void_p(offsets.data_ptr()), C.c_void_p(records.data_ptr()),
            C.c_void_p(stats.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == trd.TRD_OK
    torch.cuda.synchronize()

    ref = ctx.index_build(dev, w)
    ref_off, ref_ids = ref.copy_out()
    info = ref.info()
    off = offsets.cpu().numpy()
    np.testing.assert_array_equal(off, ref_off)
    total = int(off[-1])
    assert total == info["n_indexed"]
    rec = records[:total].cpu().numpy()
    ids = rec[:, 3].view(np.int32)
    # same tracklets in every bucket (the order inside a bucket is free)
    counts = np.diff(off)
    bucket_of_pos = np.repeat(np.arange(n_buckets), counts)
    ref_bucket = np.empty(n, np.int64)
    ref_bucket[ref_ids] = np.repeat(np.arange(n_buckets), np.diff(ref_off))
    np.testing.assert_array_equal(ref_bucket[ids], bucket_of_pos)
    assert np.array_equal(np.sort(ids), np.sort(ref_ids))
    # each record carries exactly its tracklet's values
    for col, key in ((0, "y"), (1, "z"), (2, "dy"), (4, "vyy"), (5, "vzz"), (6, "vyz")):
        np.testing.assert_array_equal(rec[:, col], trk_np[key][ids], err_msg=key)
    st = stats.cpu().numpy().view(np.uint32)
    assert int(st[2]) == info["n_rejected"]
    valid = np.zeros(n, bool)
    valid[ids] = True
    assert st[0] == np.float32(trk_np["vyy"][valid].max()).view(np.uint32)
    assert st[1] == np.float32(trk_np["vzz"][valid].max()).view(np.uint32)
    ref.free()


def test_noalloc_index_matches_index_build_on_two_calls_in_a_row():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = trd.Context(0)
    stream = torch.cuda.Stream()
    first = _with_invalid(make_workload("timeframe", seed=31, n_seeds=60_000).tracklets, 30)
    second = make_workload("tiny", seed=32).tracklets  # smaller: stale scratch must not leak
    _check_one(ctx, first, 2.0, stream)
    _check_one(ctx, second, 1.5, stream, shift=4, off_shift=1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _noalloc_fn()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    too_many = trd.Tracklets(*([p] * 7), MAX_TRACKLETS + 1)
    assert fn(C.byref(too_many), 2.0, p, p, p, None) == trd.TRD_EINVAL
    small = trd.Tracklets(*([p] * 7), 4)
    assert fn(C.byref(small), 0.5, p, p, p, None) == trd.TRD_EINVAL  # bins narrower than 1 cm
    assert fn(C.byref(small), 2.0, None, p, p, None) == trd.TRD_EINVAL
