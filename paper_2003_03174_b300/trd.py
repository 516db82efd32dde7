"""Python binding of libtrd.so: argument marshalling only.

Every step of the follower runs in the library's CUDA kernels; this module
turns torch tensors into the plain pointers and sizes of the C ABI
(include/trd_abi.h) and back.  There is no CPU path: if the shared library
is missing or cannot be loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrd.so")

TRD_OK, TRD_EINVAL, TRD_ENOMEM, TRD_EAGAIN, TRD_ETIMEOUT, TRD_ECUDA = 0, -1, -2, -3, -4, -5
ST_OK, ST_PROP_FAIL, ST_STOPPED, ST_SEED_INVALID = 0, 1, 2, 4
MAX_HYP = 8
_ERRNAMES = {-1: "TRD_EINVAL", -2: "TRD_ENOMEM", -3: "TRD_EAGAIN", -4: "TRD_ETIMEOUT", -5: "TRD_ECUDA"}

EXPORTED = [
    "trd_ctx_create", "trd_ctx_destroy", "trd_ctx_sm_count", "trd_index_build", "trd_index_free",
    "trd_index_create", "trd_index_rebuild", "trd_index_info", "trd_follow", "trd_follow_tuned",
    "trd_geometry", "trd_version", "trd_index_copy_out", "trd_batch_create", "trd_batch_run",
    "trd_batch_free", "trd_server_create", "trd_server_submit", "trd_server_poll", "trd_server_wait",
    "trd_server_stats", "trd_server_destroy", "trd_index_build_noalloc", "trd_measure_fp32_peak",
    "trd_refit", "trd_residuals", "trd_voxel_solve", "trd_follow_aligned", "trd_follow_timed",
]
TPC_ROWS, VOX_Y_BINS, VOX_Z_BINS, VOX_SUMS = 152, 15, 5, 11
N_VOXELS = 2 * 18 * TPC_ROWS * VOX_Y_BINS * VOX_Z_BINS


class TrdError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {_ERRNAMES.get(code, code)}")
        self.code = code


class Seeds(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt", "cov")] + [
        ("n", C.c_int32), ("trigger", C.c_void_p)]


class Tracklets(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("chamber", "y", "z", "dy", "vyy", "vzz", "vyz")] + [
        ("n", C.c_int32), ("trigger", C.c_void_p), ("x", C.c_void_p)]


class Alignment(C.Structure):
    _fields_ = [("chamber_x", C.c_void_p), ("bz_map", C.c_void_p), ("nr", C.c_int32), ("nz", C.c_int32),
                ("r_min", C.c_float), ("r_max", C.c_float), ("z_min", C.c_float), ("z_max", C.c_float)]


class Params(C.Structure):
    _fields_ = [("bz", C.c_float), ("n_sigma_road", C.c_float), ("chi2_cut", C.c_float),
                ("p_miss", C.c_float), ("dy_gate_sigma", C.c_float), ("n_hyp", C.c_int32),
                ("max_missing", C.c_int32), ("res_mode", C.c_int32), ("material_on", C.c_int32)]


class Launch(C.Structure):
    _fields_ = [("lanes_per_track", C.c_int32), ("block_threads", C.c_int32),
                ("min_blocks_per_sm", C.c_int32)]


class Results(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("alpha", "x", "par", "cov", "chi2", "n_trk", "n_miss",
                                          "status", "tracklet_id")]


class RefitOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("alpha", "x", "par", "cov", "chi2", "n_upd", "status")]


class States(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("alpha", "x", "par", "cov", "status")]


class TpcClusters(C.Structure):
    _fields_ = [("y", C.c_void_p), ("z", C.c_void_p), ("sector", C.c_void_p)]


class ServerCfg(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_uint64), ("max_slots", C.c_int32), ("max_queue", C.c_int32),
                ("y_bin_width", C.c_float), ("params", Params), ("launch", Launch)]


class Timing(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("gpu_ms", C.c_float), ("slot", C.c_int32), ("start_ms", C.c_float), ("inputs_ms", C.c_float),
                ("kernels_ms", C.c_float), ("results_ms", C.c_float)]


_lib = None


def lib():
    """Load libtrd.so (raises if it is absent: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtrd.so not built ({LIB_PATH}); run "
                               "`python -m paper_2003_03174_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, f32 = C.c_void_p, C.c_int32, C.c_float
        L.trd_ctx_create.argtypes = [C.c_int, C.POINTER(vp)]
        L.trd_ctx_destroy.argtypes = [vp]
        L.trd_ctx_sm_count.argtypes = [vp]
        L.trd_index_build.argtypes = [vp, C.POINTER(Tracklets), f32, vp, C.POINTER(vp)]
        L.trd_index_create.argtypes = [vp, i32, f32, C.POINTER(vp)]
        L.trd_index_rebuild.argtypes = [vp, C.POINTER(Tracklets), vp]
        L.trd_index_free.argtypes = [vp]
        L.trd_index_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.trd_follow.argtypes = [vp, C.POINTER(Seeds), vp, C.POINTER(Params), C.POINTER(Results), vp]
        L.trd_follow_tuned.argtypes = [vp, C.POINTER(Seeds), vp, C.POINTER(Params),
                                       C.POINTER(Results), vp, C.POINTER(Launch)]
        L.trd_follow_aligned.argtypes = [vp, C.POINTER(Seeds), vp, C.POINTER(Params), C.POINTER(Alignment),
                                         C.POINTER(Results), vp, C.POINTER(Launch)]
        L.trd_follow_timed.argtypes = [vp, C.POINTER(Seeds), vp, C.POINTER(Params), C.POINTER(Results), vp,
                                       C.POINTER(Launch), vp, vp]
        L.trd_geometry.argtypes = [C.POINTER(C.c_double), C.c_int]
        L.trd_index_copy_out.argtypes = [vp, vp, vp]
        L.trd_batch_create.argtypes = [vp, i32, vp, vp, C.POINTER(Seeds), C.POINTER(Tracklets),
                                       C.POINTER(Params), C.POINTER(Results), f32, C.POINTER(Launch),
                                       C.POINTER(vp)]
        L.trd_batch_run.argtypes = [vp, vp]
        L.trd_batch_free.argtypes = [vp]
        L.trd_server_create.argtypes = [vp, C.POINTER(ServerCfg), C.POINTER(vp)]
        L.trd_server_submit.argtypes = [vp, C.POINTER(Seeds), C.POINTER(Tracklets),
                                        C.POINTER(Results), C.POINTER(C.c_uint64)]
        L.trd_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(Timing)]
        L.trd_server_wait.argtypes = [vp, C.c_uint64, C.c_int32, C.POINTER(Timing)]
        L.trd_server_stats.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_uint64)]
        L.trd_server_destroy.argtypes = [vp]
        L.trd_index_build_noalloc.argtypes = [C.POINTER(Tracklets), f32, vp, vp, vp, vp]
        L.trd_measure_fp32_peak.argtypes = [vp, C.POINTER(C.c_double)]
        L.trd_refit.argtypes = [vp, C.POINTER(Results), i32, C.POINTER(Tracklets), C.POINTER(Params),
                                f32, C.POINTER(RefitOut), vp]
        L.trd_residuals.argtypes = [vp, i32, C.POINTER(States), C.POINTER(States), C.POINTER(TpcClusters), f32,
                                    vp, vp, vp]
        L.trd_voxel_solve.argtypes = [vp, vp, i32, vp, vp]
        L.trd_version.restype = C.c_char_p
        for fn in EXPORTED:
            if fn != "trd_version":
                getattr(L, fn).restype = C.c_int
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != TRD_OK:
        raise TrdError(fn, rc)


def version() -> str:
    return lib().trd_version().decode()


def geometry() -> dict:
    names = ["n_sectors", "n_stacks", "n_layers", "n_chambers", "x_layer0", "dx_layer",
             "stack_length", "z_min", "tilt_deg", "drift_length", "lorentz_deg", "c_light",
             "max_snp"]
    out = (C.c_double * len(names))()
    _check("trd_geometry", lib().trd_geometry(out, len(names)))
    return dict(zip(names, list(out)))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def params_struct(p: dict) -> Params:
    return Params(float(p["bz"]), float(p["n_sigma_road"]), float(p["chi2_cut"]),
                  float(p["p_miss"]), float(p["dy_gate_sigma"]), int(p["n_hyp"]),
                  int(p["max_missing"]), int(p["res_mode"]), int(p["material_on"]))


def seeds_struct(s: dict) -> Seeds:
    n = int(s["alpha"].shape[0])
    return Seeds(*[_ptr(s[k]) for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt", "cov")], n,
                 _ptr(s.get("trigger")))


def tracklets_struct(t: dict) -> Tracklets:
    n = int(t["chamber"].shape[0])
    return Tracklets(*[_ptr(t[k]) for k in ("chamber", "y", "z", "dy", "vyy", "vzz", "vyz")], n,
                     _ptr(t.get("trigger")), _ptr(t.get("x")))


def alignment_struct(chamber_x=None, field=None) -> Alignment:
    """chamber_x: device float [540] or None; field: dict(bz = device float
    [nz, nr], r_min, r_max, z_min, z_max) or None."""
    if field is None:
        return Alignment(_ptr(chamber_x), None, 0, 0, 0.0, 0.0, 0.0, 0.0)
    nz, nr = int(field["bz"].shape[0]), int(field["bz"].shape[1])
    return Alignment(_ptr(chamber_x), _ptr(field["bz"]), nr, nz, float(field["r_min"]), float(field["r_max"]),
                     float(field["z_min"]), float(field["z_max"]))


def alloc_results(n: int, device="cuda"):
    import torch
    f = dict(dtype=torch.float32, device=device)
    i = dict(dtype=torch.int32, device=device)
    return dict(alpha=torch.empty(n, **f), x=torch.empty(n, **f), par=torch.empty(5, n, **f),
                cov=torch.empty(15, n, **f), chi2=torch.empty(n, **f), n_trk=torch.empty(n, **i),
                n_miss=torch.empty(n, **i), status=torch.empty(n, **i),
                tracklet_id=torch.empty(6, n, **i))


def results_struct(r: dict) -> Results:
    return Results(*[_ptr(r[k]) for k in ("alpha", "x", "par", "cov", "chi2", "n_trk", "n_miss",
                                          "status", "tracklet_id")])


def alloc_refit(n: int, device="cuda"):
    import torch
    f = dict(dtype=torch.float32, device=device)
    i = dict(dtype=torch.int32, device=device)
    return dict(alpha=torch.empty(n, **f), x=torch.empty(n, **f), par=torch.empty(5, n, **f),
                cov=torch.empty(15, n, **f), chi2=torch.empty(n, **f), n_upd=torch.empty(n, **i),
                status=torch.empty(n, **i))


def to_device(arrays: dict, device="cuda") -> dict:
    """Copy a dict of numpy arrays to contiguous device tensors."""
    import torch
    return {k: torch.from_numpy(v).contiguous().to(device) for k, v in arrays.items()}


class Index:
    """A device-resident tracklet index owned by the library."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, keep=None):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep  # the input tensors must outlive the asynchronous build

    def rebuild(self, tracklets: dict, stream=None):
        ts = tracklets_struct(tracklets)
        _check("trd_index_rebuild", lib().trd_index_rebuild(self.handle, C.byref(ts),
                                                            _stream_handle(stream)))
        self._keep = tracklets

    def info(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check("trd_index_info", lib().trd_index_info(self.handle, C.byref(a), C.byref(b),
                                                      C.byref(c)))
        return dict(n_indexed=a.value, n_rejected=b.value, n_buckets=c.value)

    def copy_out(self):
        """(offsets, ids) as numpy arrays (synchronises)."""
        import numpy as np
        info = self.info()
        off = np.zeros(info["n_buckets"] + 1, np.int32)
        ids = np.zeros(max(info["n_indexed"], 1), np.int32)
        _check("trd_index_copy_out", lib().trd_index_copy_out(
            self.handle, off.ctypes.data_as(C.c_void_p), ids.ctypes.data_as(C.c_void_p)))
        return off, ids[:info["n_indexed"]]

    def free(self):
        if self.handle:
            lib().trd_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _hptr(a):
    """Host pointer of a numpy array or a CPU (possibly pinned) torch tensor."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


_RESULT_ROWS = (("alpha", 1, "f"), ("x", 1, "f"), ("par", 5, "f"), ("cov", 15, "f"), ("chi2", 1, "f"),
                ("n_trk", 1, "i"), ("n_miss", 1, "i"), ("status", 1, "i"), ("tracklet_id", 6, "i"))


def _pinned_views(block, rows, n):
    """Views of one pinned int32 block: (name, rows, 'f' | 'i') in order."""
    import torch
    out, o = {}, 0
    for name, r, kind in rows:
        v = block[o:o + r * n]
        v = v.view(torch.float32) if kind == "f" else v
        out[name] = v.view(r, n) if r > 1 else v
        o += r * n
    return out


def host_results(n: int, pinned: bool = False):
    """Host result arrays (numpy, or views of one pinned block in the order
    the server copies them back, so each request's results come in one copy)."""
    if pinned:
        import torch
        block = torch.empty(32 * n, dtype=torch.int32, pin_memory=True)
        return _pinned_views(block, _RESULT_ROWS, n)
    import numpy as np
    f, i = np.float32, np.int32
    return dict(alpha=np.empty(n, f), x=np.empty(n, f), par=np.empty((5, n), f), cov=np.empty((15, n), f),
                chi2=np.empty(n, f), n_trk=np.empty(n, i), n_miss=np.empty(n, i), status=np.empty(n, i),
                tracklet_id=np.empty((6, n), i))


def pinned_inputs(seeds: dict, tracklets: dict, pin: bool = True):
    """A timeframe's host inputs copied into one (pinned) block in the order
    the server copies them to the device (seeds, tracklets, interaction ids of
    seeds and tracklets, tracklet radii), so each request's inputs go in one
    copy.  Returns (seeds, tracklets) dicts of views into the block."""
    import numpy as np
    import torch
    n, m = len(seeds["alpha"]), len(tracklets["chamber"])
    srows = [(k, 1, "f") for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt")] + [("cov", 15, "f")]
    trows = [("chamber", 1, "i")] + [(k, 1, "f") for k in ("y", "z", "dy", "vyy", "vzz", "vyz")]
    words = 22 * n + 7 * m + (n if "trigger" in seeds else 0) + \
        (m if "trigger" in tracklets else 0) + (m if "x" in tracklets else 0)
    block = torch.empty(words, dtype=torch.int32, pin_memory=pin)
    hs = _pinned_views(block[:22 * n], srows, n)
    ht = _pinned_views(block[22 * n:22 * n + 7 * m], trows, m)
    o = 22 * n + 7 * m
    if "trigger" in seeds:
        hs["trigger"] = block[o:o + n]
        o += n
    if "trigger" in tracklets:
        ht["trigger"] = block[o:o + m]
        o += m
    if "x" in tracklets:
        ht["x"] = block[o:o + m].view(torch.float32)
        o += m
    for src, dst in ((seeds, hs), (tracklets, ht)):
        for k, v in dst.items():
            v.copy_(torch.from_numpy(np.ascontiguousarray(src[k])).reshape(v.shape))
    return hs, ht


class Server:
    """Serving loop (trd_server_t): submit host timeframes, poll tickets."""

    def __init__(self, ctx: "Context", params: dict, mem_budget_bytes: int = 0, max_slots: int = 0,
                 max_queue: int = 0, y_bin_width: float = 0.0, lanes_per_track: int = 0,
                 block_threads: int = 0, min_blocks_per_sm: int = 0):
        cfg = ServerCfg(int(mem_budget_bytes), int(max_slots), int(max_queue), float(y_bin_width),
                        params_struct(params),
                        Launch(int(lanes_per_track), int(block_threads), int(min_blocks_per_sm)))
        h = C.c_void_p()
        _check("trd_server_create", lib().trd_server_create(ctx.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self.ctx = ctx
        self._live = {}

    def submit(self, seeds: dict, tracklets: dict, results: dict) -> int:
        n = int(seeds["alpha"].shape[0])
        m = int(tracklets["chamber"].shape[0])
        ss = Seeds(*[_hptr(seeds[k]) for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt", "cov")], n,
                   _hptr(seeds["trigger"]) if seeds.get("trigger") is not None else None)
        ts = Tracklets(*[_hptr(tracklets[k]) for k in ("chamber", "y", "z", "dy", "vyy", "vzz", "vyz")], m,
                       _hptr(tracklets["trigger"]) if tracklets.get("trigger") is not None else None,
                       _hptr(tracklets["x"]) if tracklets.get("x") is not None else None)
        rs = Results(*[_hptr(results[k]) for k in ("alpha", "x", "par", "cov", "chi2", "n_trk",
                                                   "n_miss", "status", "tracklet_id")])
        t = C.c_uint64()
        _check("trd_server_submit", lib().trd_server_submit(self.handle, C.byref(ss), C.byref(ts),
                                                            C.byref(rs), C.byref(t)))
        self._live[t.value] = (seeds, tracklets, results)
        return t.value

    def _done(self, fn, ticket, rc, tm):
        if rc == TRD_EAGAIN or rc == TRD_ETIMEOUT:
            return None
        self._live.pop(ticket, None)
        _check(fn, rc)
        return dict(submit_s=tm.submit_s, admit_s=tm.admit_s, done_s=tm.done_s, gpu_ms=tm.gpu_ms,
                    slot=tm.slot, start_ms=tm.start_ms, inputs_ms=tm.inputs_ms, kernels_ms=tm.kernels_ms,
                    results_ms=tm.results_ms)

    def poll(self, ticket: int):
        """Timing dict when finished, None while pending (raises on failure)."""
        tm = Timing()
        rc = lib().trd_server_poll(self.handle, C.c_uint64(ticket), C.byref(tm))
        return self._done("trd_server_poll", ticket, rc, tm)

    def wait(self, ticket: int, timeout_ms: int = 60_000):
        """Timing dict, or None if the bounded host wait ran out."""
        tm = Timing()
        rc = lib().trd_server_wait(self.handle, C.c_uint64(ticket), int(timeout_ms), C.byref(tm))
        return self._done("trd_server_wait", ticket, rc, tm)

    def stats(self):
        q, f, b = C.c_int32(), C.c_int32(), C.c_uint64()
        _check("trd_server_stats", lib().trd_server_stats(self.handle, C.byref(q), C.byref(f), C.byref(b)))
        return dict(queued=q.value, in_flight=f.value, device_bytes=b.value)

    def close(self):
        if self.handle:
            lib().trd_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many timeframes followed by one CUDA-graph replay (trd_batch_t)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep  # bound device buffers must outlive the graph

    def run(self, stream=None):
        _check("trd_batch_run", lib().trd_batch_run(self.handle, _stream_handle(stream)))

    def free(self):
        if self.handle:
            lib().trd_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """Binds one CUDA device (trd_ctx_t)."""

    def __init__(self, device: int = 0):
        import torch
        torch.cuda.init()
        h = C.c_void_p()
        _check("trd_ctx_create", lib().trd_ctx_create(int(device), C.byref(h)))
        self.handle = h
        self.device = device

    def fp32_peak_tflops(self) -> float:
        v = C.c_double()
        _check("trd_measure_fp32_peak", lib().trd_measure_fp32_peak(self.handle, C.byref(v)))
        return v.value

    @property
    def sm_count(self) -> int:
        return lib().trd_ctx_sm_count(self.handle)

    def index_build(self, tracklets: dict, y_bin_width: float = 0.0, stream=None) -> Index:
        ts = tracklets_struct(tracklets)
        h = C.c_void_p()
        _check("trd_index_build", lib().trd_index_build(self.handle, C.byref(ts),
                                                        float(y_bin_width),
                                                        _stream_handle(stream), C.byref(h)))
        return Index(self, h, keep=tracklets)

    def index_create(self, capacity: int, y_bin_width: float = 0.0) -> Index:
        h = C.c_void_p()
        _check("trd_index_create", lib().trd_index_create(self.handle, int(capacity),
                                                          float(y_bin_width), C.byref(h)))
        return Index(self, h)

    def follow(self, seeds: dict, index: Index, params: dict, results: dict | None = None,
               stream=None, lanes_per_track: int = 0, block_threads: int = 0,
               min_blocks_per_sm: int = 0, chamber_x=None, field=None, kernel_events=None) -> dict:
        """trd_follow (trd_follow_tuned with a launch shape; trd_follow_aligned
        with chamber radii and/or a field map, see alignment_struct;
        trd_follow_timed with kernel_events = (start, end), two
        torch.cuda.Event(enable_timing=True) that have been recorded once, so
        that their CUDA events exist)."""
        n = int(seeds["alpha"].shape[0])
        if results is None:
            results = alloc_results(n, device=seeds["alpha"].device)
        ss, ps, rs = seeds_struct(seeds), params_struct(params), results_struct(results)
        if kernel_events is not None and (chamber_x is not None or field is not None):
            raise ValueError("kernel_events: the timed entry point takes no alignment")
        if chamber_x is not None or field is not None:
            al = alignment_struct(chamber_x, field)
            ln = Launch(int(lanes_per_track), int(block_threads), int(min_blocks_per_sm))
            rc = lib().trd_follow_aligned(self.handle, C.byref(ss), index.handle, C.byref(ps), C.byref(al),
                                          C.byref(rs), _stream_handle(stream), C.byref(ln))
            _check("trd_follow_aligned", rc)
            return results
        if kernel_events is not None:
            ev0, ev1 = (C.c_void_p(int(e.cuda_event)) for e in kernel_events)
            if not ev0.value or not ev1.value:
                raise ValueError("kernel_events: record each event once first (it is created lazily)")
            ln = Launch(int(lanes_per_track), int(block_threads), int(min_blocks_per_sm))
            rc = lib().trd_follow_timed(self.handle, C.byref(ss), index.handle, C.byref(ps), C.byref(rs),
                                        _stream_handle(stream), C.byref(ln), ev0, ev1)
            _check("trd_follow_timed", rc)
            return results
        if lanes_per_track or block_threads or min_blocks_per_sm:
            ln = Launch(int(lanes_per_track), int(block_threads), int(min_blocks_per_sm))
            rc = lib().trd_follow_tuned(self.handle, C.byref(ss), index.handle, C.byref(ps),
                                        C.byref(rs), _stream_handle(stream), C.byref(ln))
            _check("trd_follow_tuned", rc)
        else:
            rc = lib().trd_follow(self.handle, C.byref(ss), index.handle, C.byref(ps),
                                  C.byref(rs), _stream_handle(stream))
            _check("trd_follow", rc)
        return results

    def refit(self, tracks: dict, tracklets: dict, params: dict, cov_scale: float = 100.0,
              out: dict | None = None, stream=None) -> dict:
        """TRD-only refit (trd_refit) of the follower's results `tracks`
        against the device tracklet arrays their ids refer to."""
        n = int(tracks["alpha"].shape[0])
        if out is None:
            out = alloc_refit(n, device=tracks["alpha"].device)
        rs = results_struct(tracks)
        ts, ps = tracklets_struct(tracklets), params_struct(params)
        os_ = RefitOut(*[_ptr(out[k]) for k in ("alpha", "x", "par", "cov", "chi2", "n_upd", "status")])
        rc = lib().trd_refit(self.handle, C.byref(rs), n, C.byref(ts), C.byref(ps), float(cov_scale),
                             C.byref(os_), _stream_handle(stream))
        _check("trd_refit", rc)
        return out

    def residuals(self, its: dict, trd: dict, clusters: dict, bz: float, sums=None,
                  cluster_res: bool = False, stream=None):
        """Accumulate the residuals of the tracks' TPC clusters into the voxel
        sums (trd_residuals; int64 [N_VOXELS, 11], zeroed here when not
        given).  Returns the sums, and with cluster_res the per-cluster
        (dy, dz, t, u) float [4, 152, n]."""
        import torch
        n = int(its["alpha"].shape[0])
        dev = its["alpha"].device
        if sums is None:
            sums = torch.zeros(N_VOXELS, VOX_SUMS, dtype=torch.int64, device=dev)
        res = torch.empty(4, TPC_ROWS, n, dtype=torch.float32, device=dev) if cluster_res else None
        st = [States(*[_ptr(d[k]) for k in ("alpha", "x", "par", "cov", "status")]) for d in (its, trd)]
        cl = TpcClusters(_ptr(clusters["y"]), _ptr(clusters["z"]), _ptr(clusters["sector"]))
        rc = lib().trd_residuals(self.handle, n, C.byref(st[0]), C.byref(st[1]), C.byref(cl), float(bz),
                                 _ptr(sums), _ptr(res), _stream_handle(stream))
        _check("trd_residuals", rc)
        return (sums, res) if cluster_res else sums

    def voxel_solve(self, sums, min_count: int = 10, out=None, stream=None):
        """Distortion vector per voxel (trd_voxel_solve): float [N_VOXELS, 6]
        = Dx, Dy, Dz, n, rms dy, rms dz."""
        import torch
        if out is None:
            out = torch.empty(N_VOXELS, 6, dtype=torch.float32, device=sums.device)
        rc = lib().trd_voxel_solve(self.handle, _ptr(sums), int(min_count), _ptr(out), _stream_handle(stream))
        _check("trd_voxel_solve", rc)
        return out

    def batch_create(self, seeds: dict, tracklets: dict, seed_offsets, tracklet_offsets,
                     params: dict, results: dict, y_bin_width: float = 0.0,
                     lanes_per_track: int = 0, block_threads: int = 0,
                     min_blocks_per_sm: int = 0) -> Batch:
        import numpy as np
        so = np.ascontiguousarray(np.asarray(seed_offsets, dtype=np.int32))
        to = np.ascontiguousarray(np.asarray(tracklet_offsets, dtype=np.int32))
        n_tf = int(so.shape[0]) - 1
        ss, ts = seeds_struct(seeds), tracklets_struct(tracklets)
        ps, rs = params_struct(params), results_struct(results)
        ln = Launch(int(lanes_per_track), int(block_threads), int(min_blocks_per_sm))
        h = C.c_void_p()
        _check("trd_batch_create", lib().trd_batch_create(
            self.handle, n_tf, so.ctypes.data_as(C.c_void_p), to.ctypes.data_as(C.c_void_p),
            C.byref(ss), C.byref(ts), C.byref(ps), C.byref(rs), float(y_bin_width), C.byref(ln),
            C.byref(h)))
        return Batch(h, keep=(seeds, tracklets, results))

    def close(self):
        if self.handle:
            lib().trd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
