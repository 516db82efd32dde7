"""ctypes front end of the FP64 oracle (test infrastructure only).

Each function wraps one entry point of trd_oracle.c; see that file for the
passage of the paper each one follows.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None
_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
STATUS_PROP_FAIL, STATUS_STOPPED, STATUS_SEED_INVALID = 1, 2, 4


class use_library:
    """Run the wrappers against another build of trd_oracle.c (tests that plant
    a mistake in a copy of the oracle use this)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def _load(path):
    if True:
        L = C.CDLL(path)
        L.ora_propagate.argtypes = [_d, _d, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.ora_propagate.restype = C.c_int
        L.ora_rotate.argtypes = [_d, _d, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.ora_rotate.restype = C.c_int
        L.ora_material.argtypes = [_d, _d]
        L.ora_material_inward.argtypes = [_d, _d]
        L.ora_material.restype = C.c_int
        L.ora_bethe.argtypes = [C.c_double]
        L.ora_bethe.restype = C.c_double
        L.ora_bethe_dbg.argtypes = [C.c_double]
        L.ora_bethe_dbg.restype = C.c_double
        L.ora_highland.argtypes = [C.c_double, C.c_double, C.c_double]
        L.ora_highland.restype = C.c_double
        L.ora_update.argtypes = [_d, _d, C.c_int, _d, C.c_int]
        L.ora_update.restype = C.c_double
        L.ora_chi2.argtypes = [_d, _d, C.c_int, _d]
        L.ora_chi2.restype = C.c_double
        L.ora_cov_is_pd.argtypes = [_d]
        L.ora_cov_is_pd.restype = C.c_int
        L.ora_constants.argtypes = [_d, C.c_int]
        L.ora_constants.restype = None
        L.ora_follow.restype = C.c_int
        L.ora_refit.restype = C.c_int
        L.ora_propagate_map.restype = C.c_int
        L.ora_voxel_of.argtypes = [C.c_float, C.c_float, C.c_int, C.c_int]
        L.ora_voxel_of.restype = C.c_int
        L.ora_residuals.restype = C.c_int
        L.ora_voxel_solve.restype = C.c_int
        L.ora_to_layer.argtypes = [_d, _d, C.c_void_p, C.c_int, _d, _i, C.c_void_p]
        L.ora_to_layer.restype = C.c_int
        L.ora_candidates.argtypes = [_d, _d, C.c_int, C.c_int, C.c_int, _i, _f, _f, _f, _f, _f,
                                     _f, _d, _i, C.c_int, _i, _d]
        L.ora_candidates.restype = C.c_int
        return L


def _vec(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).copy())
    assert a.shape == (n,)
    return a


def propagate(st, cov, x_to, bz, with_cov=True):
    """Helix transport to radius x_to.  Returns (ok, st, cov, J[5,5])."""
    s, c = _vec(st, 7), _vec(cov, 15)
    J = np.zeros(25)
    ok = lib().ora_propagate(s, c, float(x_to), float(bz), J.ctypes.data, None) == 0
    return ok, s, c, J.reshape(5, 5)


def rotate(st, cov, alpha_new, bz):
    """Rotation into the frame of azimuth alpha_new.  Returns (ok, st, cov, J)."""
    s, c = _vec(st, 7), _vec(cov, 15)
    J = np.zeros(25)
    ok = lib().ora_rotate(s, c, float(alpha_new), float(bz), J.ctypes.data, None) == 0
    return ok, s, c, J.reshape(5, 5)


def material(st, cov):
    s, c = _vec(st, 7), _vec(cov, 15)
    ok = lib().ora_material(s, c) == 0
    return ok, s, c


def material_inward(st, cov):
    """The material step of a track moving inward (energy loss added back)."""
    s, c = _vec(st, 7), _vec(cov, 15)
    ok = lib().ora_material_inward(s, c) == 0
    return ok, s, c


def propagate_map(st, cov, x_to, bz, field=None):
    """One transport step with the field map's midpoint field (the
    follower's step when a map is given).  Returns (ok, st, cov)."""
    s_, c_ = _vec(st, 7), _vec(cov, 15)
    if field is not None:
        fb = _f32(field["bz"])
        box = np.array([field["r_min"], field["r_max"], field["z_min"], field["z_max"]], dtype=np.float64)
        ok = lib().ora_propagate_map(s_.ctypes.data_as(C.c_void_p), c_.ctypes.data_as(C.c_void_p),
                                     C.c_double(x_to), C.c_double(bz), fb.ctypes.data_as(C.c_void_p),
                                     C.c_int(fb.shape[1]), C.c_int(fb.shape[0]), box.ctypes.data_as(C.c_void_p)) == 0
    else:
        ok = lib().ora_propagate_map(s_.ctypes.data_as(C.c_void_p), c_.ctypes.data_as(C.c_void_p),
                                     C.c_double(x_to), C.c_double(bz), None, C.c_int(0), C.c_int(0), None) == 0
    return ok, s_, c_


def bethe(bg: float) -> float:
    return lib().ora_bethe(float(bg))


def bethe_dbg(bg: float) -> float:
    """Slope of the Bethe curve, d(dE/dx)/d(beta gamma), MeV cm^2/g."""
    return lib().ora_bethe_dbg(float(bg))


def highland(p: float, beta: float, xx0: float) -> float:
    return lib().ora_highland(float(p), float(beta), float(xx0))


def update(st, cov, layer, meas, joseph=False):
    """Kalman update with meas = (y_tl, z_tl, vyy, vzz, vyz).  Returns (chi2, st, cov)."""
    s, c = _vec(st, 7), _vec(cov, 15)
    chi2 = lib().ora_update(s, c, int(layer), _vec(meas, 5), int(bool(joseph)))
    return chi2, s, c


def chi2(st, cov, layer, meas):
    return lib().ora_chi2(_vec(st, 7), _vec(cov, 15), int(layer), _vec(meas, 5))


def cov_is_pd(cov) -> bool:
    return bool(lib().ora_cov_is_pd(_vec(cov, 15)))


def constants() -> dict:
    names = ["n_sectors", "n_stacks", "n_layers", "n_chambers", "x_layer0", "dx_layer",
             "stack_length", "z_min", "tilt_deg", "drift_length", "lorentz_deg", "c_light",
             "max_snp"]
    out = np.zeros(len(names))
    lib().ora_constants(out, len(names))
    return dict(zip(names, out.tolist()))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def follow(seeds: dict, tracklets: dict, params: dict, seed_index=None, brute=False,
           n_threads=0, chamber_x=None, field=None) -> dict:
    """Run the FP64 follower.  seeds/tracklets are the FP32 input arrays
    (the same ones the library reads).  Returns numpy arrays keyed like the
    library's results, plus 'margin' [6, n] and 'nroad' [6, n]."""
    L = lib()
    n = int(seeds["alpha"].shape[0])
    m = int(tracklets["chamber"].shape[0])
    if seed_index is None:
        n_out, sidx = n, None
    else:
        sidx = np.ascontiguousarray(np.asarray(seed_index, dtype=np.int32))
        n_out = int(sidx.shape[0])
    cov = _f32(seeds["cov"]).reshape(15, n)
    pd = np.array([params["bz"], params["n_sigma_road"], params["chi2_cut"], params["p_miss"],
                   params["dy_gate_sigma"]], dtype=np.float64)
    pi = np.array([params["n_hyp"], params["max_missing"], params["res_mode"],
                   params["material_on"]], dtype=np.int32)
    st = np.zeros((7, n_out))
    cv = np.zeros((15, n_out))
    chi2_ = np.zeros(n_out)
    ntrk = np.zeros(n_out, np.int32)
    nmiss = np.zeros(n_out, np.int32)
    status = np.zeros(n_out, np.int32)
    ids = np.zeros((6, n_out), np.int32)
    margin = np.zeros((6, n_out))
    nroad = np.zeros((6, n_out), np.int32)
    keep = [_f32(seeds[k]) for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt")]
    tk = [np.ascontiguousarray(np.asarray(tracklets["chamber"], dtype=np.int32))] + [
        _f32(tracklets[k]) for k in ("y", "z", "dy", "vyy", "vzz", "vyz")]
    args = [C.c_int(n)] + [a.ctypes.data_as(C.c_void_p) for a in keep] + [
        cov.ctypes.data_as(C.c_void_p), C.c_int(m)] + [a.ctypes.data_as(C.c_void_p) for a in tk] + [
        pd.ctypes.data_as(C.c_void_p), pi.ctypes.data_as(C.c_void_p), C.c_int(n_out),
        sidx.ctypes.data_as(C.c_void_p) if sidx is not None else None, C.c_int(int(brute)),
        C.c_int(n_threads)] + [a.ctypes.data_as(C.c_void_p) for a in
                               (st, cv, chi2_, ntrk, nmiss, status, ids, margin, nroad)]
    trig = [np.ascontiguousarray(np.asarray(d["trigger"], dtype=np.int32)) if d.get("trigger") is not None
            else None for d in (seeds, tracklets)]
    args += [t.ctypes.data_as(C.c_void_p) if t is not None else None for t in trig]
    # misalignment and field map (Sec. 3): per-tracklet radius, per-chamber
    # average radius, Bz map = dict(bz [nz, nr], r_min, r_max, z_min, z_max)
    tx = _f32(tracklets["x"]) if tracklets.get("x") is not None else None
    cx = _f32(chamber_x) if chamber_x is not None else None
    if field is not None:
        fb = _f32(field["bz"])
        box = np.array([field["r_min"], field["r_max"], field["z_min"], field["z_max"]], dtype=np.float64)
        fargs = [fb.ctypes.data_as(C.c_void_p), C.c_int(fb.shape[1]), C.c_int(fb.shape[0]),
                 box.ctypes.data_as(C.c_void_p)]
    else:
        fargs = [None, C.c_int(0), C.c_int(0), None]
    args += [tx.ctypes.data_as(C.c_void_p) if tx is not None else None,
             cx.ctypes.data_as(C.c_void_p) if cx is not None else None] + fargs
    rc = L.ora_follow(*args)
    if rc != 0:
        raise ValueError(f"ora_follow rejected its arguments ({rc})")
    return dict(alpha=st[0], x=st[1], par=st[2:7], cov=cv, chi2=chi2_, n_trk=ntrk,
                n_miss=nmiss, status=status, tracklet_id=ids, margin=margin, nroad=nroad)


def refit(results: dict, tracklets: dict, params: dict, cov_scale: float = 100.0,
          n_threads=0) -> dict:
    """Run the FP64 TRD-only refit (Sec. 2, step 3) on the follower's results.

    results: arrays in the library's result layout (alpha, x [n]; par [5, n];
    cov [15, n]; status [n]; tracklet_id [6, n]), taken as FP32 like the
    library reads them.  Returns alpha, x, par, cov, chi2, n_upd, status."""
    L = lib()
    n = int(np.asarray(results["alpha"]).shape[0])
    m = int(tracklets["chamber"].shape[0])
    a = [_f32(results["alpha"]), _f32(results["x"]), _f32(results["par"]).reshape(5, n),
         _f32(results["cov"]).reshape(15, n)]
    st_in = np.ascontiguousarray(np.asarray(results["status"], dtype=np.int32))
    ids = np.ascontiguousarray(np.asarray(results["tracklet_id"], dtype=np.int32).reshape(6, n))
    tk = [np.ascontiguousarray(np.asarray(tracklets["chamber"], dtype=np.int32))] + [
        _f32(tracklets[k]) for k in ("y", "z", "vyy", "vzz", "vyz")]
    pd, pi = _params_arrays(params)
    st = np.zeros((7, n))
    cv = np.zeros((15, n))
    chi2_ = np.zeros(n)
    nupd = np.zeros(n, np.int32)
    status = np.zeros(n, np.int32)
    margin = np.zeros(n)
    ptr = lambda v: v.ctypes.data_as(C.c_void_p)  # noqa: E731
    rc = L.ora_refit(C.c_int(n), *[ptr(v) for v in a], ptr(st_in), ptr(ids), C.c_int(m),
                     *[ptr(v) for v in tk], ptr(pd), ptr(pi), C.c_double(cov_scale),
                     C.c_int(n_threads), ptr(st), ptr(cv), ptr(chi2_), ptr(nupd), ptr(status),
                     ptr(margin), ptr(_f32(tracklets["x"])) if tracklets.get("x") is not None else None)
    if rc != 0:
        raise ValueError(f"ora_refit rejected its arguments ({rc})")
    return dict(alpha=st[0], x=st[1], par=st[2:7], cov=cv, chi2=chi2_, n_upd=nupd, status=status,
                margin=margin)


N_TPC_ROWS = 152
N_VOXELS = 36 * 152 * 15 * 5
N_VOX_SUMS = 11


def voxel_of(y, z, sector, row) -> int:
    return int(lib().ora_voxel_of(C.c_float(y), C.c_float(z), int(sector), int(row)))


def residuals(its: dict, trd: dict, clusters: dict, bz: float, sums=None, with_clusters=False,
              n_threads=0) -> dict:
    """FP64 residual collection (Sec. 2, step 4).  its/trd: refit states in
    the library's layout (alpha, x, par, cov, status); clusters: y, z [152, n]
    float32 and sector [152, n] int8.  Returns the voxel sums [N_VOXELS, 11]
    (added to `sums` when given), their absolute-value twins, and with
    with_clusters the per-cluster dy, dz, t, u [4, 152, n], voxel [152, n],
    combined variances [2, 152, n] and per-track slack."""
    L = lib()
    n = int(np.asarray(its["alpha"]).shape[0])
    st = []
    for d in (its, trd):
        st += [_f32(d["alpha"]), _f32(d["x"]), _f32(d["par"]).reshape(5, n), _f32(d["cov"]).reshape(15, n),
               np.ascontiguousarray(np.asarray(d["status"], dtype=np.int32))]
    cy, cz = _f32(clusters["y"]).reshape(N_TPC_ROWS, n), _f32(clusters["z"]).reshape(N_TPC_ROWS, n)
    cs = np.ascontiguousarray(np.asarray(clusters["sector"], dtype=np.int8).reshape(N_TPC_ROWS, n))
    S = np.zeros((N_VOXELS, N_VOX_SUMS)) if sums is None else sums
    A = np.zeros((N_VOXELS, N_VOX_SUMS))
    ptr = lambda v: v.ctypes.data_as(C.c_void_p)  # noqa: E731
    extra = [None, None, None, None]
    if with_clusters:
        res = np.zeros((4, N_TPC_ROWS, n), np.float32)
        vox = np.zeros((N_TPC_ROWS, n), np.int32)
        var = np.zeros((2, N_TPC_ROWS, n), np.float32)
        slack = np.zeros(n)
        extra = [ptr(res), ptr(vox), ptr(var), ptr(slack)]
    rc = L.ora_residuals(C.c_int(n), *[ptr(v) for v in st], ptr(cy), ptr(cz), ptr(cs), C.c_double(bz),
                         C.c_int(n_threads), ptr(S), ptr(A), *extra)
    if rc != 0:
        raise ValueError(f"ora_residuals rejected its arguments ({rc})")
    out = dict(sums=S, abs_sums=A)
    if with_clusters:
        out.update(res=res, vox=vox, var=var, slack=slack)
    return out


def voxel_solve(sums, min_count=1) -> np.ndarray:
    """Distortion vector per voxel (Sec. 2, step 5): [N, 6] = Dx, Dy, Dz, n,
    rms dy, rms dz (NaN where undetermined)."""
    S = np.ascontiguousarray(np.asarray(sums, dtype=np.float64))
    nv = S.shape[0]
    out = np.zeros((nv, 6))
    rc = lib().ora_voxel_solve(S.ctypes.data_as(C.c_void_p), C.c_int(nv), C.c_int(min_count),
                               out.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise ValueError("ora_voxel_solve rejected its arguments")
    return out


def to_layer(st, cov, sector, layer, params):
    """Carry a state to the plane of `layer` (transport, sector change,
    material).  Returns (ok, st, cov, sector, chamber)."""
    s, c = _vec(st, 7), _vec(cov, 15)
    sec = C.c_int(int(sector))
    ch = C.c_int(-1)
    pd, pi = _params_arrays(params)
    ok = lib().ora_to_layer(s, c, C.byref(sec), int(layer), pd, pi, C.byref(ch)) == 0
    return ok, s, c, sec.value, ch.value


def candidates(st, cov, layer, chamber, tracklets, params, max_out=4096):
    """Accepted tracklets (input ids, chi2) of `chamber` for a state at `layer`."""
    tk = [np.ascontiguousarray(np.asarray(tracklets["chamber"], dtype=np.int32))] + [
        _f32(tracklets[k]) for k in ("y", "z", "dy", "vyy", "vzz", "vyz")]
    pd, pi = _params_arrays(params)
    ids = np.zeros(max_out, np.int32)
    ch2 = np.zeros(max_out)
    n = lib().ora_candidates(_vec(st, 7), _vec(cov, 15), int(layer), int(chamber),
                             int(tk[0].shape[0]), *tk, pd, pi, max_out, ids, ch2)
    n = min(n, max_out)
    return ids[:n].copy(), ch2[:n].copy()


def _params_arrays(params):
    pd = np.array([params["bz"], params["n_sigma_road"], params["chi2_cut"], params["p_miss"],
                   params["dy_gate_sigma"]], dtype=np.float64)
    pi = np.array([params["n_hyp"], params["max_missing"], params["res_mode"],
                   params["material_on"]], dtype=np.int32)
    return pd, pi


__all__ = ["use_library", "propagate", "rotate", "material", "bethe", "bethe_dbg", "highland", "update", "chi2",
           "cov_is_pd", "constants", "follow", "refit", "to_layer", "candidates", "lib",
           "material_inward", "propagate_map", "residuals", "voxel_solve", "voxel_of", "N_VOXELS", "N_TPC_ROWS"]
