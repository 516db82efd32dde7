"""Comparison of the CUDA follower's results with the FP64 oracle.

Tolerances (per track):
  * track parameters: |gpu - oracle| <= 1e-4 * max(|oracle|, sigma), sigma the
    oracle's sqrt(C_ii) (a parameter near zero is judged on its own scale);
  * chi2: within 1e-3 absolute;
  * covariance: |dC_ij| <= 1e-3 * sqrt(C_ii C_jj) (FP32 transport and Joseph
    update carry ~1e-6 relative per step; 1e-3 leaves room for 6 layers);
  * tracklet ids, counts and status identical, except where the oracle's
    smallest decision margin up to the first differing layer is below 1e-3
    (a near tie of chi2 against the cut or the runner-up, of a road or dy-gate
    boundary in sigma, of a sector edge or stack boundary in cm, or of the
    sin(phi) limit).  Such a track is exempt from the rest of the comparison.
  * a track with the same ids, counts and status whose other results are
    outside the tolerances is exempt too when the oracle's smallest margin
    over its layers is below 1e-3: a near tie can move the state without
    changing which tracklets are attached (with misaligned chambers, a
    hypothesis found inside a stack is carried on to the chamber's radius,
    one just outside is not, and both then miss the layer).
"""
from __future__ import annotations

import numpy as np

MARGIN = 1e-3
PAR_REL = 1e-4
CHI2_ABS = 1e-3
COV_REL = 1e-3


def to_numpy(res: dict) -> dict:
    out = {}
    for k, v in res.items():
        out[k] = v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)
    return out


def compare(gpu: dict, ora: dict, sel=None, max_exempt_frac=0.02) -> dict:
    """gpu: numpy results of the library (full arrays); ora: oracle results for
    the seeds `sel` (indices into gpu arrays; None = all).  Returns a report
    and raises AssertionError listing the first failures."""
    n = ora["chi2"].shape[0]
    idx = np.arange(n) if sel is None else np.asarray(sel)
    g = {k: (v[..., idx] if v.ndim > 0 else v) for k, v in gpu.items()}
    ids_eq = g["tracklet_id"] == ora["tracklet_id"]  # [6, n]
    same_path = ids_eq.all(0) & (g["status"] == ora["status"]) & (g["n_trk"] == ora["n_trk"]) & (
        g["n_miss"] == ora["n_miss"])
    first = np.where(ids_eq.all(0), 5, np.argmax(~ids_eq, axis=0))
    cm = np.minimum.accumulate(ora["margin"], axis=0)  # min margin over layers <= l
    margin_at = cm[first, np.arange(n)]
    sig = np.sqrt(np.maximum(ora["cov"][[0, 2, 5, 9, 14]], 0.0))
    scale = np.maximum(np.abs(ora["par"]), sig)
    par_err = np.abs(g["par"] - ora["par"]) / np.maximum(scale, 1e-30)
    chi2_err = np.abs(g["chi2"] - ora["chi2"])
    d = np.sqrt(np.maximum(ora["cov"][[0, 2, 5, 9, 14]], 1e-30))
    cov_scale = np.empty_like(ora["cov"])
    k = 0
    for i in range(5):
        for j in range(i + 1):
            cov_scale[k] = d[i] * d[j]
            k += 1
    cov_err = np.abs(g["cov"] - ora["cov"]) / cov_scale
    x_err = np.abs(g["x"] - ora["x"])
    a_err = np.abs(np.angle(np.exp(1j * (g["alpha"].astype(np.float64) - ora["alpha"]))))
    off_par = par_err.max(0) > PAR_REL
    off_chi2 = chi2_err > CHI2_ABS
    off_cov = cov_err.max(0) > COV_REL
    off_geo = (x_err > 1e-4 * np.abs(ora["x"])) | (a_err > 1e-6)
    off = off_par | off_chi2 | off_cov | off_geo
    exempt = (~same_path | off) & (margin_at < MARGIN)
    bad_path = ~same_path & ~exempt
    chk = same_path & ~exempt
    bad_par = chk & off_par
    bad_chi2 = chk & off_chi2
    bad_cov = chk & off_cov
    bad_geo = chk & off_geo
    rep = dict(
        n=int(n), same_path=int(chk.sum()), exempt=int(exempt.sum()),
        bad_path=int(bad_path.sum()), bad_par=int(bad_par.sum()), bad_chi2=int(bad_chi2.sum()),
        bad_cov=int(bad_cov.sum()), bad_geo=int(bad_geo.sum()),
        max_par_rel=float(par_err[:, chk].max(initial=0.0)),
        p99_par_rel=[float(np.percentile(par_err[i, chk], 99)) if chk.any() else 0.0 for i in range(5)],
        max_par_rel_each=[float(par_err[i, chk].max(initial=0.0)) for i in range(5)],
        max_chi2_abs=float(chi2_err[chk].max(initial=0.0)),
        p99_chi2_abs=float(np.percentile(chi2_err[chk], 99)) if chk.any() else 0.0,
        max_cov_rel=float(cov_err[:, chk].max(initial=0.0)),
    )
    msgs = []
    for name, mask in (("path", bad_path), ("par", bad_par), ("chi2", bad_chi2), ("cov", bad_cov),
                       ("geo", bad_geo)):
        if mask.any():
            j = int(np.nonzero(mask)[0][0])
            msgs.append(f"{name}: {int(mask.sum())} tracks, first seed {int(idx[j])}: gpu ids "
                        f"{g['tracklet_id'][:, j].tolist()} st {int(g['status'][j])} chi2 "
                        f"{float(g['chi2'][j]):.6g} par {g['par'][:, j].tolist()} | oracle ids "
                        f"{ora['tracklet_id'][:, j].tolist()} st {int(ora['status'][j])} chi2 "
                        f"{float(ora['chi2'][j]):.6g} par {ora['par'][:, j].tolist()} margin "
                        f"{float(margin_at[j]):.3g}")
    assert not msgs, "\n".join(msgs) + f"\nreport: {rep}"
    assert rep["exempt"] <= max_exempt_frac * n + 2, rep
    return rep


def _cov_norm(cov):
    d = np.sqrt(np.maximum(cov[[0, 2, 5, 9, 14]], 1e-30))
    out = np.empty_like(cov)
    k = 0
    for i in range(5):
        for j in range(i + 1):
            out[k] = d[i] * d[j]
            k += 1
    return out


def compare_refit(gpu: dict, ora: dict, sel=None, max_exempt_frac=0.02) -> dict:
    """The refit's results against the oracle's, with the follower's
    tolerances (parameters 1e-4 of max(|v|, sigma), chi2 1e-3 absolute,
    covariance 1e-3 of sqrt(C_ii C_jj)); status and update count identical
    unless the oracle's smallest decision slack (|snp| limit, sector edge)
    is below 1e-3, in which case the track is exempt."""
    n = ora["chi2"].shape[0]
    idx = np.arange(n) if sel is None else np.asarray(sel)
    g = {k: v[..., idx] for k, v in gpu.items()}
    same = (g["status"] == ora["status"]) & (g["n_upd"] == ora["n_upd"])
    exempt = ~same & (ora["margin"] < MARGIN)
    bad_path = ~same & ~exempt
    sig = np.sqrt(np.maximum(ora["cov"][[0, 2, 5, 9, 14]], 0.0))
    par_err = np.abs(g["par"] - ora["par"]) / np.maximum(np.maximum(np.abs(ora["par"]), sig), 1e-30)
    chi2_err = np.abs(g["chi2"] - ora["chi2"])
    cov_err = np.abs(g["cov"] - ora["cov"]) / _cov_norm(ora["cov"])
    x_err = np.abs(g["x"] - ora["x"])
    a_err = np.abs(np.angle(np.exp(1j * (g["alpha"].astype(np.float64) - ora["alpha"]))))
    bad = {
        "path": bad_path,
        "par": same & (par_err.max(0) > PAR_REL),
        "chi2": same & (chi2_err > CHI2_ABS),
        "cov": same & (cov_err.max(0) > COV_REL),
        "geo": same & ((x_err > 1e-4 * np.abs(ora["x"])) | (a_err > 1e-6)),
    }
    rep = dict(n=int(n), same=int(same.sum()), exempt=int(exempt.sum()),
               refitted=int((same & (ora["status"] == 0)).sum()),
               max_par_rel_each=[float(par_err[i, same].max(initial=0.0)) for i in range(5)],
               max_chi2_abs=float(chi2_err[same].max(initial=0.0)),
               max_cov_rel=float(cov_err[:, same].max(initial=0.0)))
    msgs = []
    for name, mask in bad.items():
        if mask.any():
            j = int(np.nonzero(mask)[0][0])
            msgs.append(f"{name}: {int(mask.sum())} tracks, first {int(idx[j])}: gpu st {int(g['status'][j])} "
                        f"n_upd {int(g['n_upd'][j])} chi2 {float(g['chi2'][j]):.6g} par {g['par'][:, j].tolist()} "
                        f"| oracle st {int(ora['status'][j])} n_upd {int(ora['n_upd'][j])} chi2 "
                        f"{float(ora['chi2'][j]):.6g} par {ora['par'][:, j].tolist()} margin "
                        f"{float(ora['margin'][j]):.3g}")
    assert not msgs, "\n".join(msgs) + f"\nreport: {rep}"
    assert rep["exempt"] <= max_exempt_frac * n + 2, rep
    return rep
