"""Seeded synthetic inputs for the residual collection in TPC sub-volumes
(Sec. 2, steps 4 and 5 of the calibration chain).

Per track: the TPC clusters of its crossings with the 152 pad-row planes,
displaced by a smooth space-charge-like distortion field and smeared; an
ITS-only refit state at x = 40 cm and a TRD-only refit state at x = 300 cm,
each the truth smeared by a known diagonal covariance (an honest Gaussian
input).  The truth helices come from the timeframe generator's global-helix
arithmetic; nothing here transports a state or touches a covariance.

Readings (the paper gives no TPC geometry): 152 pad rows equally spaced
between 85 and 245 cm (centres at 85 + 160 (r + 1/2) / 152 cm); the drift
volume |z| < 250 cm; the 18 sectors of the TRD's segmentation on each side.
Distortion: an electron freed at the track point (x', y', z') reaches pad row
x' + dx with local y' + dy and z' + dz, so the cluster at row x_r belongs to
the track point at x_r - dx.  The field (cm), with g = (1 - |z|/250) (245 -
x) / 160 in [0, 1] (space charge grows towards the inner radius and the
central electrode):
    dx = -1.5 g + 0.3 cos(phi),  dy = (0.5 + 1.5 sin(2 phi)) g,
    dz = 0.5 g sign(z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import timeframe as T

N_ROWS = 152
X_ROW_FIRST, X_ROW_LAST = 85.0, 245.0
Z_DRIFT = 250.0
X_ITS = 40.0
X_TRD = 300.0
ITS_SIGMA = (0.005, 0.005, 5e-4, 5e-4, 0.01)   # y, z, snp, tgl (abs); q/pT (relative)
TRD_SIGMA = (0.03, 1.0, 2e-3, 2e-2, 0.05)


def row_x() -> np.ndarray:
    """Pad-row radii as float32 (the values both sides bin and transport with)."""
    r = np.arange(N_ROWS, dtype=np.float64)
    return (X_ROW_FIRST + (r + 0.5) * (X_ROW_LAST - X_ROW_FIRST) / N_ROWS).astype(np.float32)


def distortion(x, phi, z):
    """The field (dx, dy, dz) in cm at radius x, global azimuth phi, z."""
    g = np.clip(1.0 - np.abs(z) / Z_DRIFT, 0.0, 1.0) * np.clip((X_ROW_LAST - x) / (X_ROW_LAST - X_ROW_FIRST), 0, 1)
    dx = -1.5 * g + 0.3 * np.cos(phi)
    dy = (0.5 + 1.5 * np.sin(2.0 * phi)) * g
    dz = 0.5 * g * np.sign(z)
    return dx, dy, dz


@dataclass
class ResidualWorkload:
    its: dict       # alpha, x [n]; par [5, n]; cov [15, n]; status [n]  (float32 / int32)
    trd: dict       # the same at x = 300 cm
    clusters: dict  # y, z: float32 [152, n]; sector: int8 [152, n] (-1 = no cluster)
    truth: dict     # phi0, kcurv, tgl, q2pt: float64 [n]
    bz: float
    applied: dict = None  # dx, dy, dz: float32 [152, n], the displacement given to each cluster

    @property
    def n_tracks(self) -> int:
        return int(self.its["alpha"].shape[0])

    @property
    def n_clusters(self) -> int:
        return int((self.clusters["sector"] >= 0).sum())


def _smeared_state(rng, truth, x, sigma, bz, smear=True):
    sec, s, y, f, ok = T._cross_chamber_plane(truth["phi0"], truth["kcurv"], x)
    n = y.shape[0]
    z = truth["tgl"] * s
    k = truth["q2pt"]
    sig = np.stack([np.full(n, sigma[0]), np.full(n, sigma[1]), np.full(n, sigma[2]), np.full(n, sigma[3]),
                    sigma[4] * np.abs(k)])
    par = np.stack([y, z, f, truth["tgl"], k]) + rng.normal(size=(5, n)) * sig * (1.0 if smear else 0.0)
    cov = np.zeros((15, n))
    cov[[0, 2, 5, 9, 14]] = sig ** 2
    return dict(alpha=T.sector_alpha(sec).astype(np.float32), x=np.full(n, x, np.float32),
                par=par.astype(np.float32), cov=cov.astype(np.float32),
                status=np.where(ok & (np.abs(par[2]) < 0.9), 0, 1).astype(np.int32))


def make_residual_workload(n_tracks: int, seed: int = 0, distorted: bool = True, smear: float = 0.1,
                           eff: float = 0.9, bz: float = 0.5, fail_frac: float = 0.02,
                           refit_smear: bool = True, phi_range=(0.0, 2.0 * math.pi),
                           eta_range=(-0.9, 0.9), uniform=None) -> ResidualWorkload:
    """n_tracks truth tracks that reach the TRD, their clusters on the 152
    pad rows (distorted by `distortion` when `distorted`, smeared by `smear`
    cm, each present with probability `eff`), and the two refit states
    (smeared by their own sigma unless refit_smear is False; the covariance
    is that sigma squared either way).  A fraction fail_frac of the refits
    is marked failed (status 1).  phi_range and eta_range restrict the truth
    directions (to fill a few voxels densely in tests).  uniform = (dx, dy,
    dz) replaces the smooth field by that constant displacement (sign(z)
    applied to dz)."""
    rng = np.random.Generator(np.random.Philox(key=seed + 5_000_000))
    n_draw = int(n_tracks * 1.6) + 256
    pt = np.clip(rng.exponential(0.6, n_draw), 0.3, 20.0)
    q = rng.choice(np.array([-1.0, 1.0]), n_draw)
    eta = rng.uniform(eta_range[0], eta_range[1], n_draw)
    phi0 = rng.uniform(phi_range[0], phi_range[1], n_draw)
    tgl = np.sinh(eta)
    kc = -T.C_LIGHT * bz * q / pt
    # keep tracks that reach the TRD
    _, _, _, f300, ok300 = T._cross_chamber_plane(phi0, kc, X_TRD)
    keep = np.nonzero(ok300 & (np.abs(f300) < 0.85) & (np.abs(tgl * X_TRD) < 350.0))[0][:n_tracks]
    if keep.shape[0] < n_tracks:
        raise RuntimeError("not enough truth tracks reach the TRD")
    truth = dict(phi0=phi0[keep], kcurv=kc[keep], tgl=tgl[keep], q2pt=(q / pt)[keep])
    its, trd, cl, app = _clusters_and_refits(rng, truth, bz, distorted, smear, eff, refit_smear, uniform)
    # a few refits that failed upstream: their tracks must contribute nothing
    for st in (its, trd):
        st["status"][rng.uniform(0, 1, n_tracks) < fail_frac / 2] = 1
    return ResidualWorkload(its=its, trd=trd, clusters=cl, truth=truth, bz=bz, applied=app)


def clusters_for_truth(truth: dict, bz: float = 0.5, seed: int = 0, distorted: bool = True, smear: float = 0.1,
                       eff: float = 0.9, uniform=None):
    """TPC clusters and an ITS refit state for given truth tracks (e.g. a
    timeframe's, to run the whole calibration chain on them): returns (its,
    clusters, applied displacements).  truth: phi0, kcurv, tgl, q2pt."""
    rng = np.random.Generator(np.random.Philox(key=seed + 6_000_000))
    its, _, cl, app = _clusters_and_refits(rng, truth, bz, distorted, smear, eff, True, uniform)
    return its, cl, app


def _clusters_and_refits(rng, truth, bz, distorted, smear, eff, refit_smear, uniform):
    n = truth["phi0"].shape[0]
    xr = row_x().astype(np.float64)
    cy = np.zeros((N_ROWS, n), np.float32)
    cz = np.zeros((N_ROWS, n), np.float32)
    cs = np.full((N_ROWS, n), -1, np.int8)
    app = np.zeros((3, N_ROWS, n), np.float32)
    for r in range(N_ROWS):
        sec, s, yl, sinl, ok = T._cross_chamber_plane(truth["phi0"], truth["kcurv"], xr[r])
        a = T.sector_alpha(sec)
        if distorted:
            zt = truth["tgl"] * s
            if uniform is None:
                dx, dy, dz = distortion(xr[r], a + np.arctan2(yl, xr[r]), zt)
            else:
                dx, dy, dz = (np.full(n, uniform[0]), np.full(n, uniform[1]), uniform[2] * np.sign(zt))
            s2, ok2 = T._cross_plane(truth["phi0"], truth["kcurv"], a, xr[r] - dx, s0=s)
            _, y2 = T._local_xy(s2, truth["phi0"], truth["kcurv"], a)
            y_cl, z_cl = y2 + dy, truth["tgl"] * s2 + dz
            ok &= ok2
            app[:, r] = dx, dy, dz
        else:
            y_cl, z_cl = yl, truth["tgl"] * s
        y_cl = y_cl + rng.normal(0.0, smear, n)
        z_cl = z_cl + rng.normal(0.0, smear, n)
        ok &= (np.abs(z_cl) < Z_DRIFT) & (np.abs(sinl) < 0.9) & (rng.uniform(0, 1, n) < eff)
        cy[r], cz[r] = y_cl, z_cl
        cs[r] = np.where(ok, sec, -1)
    its = _smeared_state(rng, truth, X_ITS, ITS_SIGMA, bz, refit_smear)
    trd = _smeared_state(rng, truth, X_TRD, TRD_SIGMA, bz, refit_smear)
    return its, trd, dict(y=cy, z=cz, sector=cs), dict(dx=app[0], dy=app[1], dz=app[2])


def _chunk(args):
    n, seed, kw = args
    return make_residual_workload(n, seed=seed, **kw)


def concat_workloads(parts) -> ResidualWorkload:
    """Tracks of several workloads side by side (same field, same bz)."""
    cat = lambda key, d: np.concatenate([getattr(p, d)[key] for p in parts], axis=-1)  # noqa: E731
    its = {k: cat(k, "its") for k in parts[0].its}
    trd = {k: cat(k, "trd") for k in parts[0].trd}
    cl = {k: cat(k, "clusters") for k in parts[0].clusters}
    truth = {k: cat(k, "truth") for k in parts[0].truth}
    app = {k: cat(k, "applied") for k in parts[0].applied}
    return ResidualWorkload(its=its, trd=trd, clusters=cl, truth=truth, bz=parts[0].bz, applied=app)


def make_map_workload(n_tracks: int = 450_000, seed: int = 0, chunk: int = 15_000, workers: int = 0,
                      **kw) -> ResidualWorkload:
    """The tracks of one distortion map (Sec. 2: a map needs at least 450k
    matched tracks), drawn in chunks of `chunk` tracks (chunk k seeded with
    seed * 100003 + k) by a spawn-started process pool."""
    import multiprocessing as mp
    import os
    sizes = [min(chunk, n_tracks - a) for a in range(0, n_tracks, chunk)]
    jobs = [(m, seed * 100003 + k, kw) for k, m in enumerate(sizes)]
    workers = workers or min(len(jobs), os.cpu_count() or 1)
    if workers <= 1 or len(jobs) == 1:
        parts = [_chunk(j) for j in jobs]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_chunk, jobs)
    return concat_workloads(parts)
