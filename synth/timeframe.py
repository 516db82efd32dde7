"""Seeded synthetic timeframes: truth helices, TRD tracklets and smeared seeds.

The paper's Pb-Pb simulation and data are not available, so these inputs
stand in for them.  The detector follows Sec. 3 of the paper: 18 sectors in
azimuth, 5 stacks along the beam, 6 layers in radius (all 540 chambers are
active), a 3 cm drift region, pads tilted by +-2 degrees, and a Lorentz angle
of about 8 degrees at 0.5 T.  A tracklet carries a local y, a z snapped to its
pad-row centre, a deflection dy over the drift length, and a 2x2 covariance.

The truth track is a helix from the origin written in global coordinates
(position as a function of transverse arc length); its crossing with a
chamber plane is found by Newton iteration on that parametrisation.  This is
simulation arithmetic of its own and shares nothing with the follower.

Random numbers come from numpy's counter-based Philox generator keyed by the
workload seed, so every input is reproducible.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --- detector description (Sec. 3; radii and pad rows are readings) --------
N_SECTORS = 18
N_STACKS = 5
N_LAYERS = 6
N_CHAMBERS = N_SECTORS * N_STACKS * N_LAYERS  # 540
ROWS_PER_STACK = 18
ROW_LENGTH = 8.0  # cm
STACK_LENGTH = ROWS_PER_STACK * ROW_LENGTH  # 144 cm
Z_MIN = -0.5 * N_STACKS * STACK_LENGTH  # -360 cm
X_SEED = 290.0  # cm, plane of the extrapolated ITS-TPC seeds
SECTOR_WIDTH_DEG = 360.0 / N_SECTORS
DRIFT_LENGTH = 3.0  # cm
PAD_TILT_DEG = 2.0
LORENTZ_DEG = 8.0
C_LIGHT = 2.99792458e-3  # 1/R[cm] = C_LIGHT * |B[T]| / pT[GeV/c]


def layer_x(layer: int) -> float:
    """Radius of the chamber plane of a layer (cm)."""
    return 300.0 + 12.6 * layer


def sector_alpha(sector):
    """Azimuth of the centre of a sector (rad)."""
    return np.deg2rad(SECTOR_WIDTH_DEG * (np.asarray(sector) + 0.5))


def sector_of_phi(phi):
    w = 2.0 * math.pi / N_SECTORS
    return np.floor(np.mod(phi, 2.0 * math.pi) / w).astype(np.int64) % N_SECTORS


# --- truth helix in global coordinates --------------------------------------
# Position after transverse arc length s, for a track leaving the origin with
# azimuth phi0 and signed curvature k (d(phi)/ds):
#   X(s) = s * sinc(k s / 2) * cos(phi0 + k s / 2)
#   Y(s) = s * sinc(k s / 2) * sin(phi0 + k s / 2)
#   Z(s) = tan(lambda) * s
# The local coordinates in a frame of azimuth a are X cos a + Y sin a and
# -X sin a + Y cos a; the local direction is phi0 + k s - a.

def _local_xy(s, phi0, k, a):
    half = 0.5 * k * s
    ch = s * np.sinc(half / math.pi)
    return ch * np.cos(phi0 + half - a), ch * np.sin(phi0 + half - a)


def _cross_plane(phi0, k, a, xp, s0=None):
    """Smallest arc length at which the helix crosses local x = xp, by Newton
    (started from s0 when given, e.g. the crossing of a nearby plane).

    Returns (s, ok).  ok is False where the helix turns back before reaching
    the plane or the iteration did not converge.
    """
    d0 = np.cos(phi0 - a)
    s = xp / np.maximum(d0, 0.3) if s0 is None else np.asarray(s0, dtype=np.float64).copy()
    smax = np.where(np.abs(k) > 0, math.pi / np.maximum(np.abs(k), 1e-12), 1e9)
    for _ in range(40):
        xl, _ = _local_xy(s, phi0, k, a)
        if np.all(np.abs(xl - xp) < 1e-9 * xp):
            break
        der = np.cos(phi0 + k * s - a)
        der = np.where(np.abs(der) < 0.05, np.copysign(0.05, der), der)
        s = np.clip(s - (xl - xp) / der, 0.0, smax)
    xl, _ = _local_xy(s, phi0, k, a)
    outgoing = np.cos(phi0 + k * s - a) > 0.05
    ok = (np.abs(xl - xp) < 1e-7 * np.maximum(xp, 1.0)) & outgoing & (s > 0)
    return s, ok


def _cross_chamber_plane(phi0, k, xp):
    """Crossing of the layer polygon at radius xp: find the sector whose plane
    is crossed inside the sector's azimuthal extent.

    Returns (sector, s, y_local, sin_local, ok).
    """
    guess = sector_of_phi(phi0 + 0.5 * k * xp)
    sec = guess.copy()
    ylim = xp * math.tan(math.radians(0.5 * SECTOR_WIDTH_DEG))
    a = sector_alpha(sec)
    s, ok = _cross_plane(phi0, k, a, xp)
    _, yl = _local_xy(s, phi0, k, a)
    for _ in range(3):
        move = np.where(ok & (yl > ylim), 1, np.where(ok & (yl < -ylim), -1, 0))
        sel = np.nonzero(move)[0]
        if sel.size == 0:
            break
        sec[sel] = (sec[sel] + move[sel]) % N_SECTORS
        a = sector_alpha(sec)
        s2, ok2 = _cross_plane(phi0[sel], k[sel], a[sel], xp)
        _, y2 = _local_xy(s2, phi0[sel], k[sel], a[sel])
        s[sel], ok[sel], yl[sel] = s2, ok2, y2
    ok &= np.abs(yl) <= ylim
    sinl = np.sin(phi0 + k * s - a)
    return sec, s, yl, sinl, ok


def truth_at_plane(truth: dict, alpha, xp):
    """The truth track's local state where it crosses the plane x = xp of the
    frame of azimuth alpha: (y, z, sin(phi), tan(lambda), q/pT, ok), arrays
    over the truth entries (alpha may be an array)."""
    phi0, k, tgl = truth["phi0"], truth["kcurv"], truth["tgl"]
    a = np.broadcast_to(np.asarray(alpha, dtype=np.float64), phi0.shape)
    s, ok = _cross_plane(phi0, k, a, xp)
    _, y = _local_xy(s, phi0, k, a)
    return y, tgl * s, np.sin(phi0 + k * s - a), tgl, truth["q2pt"], ok


def pad_tilt_tan(layer: int) -> float:
    """tan of the pad tilt: +2 degrees on even layers, -2 on odd (a reading)."""
    return math.tan(math.radians(PAD_TILT_DEG if layer % 2 == 0 else -PAD_TILT_DEG))


def _deflection_model(phi_local, bz):
    """Detector response for dy: the drift-length deflection of a track with
    local direction phi_local, and its spread.  The spread is best for tracks
    entering at the Lorentz angle (Sec. 3, Fig. 3)."""
    tpsi = math.tan(math.radians(LORENTZ_DEG)) * (1.0 if bz >= 0 else -1.0)
    u = np.tan(phi_local) - tpsi
    return DRIFT_LENGTH * u, np.sqrt(0.04 ** 2 + (0.1 * u) ** 2)


# --- workloads ---------------------------------------------------------------
WORKLOADS = {
    # name: (n_seeds, noise fraction, n_hyp, road sigma, chi2 cut, max missing,
    #        distortion + relaxed seed tolerance)
    "tiny": dict(n_seeds=1_000, noise=0.20, n_hyp=1, road=3.0, chi2_cut=15.0,
                 max_missing=2, distortion=False),
    "timeframe": dict(n_seeds=200_000, noise=0.30, n_hyp=1, road=3.0, chi2_cut=15.0,
                      max_missing=2, distortion=False),
    "calibration": dict(n_seeds=450_000, noise=0.30, n_hyp=6, road=5.0, chi2_cut=15.0,
                        max_missing=2, distortion=True),
}


@dataclass
class Timeframe:
    """One timeframe of inputs plus the truth kept for diagnostics."""
    name: str
    seeds: dict  # alpha, x, y, z, snp, tgl, q2pt: float32[n]; cov: float32[15, n]
    tracklets: dict  # chamber: int32[m]; y, z, dy, vyy, vzz, vyz: float32[m]
    params: dict  # follower parameters of the workload
    truth_ids: np.ndarray  # int32[n, 6]: input index of the seed's true tracklet, -1 if none
    truth_pt: np.ndarray = field(default=None)
    # truth helix per seed: azimuth at the origin phi0, signed curvature kcurv
    # (d(phi)/ds, 1/cm), tan(lambda), q/pT: float64[n] each
    truth: dict = field(default=None)
    chamber_x: np.ndarray = None  # float32[540] average chamber radii when misaligned

    @property
    def n_seeds(self) -> int:
        return int(self.seeds["alpha"].shape[0])

    @property
    def n_tracklets(self) -> int:
        return int(self.tracklets["chamber"].shape[0])


def default_params(bz=0.5, **over):
    p = dict(bz=bz, n_sigma_road=3.0, chi2_cut=15.0, p_miss=None, dy_gate_sigma=4.0,
             n_hyp=1, max_missing=2, res_mode=0, material_on=1)
    p.update(over)
    if p["p_miss"] is None:
        p["p_miss"] = p["chi2_cut"]
    return p


def make_timeframe(n_seeds: int, seed: int = 0, noise: float = 0.2, bz: float = 0.5,
                   eff: float = 0.9, smear: bool = True, snap_z: bool = True,
                   distortion: bool = False, sys_y: float = 0.0,
                   off_centre_frac: float = 0.1, name: str = "custom",
                   params: dict | None = None, n_interactions: int = 0,
                   misalign: float = 0.0, x_jitter: float = 0.0) -> Timeframe:
    """Draw one timeframe.

    Truth: |eta| < 0.9, uniform phi, q = +-1, pT exponential with mean 0.6
    GeV/c clipped to [0.3, 20].  Every chamber crossing gives a tracklet with
    probability `eff`; noise tracklets (count = noise x signal) are uniform in
    chamber, pad row and y, with dy uniform in +-1.5 cm.  Seeds are the truth
    at x = 290 cm smeared by the diagonal covariance (0.1 cm, 0.1 cm, 1e-3,
    1e-3, 1 % of q/pT).  With `distortion`, seeds get a coherent y offset of
    1-5 cm (smooth in radius and azimuth) and `sys_y` is added in quadrature
    to their y error.  With n_interactions > 0, every track belongs to one of
    that many interactions (uniform), its seed and tracklets carry the id
    ("trigger"), and noise tracklets get a uniform random id (drawn from a
    separate stream, so the rest of the timeframe is unchanged).  With
    misalign > 0 or x_jitter > 0 (cm), every chamber gets an average radius
    x_l + U(-misalign, misalign) and every tracklet a radius x_chamber +
    U(-x_jitter, x_jitter) (a third stream); the tracklet then measures the
    truth where it crosses the plane of its own radius (the chamber is still
    the one crossed at the nominal radius), and the timeframe carries
    tracklets["x"] and chamber_x.
    """
    rng = np.random.Generator(np.random.Philox(key=seed))
    n_draw = int(n_seeds * 1.5) + 256
    pt = np.clip(rng.exponential(0.6, n_draw), 0.3, 20.0)
    q = rng.choice(np.array([-1.0, 1.0]), n_draw)
    eta = rng.uniform(-0.9, 0.9, n_draw)
    phi0 = rng.uniform(0.0, 2.0 * math.pi, n_draw)
    tgl = np.sinh(eta)
    # Lorentz force on +q in +Bz bends the track clockwise (towards -y).
    kcurv = -C_LIGHT * bz * q / pt

    # seed plane: the sector frame of the crossing, sometimes rotated off-centre
    sec_s, _, _, _, ok_s = _cross_chamber_plane(phi0, kcurv, X_SEED)
    a_seed = sector_alpha(sec_s)
    off = rng.uniform(0, 1, n_draw) < off_centre_frac
    a_seed = a_seed + np.where(off, np.deg2rad(rng.uniform(-8.0, 8.0, n_draw)), 0.0)
    s_s, ok2 = _cross_plane(phi0, kcurv, a_seed, X_SEED)
    _, y_s = _local_xy(s_s, phi0, kcurv, a_seed)
    f_s = np.sin(phi0 + kcurv * s_s - a_seed)
    ok_seed = ok_s & ok2 & (np.abs(f_s) < 0.9)
    idx = np.nonzero(ok_seed)[0][:n_seeds]
    if idx.shape[0] < n_seeds:
        raise RuntimeError("not enough valid truth tracks drawn")
    pt, q, eta, phi0, tgl, kcurv = pt[idx], q[idx], eta[idx], phi0[idx], tgl[idx], kcurv[idx]
    a_seed, s_s, y_s, f_s = a_seed[idx], s_s[idx], y_s[idx], f_s[idx]
    n = n_seeds

    # tracklets from truth crossings
    aligned = misalign <= 0.0 and x_jitter <= 0.0
    chamber_x = None
    if not aligned:
        arng = np.random.Generator(np.random.Philox(key=seed + 9_999_999))
        nominal = np.repeat(np.array([layer_x(l) for l in range(N_LAYERS)])[None, :], N_SECTORS * N_STACKS, 0)
        chamber_x = (nominal.reshape(-1) + arng.uniform(-misalign, misalign, N_CHAMBERS)).astype(np.float32)
    ch_l, y_l, z_l, dy_l, owner_l, layer_l, x_l = [], [], [], [], [], [], []
    for layer in range(N_LAYERS):
        xp = layer_x(layer)
        sec, s, yl, sinl, ok = _cross_chamber_plane(phi0, kcurv, xp)
        z = tgl * s
        ok &= (z >= Z_MIN) & (z < -Z_MIN) & (np.abs(sinl) < 0.95)
        ok &= rng.uniform(0, 1, n) < eff
        stack = np.clip(np.floor((z - Z_MIN) / STACK_LENGTH), 0, N_STACKS - 1).astype(np.int64)
        if not aligned:
            # the tracklet sits at its own radius: the truth there, in the same chamber
            ch_n = sec * (N_STACKS * N_LAYERS) + stack * N_LAYERS + layer
            xt = chamber_x[ch_n].astype(np.float64) + arng.uniform(-x_jitter, x_jitter, n)
            xt = xt.astype(np.float32).astype(np.float64)
            a_s = sector_alpha(sec)
            s2, ok2 = _cross_plane(phi0, kcurv, a_s, xt, s0=s)
            _, yl = _local_xy(s2, phi0, kcurv, a_s)
            sinl = np.sin(phi0 + kcurv * s2 - a_s)
            z = tgl * s2
            # a crossing that left the chamber's stack between the two radii
            # gives no tracklet in that chamber
            ok &= ok2 & (np.abs(sinl) < 0.95) & (z >= Z_MIN + STACK_LENGTH * stack) & \
                (z < Z_MIN + STACK_LENGTH * (stack + 1))
            x_l.append(xt)
        row = np.clip(np.floor((z - Z_MIN - STACK_LENGTH * stack) / ROW_LENGTH), 0,
                      ROWS_PER_STACK - 1)
        z_row = Z_MIN + STACK_LENGTH * stack + ROW_LENGTH * (row + 0.5)
        z_meas = z_row if snap_z else z
        tt = pad_tilt_tan(layer)
        y_meas = yl - tt * (z - z_meas)
        phil = np.arcsin(np.clip(sinl, -0.999, 0.999))
        dyv, sdy = _deflection_model(phil, bz)
        if smear:
            y_meas = y_meas + rng.normal(0.0, 0.04, n)
            dyv = dyv + rng.normal(0.0, 1.0, n) * sdy
        sel = np.nonzero(ok)[0]
        if not aligned:
            x_l[-1] = x_l[-1][sel]
        ch_l.append(sec[sel] * (N_STACKS * N_LAYERS) + stack[sel] * N_LAYERS + layer)
        y_l.append(y_meas[sel])
        z_l.append(z_meas[sel])
        dy_l.append(dyv[sel])
        owner_l.append(sel)
        layer_l.append(np.full(sel.shape[0], layer))
    ch = np.concatenate(ch_l)
    ty = np.concatenate(y_l)
    tz = np.concatenate(z_l)
    tdy = np.concatenate(dy_l)
    owner = np.concatenate(owner_l)
    tlayer = np.concatenate(layer_l)
    n_sig = ch.shape[0]

    n_noise = int(round(noise * n_sig))
    tx = np.concatenate(x_l) if not aligned else None
    if n_noise:
        nch = rng.integers(0, N_CHAMBERS, n_noise)
        if not aligned:
            tx = np.concatenate([tx, chamber_x[nch] + arng.uniform(-x_jitter, x_jitter, n_noise)])
        nlayer = nch % N_LAYERS
        nstack = (nch // N_LAYERS) % N_STACKS
        nrow = rng.integers(0, ROWS_PER_STACK, n_noise)
        xl = 300.0 + 12.6 * nlayer
        ylim = xl * math.tan(math.radians(0.5 * SECTOR_WIDTH_DEG))
        ch = np.concatenate([ch, nch])
        ty = np.concatenate([ty, rng.uniform(-1.0, 1.0, n_noise) * ylim])
        tz = np.concatenate([tz, Z_MIN + STACK_LENGTH * nstack + ROW_LENGTH * (nrow + 0.5)])
        tdy = np.concatenate([tdy, rng.uniform(-1.5, 1.5, n_noise)])
        owner = np.concatenate([owner, np.full(n_noise, -1)])
        tlayer = np.concatenate([tlayer, nlayer])
    m = ch.shape[0]
    trig_trk = trig_seed = None
    if n_interactions > 0:
        irng = np.random.Generator(np.random.Philox(key=seed + 7_777_777))
        inter = irng.integers(0, n_interactions, n)
        trig_seed = inter.astype(np.int32)
        trig_trk = np.where(owner >= 0, inter[np.maximum(owner, 0)],
                            irng.integers(0, n_interactions, m)).astype(np.int32)
    perm = rng.permutation(m)
    inv = np.empty(m, dtype=np.int64)
    inv[perm] = np.arange(m)
    truth = np.full((n, N_LAYERS), -1, dtype=np.int32)
    sig_pos = inv[:n_sig]
    truth[owner[:n_sig], tlayer[:n_sig]] = sig_pos
    tracklets = dict(
        chamber=ch[perm].astype(np.int32),
        y=ty[perm].astype(np.float32),
        z=tz[perm].astype(np.float32),
        dy=tdy[perm].astype(np.float32),
        vyy=np.full(m, 0.04 ** 2, np.float32),
        vzz=np.full(m, ROW_LENGTH ** 2 / 12.0, np.float32),
        vyz=np.zeros(m, np.float32),
    )
    if trig_trk is not None:
        tracklets["trigger"] = trig_trk[perm]
    if not aligned:
        tracklets["x"] = tx[perm].astype(np.float32)

    # seeds
    z_s = tgl * s_s
    q2pt = q / pt
    sig = np.array([0.1, 0.1, 1e-3, 1e-3])
    y0, z0, f0, t0, k0 = y_s.copy(), z_s.copy(), f_s.copy(), tgl.copy(), q2pt.copy()
    if smear:
        y0 += rng.normal(0, sig[0], n)
        z0 += rng.normal(0, sig[1], n)
        f0 += rng.normal(0, sig[2], n)
        t0 += rng.normal(0, sig[3], n)
        k0 *= 1.0 + rng.normal(0, 0.01, n)
    cyy = np.full(n, sig[0] ** 2)
    if distortion:
        # coherent space-charge-like offset, 1-5 cm, smooth in azimuth and radius
        phig = a_seed + np.arctan2(y_s, X_SEED)
        y0 += 3.0 + 2.0 * np.sin(2.0 * phig) * math.cos(math.pi * (X_SEED - 250.0) / 200.0)
        cyy += sys_y ** 2
    cov = np.zeros((15, n))
    cov[0] = cyy
    cov[2] = sig[1] ** 2
    cov[5] = sig[2] ** 2
    cov[9] = sig[3] ** 2
    cov[14] = (0.01 * q2pt) ** 2
    seeds = dict(
        alpha=np.mod(a_seed, 2.0 * math.pi).astype(np.float32),
        x=np.full(n, X_SEED, np.float32),
        y=y0.astype(np.float32), z=z0.astype(np.float32), snp=f0.astype(np.float32),
        tgl=t0.astype(np.float32), q2pt=k0.astype(np.float32),
        cov=np.ascontiguousarray(cov.astype(np.float32)),
    )
    if trig_seed is not None:
        seeds["trigger"] = trig_seed
    return Timeframe(name=name, seeds=seeds, tracklets=tracklets,
                     params=params if params is not None else default_params(bz),
                     truth_ids=truth, truth_pt=pt.astype(np.float32),
                     truth=dict(phi0=phi0, kcurv=kcurv, tgl=tgl, q2pt=q / pt), chamber_x=chamber_x)


def make_workload(name: str, seed: int = 0, n_seeds: int | None = None,
                  n_interactions: int = 0, misalign: float = 0.0, x_jitter: float = 0.0) -> Timeframe:
    """One of the named workloads (tiny, timeframe, calibration), optionally
    with a different seed count (same distributions), with interaction ids
    (n_interactions > 0: per-interaction association, Sec. 4) and with
    misaligned chambers (misalign, x_jitter in cm: per-tracklet radii)."""
    w = WORKLOADS[name]
    params = default_params(0.5, n_sigma_road=w["road"], chi2_cut=w["chi2_cut"],
                            n_hyp=w["n_hyp"], max_missing=w["max_missing"])
    return make_timeframe(n_seeds or w["n_seeds"], seed=seed, noise=w["noise"],
                          distortion=w["distortion"], sys_y=2.0 if w["distortion"] else 0.0,
                          name=name, params=params, n_interactions=n_interactions,
                          misalign=misalign, x_jitter=x_jitter)


def field_map(b0: float = 0.5) -> dict:
    """A Bz(r, z) map for the misalignment/field-map workloads: b0 in the
    middle, falling 15 % towards |z| = 400 cm, rising 5 % per metre in r, on
    an 18 x 41 grid over r in [250, 420] cm and z in [-400, 400] cm."""
    rs, zs = np.linspace(250.0, 420.0, 18), np.linspace(-400.0, 400.0, 41)
    R, Z = np.meshgrid(rs, zs)
    bz = (b0 * (1.0 - 0.15 * (Z / 400.0) ** 2) * (1.0 + 0.05 * (R - 300.0) / 100.0)).astype(np.float32)
    return dict(bz=bz, r_min=250.0, r_max=420.0, z_min=-400.0, z_max=400.0)


def batched_seed_counts(n_tf=64, lo=5_000, hi=400_000, seed=0):
    """Seed counts log-uniform in [lo, hi] for a batch of timeframes."""
    rng = np.random.Generator(np.random.Philox(key=10_000 + seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n_tf)).astype(np.int64)


def served_seed_counts(n_req, median=100_000, sigma=0.8, cap=600_000, seed=0):
    """Seed counts log-normal (median, sigma), capped, for a served stream."""
    rng = np.random.Generator(np.random.Philox(key=20_000 + seed))
    return np.minimum(np.exp(rng.normal(math.log(median), sigma, n_req)), cap).astype(np.int64)


def efficiency_purity(tracklet_id: np.ndarray, truth_ids: np.ndarray) -> dict:
    """Sec. 3.1 definitions on synthetic truth.

    tracklet_id: int[6, n] attached input ids (-1 = none).  A track is
    efficient when at least 2 correct tracklets are attached; purity is the
    fraction of tracks with at least 2 tracklets that carry no fake one.
    """
    ids = np.asarray(tracklet_id).T  # [n, 6]
    attached = ids >= 0
    correct = attached & (ids == truth_ids)
    n_att = attached.sum(1)
    n_cor = correct.sum(1)
    reach = (truth_ids >= 0).sum(1) >= 2
    eff_all = float((n_cor >= 2).mean()) if ids.shape[0] else 0.0
    eff_reach = float((n_cor[reach] >= 2).mean()) if reach.any() else 0.0
    two = n_att >= 2
    purity = float((n_cor[two] == n_att[two]).mean()) if two.any() else 0.0
    return dict(efficiency=eff_all, efficiency_reachable=eff_reach, purity=purity,
                matched=int(two.sum()))


BATCH_PARAMS = dict(n_hyp=3, road=3.0, chi2_cut=15.0, max_missing=2, noise=0.30)


def _batch_member(args):
    n, seed = args
    p = default_params(0.5, n_sigma_road=BATCH_PARAMS["road"], chi2_cut=BATCH_PARAMS["chi2_cut"],
                       n_hyp=BATCH_PARAMS["n_hyp"], max_missing=BATCH_PARAMS["max_missing"])
    return make_timeframe(int(n), seed=seed, noise=BATCH_PARAMS["noise"], name=f"tf{seed}", params=p)


def make_batch(counts, seed: int = 0, workers: int = 0):
    """Timeframes with the given seed counts (timeframe t drawn with seed
    1000 * seed + t), N = 3, 3-sigma road, 30 % noise.  workers > 1 draws
    them in a process pool started with 'spawn'."""
    jobs = [(int(n), 1000 * seed + t) for t, n in enumerate(counts)]
    if workers and workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_batch_member, jobs, chunksize=1)
    return [_batch_member(j) for j in jobs]


def concat(tfs):
    """Concatenate timeframes: (seeds, tracklets, seed_offsets, tracklet_offsets)."""
    so = np.zeros(len(tfs) + 1, np.int32)
    to = np.zeros(len(tfs) + 1, np.int32)
    so[1:] = np.cumsum([t.n_seeds for t in tfs])
    to[1:] = np.cumsum([t.n_tracklets for t in tfs])
    seeds = {k: (np.concatenate([t.seeds[k] for t in tfs], axis=-1) if k == "cov" else
                 np.concatenate([t.seeds[k] for t in tfs])) for k in tfs[0].seeds}
    seeds["cov"] = np.ascontiguousarray(seeds["cov"])
    trk = {k: np.concatenate([t.tracklets[k] for t in tfs]) for k in tfs[0].tracklets}
    return seeds, trk, so, to
