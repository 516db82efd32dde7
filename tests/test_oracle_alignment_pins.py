"""Pins of the oracle's misalignment and field-map handling (Sec. 3: tracklets
at different radii are reached by extrapolating to the chamber's average
radius with the field's inhomogeneities, fast linear extrapolations for the
chi2, and a precise propagation to the matched tracklet's radius before the
update), against facts that do not come from the oracle:

* misaligned noiseless tracklets (each measured by the generator where the
  truth helix crosses its own radius) are all found with chi2 ~ 0 when their
  radii are given, and not when they are ignored;
* the track state after the last update is the truth at that tracklet's
  radius (the precise transport happened before the update);
* tracklet and chamber radii equal to the nominal ones reproduce the aligned
  follower; a uniform field map reproduces the homogeneous field, and a
  uniform map of twice the field reproduces bz doubled;
* one transport step with a non-uniform map agrees with a Runge-Kutta
  integration of the equations of motion through the same field.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth import timeframe as G

KAPPA = 2.99792458e-3


def _misaligned(n=400, seed=7, **kw):
    p = G.default_params(material_on=0)
    return p, G.make_timeframe(n, seed=seed, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p,
                               misalign=0.5, x_jitter=0.1, **kw)


def test_misaligned_truth_is_found_with_the_radii_and_not_without():
    p, tf = _misaligned()
    full = (tf.truth_ids >= 0).all(1)
    assert full.sum() > 200
    r = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x)
    np.testing.assert_array_equal(r["tracklet_id"].T[full], tf.truth_ids[full])
    # the fast linear extrapolation to the tracklet's radius is exact to
    # second order in (x_tl - x_chamber) <= 0.6 cm
    assert r["chi2"][full].max() < 0.05
    assert r["chi2"][full].mean() < 1e-3
    nox = {k: v for k, v in tf.tracklets.items() if k != "x"}
    r0 = O.follow(tf.seeds, nox, p)
    assert r0["chi2"][full].mean() > 1.0 or (r0["tracklet_id"].T[full] == tf.truth_ids[full]).mean() < 0.9


def test_state_after_the_last_update_is_the_truth_at_that_radius():
    p, tf = _misaligned(seed=8)
    r = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x)
    ok = np.nonzero((tf.truth_ids >= 0).all(1) & (r["status"] == 0))[0]
    assert ok.size > 200
    last = tf.truth_ids[ok, 5]
    np.testing.assert_array_equal(r["x"][ok], tf.tracklets["x"][last].astype(np.float64))
    y, z, f, t, k, good = G.truth_at_plane({key: v[ok] for key, v in tf.truth.items()}, r["alpha"][ok],
                                           tf.tracklets["x"][last].astype(np.float64))
    assert good.all()
    sig = np.sqrt(r["cov"][[0, 2, 5], :][:, ok])
    # exact tracklets and a precise transport: the filter sits on the truth
    assert np.all(np.abs(r["par"][0][ok] - y) < 0.02 * sig[0])
    assert np.all(np.abs(r["par"][1][ok] - z) < 0.02 * sig[1])
    assert np.all(np.abs(r["par"][2][ok] - f) < 0.05 * sig[2])


def test_a_layer_without_tracklet_ends_at_the_chamber_radius():
    """Remove the last layer's tracklet of every other full track: those
    tracks end at the average radius of the chamber they cross there, on the
    truth helix (the transport to the chamber radius happened)."""
    p, tf = _misaligned(seed=9)
    full = np.nonzero((tf.truth_ids >= 0).all(1))[0]
    drop = full[::2]
    trk = {k: v.copy() for k, v in tf.tracklets.items()}
    gone = tf.truth_ids[drop, 5]
    ch5 = trk["chamber"][gone].copy()
    trk["chamber"][gone] = -1  # not a chamber: never a candidate
    r = O.follow(tf.seeds, trk, p, chamber_x=tf.chamber_x)
    ok = r["n_trk"][drop] == 5
    assert ok.mean() > 0.95
    sel, ch = drop[ok], ch5[ok]
    np.testing.assert_array_equal(r["x"][sel], tf.chamber_x[ch].astype(np.float64))
    y, z, f, t, k, good = G.truth_at_plane({key: v[sel] for key, v in tf.truth.items()}, r["alpha"][sel],
                                           tf.chamber_x[ch].astype(np.float64))
    assert good.all()
    sig = np.sqrt(r["cov"][[0, 2], :][:, sel])
    assert np.all(np.abs(r["par"][0][sel] - y) < 0.05 * sig[0])
    assert np.all(np.abs(r["par"][1][sel] - z) < 0.05 * sig[1])


def test_nominal_radii_reproduce_the_aligned_follower():
    tf = G.make_workload("tiny", seed=3)
    nominal = np.array([300.0 + 12.6 * l for l in range(6)], np.float32)
    trk = dict(tf.tracklets, x=nominal[tf.tracklets["chamber"] % 6])
    cx = np.tile(nominal, 90)
    a = O.follow(tf.seeds, tf.tracklets, tf.params)
    b = O.follow(tf.seeds, trk, tf.params, chamber_x=cx)
    np.testing.assert_array_equal(a["tracklet_id"], b["tracklet_id"])
    np.testing.assert_array_equal(a["status"], b["status"])
    # the float radii differ from the layer radii by up to 6e-6 cm (312.6 is
    # not a float), which each update carries on: ~1e-4 cm after six layers
    np.testing.assert_allclose(b["par"], a["par"], rtol=2e-5, atol=3e-4)


def _uniform_map(b):
    return dict(bz=np.full((5, 4), b, np.float32), r_min=250.0, r_max=420.0, z_min=-400.0, z_max=400.0)


def test_uniform_field_map_is_the_homogeneous_field():
    tf = G.make_workload("tiny", seed=4)
    a = O.follow(tf.seeds, tf.tracklets, tf.params)
    b = O.follow(tf.seeds, tf.tracklets, tf.params, field=_uniform_map(tf.params["bz"]))
    np.testing.assert_array_equal(a["tracklet_id"], b["tracklet_id"])
    np.testing.assert_allclose(b["par"], a["par"], rtol=1e-12, atol=1e-12)
    # the map is what bends the tracks: a map of 2 bz with the nominal bz is bz doubled
    p2 = dict(tf.params, bz=2 * tf.params["bz"])
    c = O.follow(tf.seeds, tf.tracklets, p2)
    d = O.follow(tf.seeds, tf.tracklets, tf.params, field=_uniform_map(2 * tf.params["bz"]))
    np.testing.assert_array_equal(c["tracklet_id"], d["tracklet_id"])
    np.testing.assert_allclose(d["par"], c["par"], rtol=1e-12, atol=1e-12)
    assert not np.array_equal(a["tracklet_id"], c["tracklet_id"])


def _rk4_to_plane(st, x1, field_fn):
    """Integrate dX/ds = cos(phi), dY/ds = sin(phi), dphi/ds = -kappa Bz k,
    dZ/ds = tgl in the state's local frame (the frame is a rotation of the
    global one, and Bz depends only on r and z) until x = x1."""
    _, x, y, z, f, t, k = st
    phi = math.asin(f)
    h = 0.01

    def deriv(v):
        X, Y, Z, P = v
        bz = field_fn(math.hypot(X, Y), Z)
        return np.array([math.cos(P), math.sin(P), t, -KAPPA * bz * k])

    v = np.array([x, y, z, phi])
    while True:
        k1 = deriv(v)
        k2 = deriv(v + 0.5 * h * k1)
        k3 = deriv(v + 0.5 * h * k2)
        k4 = deriv(v + h * k3)
        nv = v + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if nv[0] >= x1:
            # finish on the plane with a straight partial step
            frac = (x1 - v[0]) / (nv[0] - v[0])
            return v + frac * (nv - v)
        v = nv


def test_field_map_step_agrees_with_runge_kutta():
    # a map that falls off along z and grows with r, 0.5 T in the middle
    rs, zs = np.linspace(250.0, 420.0, 18), np.linspace(-400.0, 400.0, 41)
    R, Z = np.meshgrid(rs, zs)
    bz = (0.5 * (1.0 - 0.15 * (Z / 400.0) ** 2) * (1.0 + 0.05 * (R - 300.0) / 100.0)).astype(np.float32)
    fmap = dict(bz=bz, r_min=250.0, r_max=420.0, z_min=-400.0, z_max=400.0)

    def field_fn(r, z):  # bilinear over the same table: the map's definition
        fr = np.clip((len(rs) - 1) * (r - 250.0) / 170.0, 0, len(rs) - 1)
        fz = np.clip((len(zs) - 1) * (z + 400.0) / 800.0, 0, len(zs) - 1)
        i, j = min(int(fr), len(rs) - 2), min(int(fz), len(zs) - 2)
        wr, wz = fr - i, fz - j
        b = bz.astype(np.float64)
        return (1 - wz) * ((1 - wr) * b[j, i] + wr * b[j, i + 1]) + wz * ((1 - wr) * b[j + 1, i] + wr * b[j + 1, i + 1])

    rng = np.random.default_rng(2)
    c = np.diag([1e-2, 1e-2, 1e-6, 1e-6, 1e-4])[np.tril_indices(5)]
    worse = 0
    for _ in range(40):
        st = np.array([0.35, 300.0, rng.uniform(-30, 30), rng.uniform(-250, 250), rng.uniform(-0.5, 0.5),
                       rng.uniform(-0.9, 0.9), rng.choice([-1, 1]) * rng.uniform(0.3, 3.0)])
        ok, out, _ = O.propagate_map(st, c, 312.6, 0.5, fmap)
        assert ok
        X, Y, Zf, P = _rk4_to_plane(st, 312.6, field_fn)
        # one constant field per step, taken at its midpoint: the turning angle
        # is right to second order; the position, a double integral, is off by
        # g L^3 / 12 for a curvature changing at the rate g along the step
        # (here <= ~4e-4 cm over L = 12.6 cm)
        assert out[2] == pytest.approx(Y, abs=1e-3)
        assert out[3] == pytest.approx(Zf, abs=1e-3)
        assert out[4] == pytest.approx(math.sin(P), abs=2e-5)
        # the map matters: the nominal 0.5 T alone misses by more
        ok2, out2, _ = O.propagate_map(st, c, 312.6, 0.5, None)
        assert ok2
        worse += abs(out2[2] - Y) > 3 * abs(out[2] - Y) + 1e-4
    assert worse > 10


def test_refit_at_the_tracklet_radii_recovers_the_truth():
    """The TRD-only refit of misaligned noiseless tracks ends at layer 0's
    tracklet radius, on the truth helix there."""
    p, tf = _misaligned(seed=10)
    r = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x)
    rf = O.refit(r, tf.tracklets, p)
    ok = np.nonzero((tf.truth_ids >= 0).all(1) & (rf["status"] == 0))[0]
    assert ok.size > 200
    x0 = tf.tracklets["x"][tf.truth_ids[ok, 0]].astype(np.float64)
    np.testing.assert_array_equal(rf["x"][ok], x0)
    y, z, f, t, k, good = G.truth_at_plane({key: v[ok] for key, v in tf.truth.items()}, rf["alpha"][ok], x0)
    assert good.all()
    sig = np.sqrt(rf["cov"][[0, 2, 5], :][:, ok])
    assert np.all(np.abs(rf["par"][0][ok] - y) < 2e-3 * sig[0] + 1e-5)
    assert np.all(np.abs(rf["par"][1][ok] - z) < 2e-3 * sig[1] + 1e-5)
    assert np.all(np.abs(rf["par"][2][ok] - f) < 2e-3 * sig[2] + 1e-7)
    # ignoring the radii, the refit is pulled off the truth
    nox = {k_: v for k_, v in tf.tracklets.items() if k_ != "x"}
    rf0 = O.refit(r, nox, p)
    y0, *_ = G.truth_at_plane({key: v[ok] for key, v in tf.truth.items()}, rf0["alpha"][ok], np.full(ok.size, 300.0))
    assert np.median(np.abs(rf0["par"][0][ok] - y0) / sig[0]) > 0.1
