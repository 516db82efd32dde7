"""Pins of the oracle's TRD-only refit (Sec. 2, step 3) against facts that do
not come from the oracle.

* With noiseless tracklets the refit lands on the generator's truth helix.
* Without material the model is a pure helix, so the refit (an extended
  Kalman filter run inward over the tracklets, started from a diagonal prior)
  must agree with the maximum a posteriori fit of the same prior and
  tracklets, solved here by nonlinear least squares over a forward model of
  its own (global circle geometry); the filter's summed update chi2 equals
  that fit's minimum, and its covariance the inverse of the fit's normal
  matrix.
* On smeared timeframes the refit's pulls against the truth are unit normal.
* Inward material gives back the outward step's energy loss.
"""
import math

import numpy as np
import pytest
from scipy.optimize import least_squares

from oracle import oracle as O
from synth import timeframe as G

KAPPA = 2.99792458e-3
SECTOR = 2.0 * math.pi / 18


def _layer_x(l):
    return 300.0 + 12.6 * l


def _tilt(l):
    return math.tan(math.radians(2.0 if l % 2 == 0 else -2.0))


def _state_at(p, alpha0, x0, alpha1, x1, bz):
    """Local state (y, z, snp, tgl, q2pt) at plane x = x1 of the frame alpha1
    of the helix whose local state at plane x0 of frame alpha0 is p.
    Global geometry: the direction angle turns at the rate rho per transverse
    arc, so sin(direction - alpha1) changes by rho times the distance
    covered along the frame's x axis."""
    y0, z0, f0, t, k = p
    rho = -KAPPA * bz * k
    X = x0 * math.cos(alpha0) - y0 * math.sin(alpha0)
    Y = x0 * math.sin(alpha0) + y0 * math.cos(alpha0)
    psi = alpha0 + math.asin(f0) - alpha1  # direction in the target frame
    psi = (psi + math.pi) % (2.0 * math.pi) - math.pi
    xa = X * math.cos(alpha1) + Y * math.sin(alpha1)
    ya = -X * math.sin(alpha1) + Y * math.cos(alpha1)
    s1 = math.sin(psi) + rho * (x1 - xa)
    if abs(s1) >= 1.0:
        return None
    psi1 = math.asin(s1)
    s = (psi1 - psi) / rho
    y1 = ya - (math.cos(psi1) - math.cos(psi)) / rho
    return np.array([y1, z0 + t * s, s1, t, k])


def _prior_terms(res, i, cov_scale):
    mean = np.array([res["par"][j][i] for j in range(5)], dtype=np.float64)
    diag_idx = [0, 2, 5, 9, 14]
    sig = np.sqrt(cov_scale * np.array([res["cov"][d][i] for d in diag_idx], dtype=np.float64))
    return float(res["alpha"][i]), float(res["x"][i]), mean.astype(np.float32).astype(np.float64), sig


def _map_fit(res, i, trk, cov_scale, alpha_out, x_out, p_start, bz):
    """MAP state at (alpha_out, x_out) from the prior and the tracklets."""
    a_end, x_end, mean, sig = _prior_terms(res, i, cov_scale)
    meas = []
    for l in range(6):
        j = int(res["tracklet_id"][l][i])
        if j < 0:
            continue
        sec = int(trk["chamber"][j]) // 30
        V = np.array([[trk["vyy"][j], trk["vyz"][j]], [trk["vyz"][j], trk["vzz"][j]]], dtype=np.float64)
        W = np.linalg.cholesky(np.linalg.inv(V)).T  # whitening: |W r|^2 = r^T V^-1 r
        meas.append((l, (sec + 0.5) * SECTOR, float(trk["y"][j]), float(trk["z"][j]), W))

    def resid(p):
        out = []
        q = _state_at(p, alpha_out, x_out, a_end, float(np.float32(x_end)), bz)
        out.extend((q - mean) / sig)
        for l, a, ytl, ztl, W in meas:
            q = _state_at(p, alpha_out, x_out, a, _layer_x(l), bz)
            r = np.array([ytl - (q[0] - _tilt(l) * (q[1] - ztl)), ztl - q[1]])
            out.extend(W @ r)
        return np.array(out)

    scale = np.array([0.05, 1.0, 1e-3, 1e-2, 1e-2])
    fit = least_squares(resid, p_start, x_scale=scale, xtol=1e-15, ftol=1e-15, gtol=1e-15,
                        method="lm", max_nfev=4000)
    # normal matrix from a central-difference Jacobian at the optimum
    J = np.zeros((fit.fun.shape[0], 5))
    for c in range(5):
        h = 1e-6 * scale[c]
        pp, pm = fit.x.copy(), fit.x.copy()
        pp[c] += h
        pm[c] -= h
        J[:, c] = (resid(pp) - resid(pm)) / (2 * h)
    return fit.x, 2.0 * fit.cost, np.linalg.inv(J.T @ J)


def _full(c):
    M = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            M[i, j] = M[j, i] = c[k]
            k += 1
    return M


def _follow_and_refit(tf, cov_scale=100.0):
    r = O.follow(tf.seeds, tf.tracklets, tf.params)
    rf = O.refit(r, tf.tracklets, tf.params, cov_scale=cov_scale)
    return r, rf


# The filter linearises each step at its running estimate, the fit at its
# optimum: they differ at second order in how far the estimate moves, which
# grows with a weaker prior.  Planted mistakes (a tilt sign, a gain index, a
# prior that is not widened, a skipped update) move the state by a sigma or
# more.
@pytest.mark.parametrize("cov_scale,bz,tol", [(100.0, 0.5, 0.05), (100.0, -0.5, 0.05), (1e4, 0.5, 0.2)])
def test_refit_equals_map_least_squares_without_material(cov_scale, bz, tol):
    p = G.default_params(bz=bz, material_on=0)
    tf = G.make_timeframe(160, seed=17, noise=0.2, bz=bz, params=p)
    r, rf = _follow_and_refit(tf, cov_scale)
    sel = np.nonzero((rf["status"] == 0) & (r["n_trk"] >= 2))[0]
    assert sel.size > 60
    n_two = 0
    for i in sel[:60]:
        p_ref = np.array([rf["par"][j][i] for j in range(5)])
        C = _full(rf["cov"][:, i])
        pm, chi2_min, Cm = _map_fit(r, i, tf.tracklets, cov_scale, rf["alpha"][i], rf["x"][i], p_ref, bz)
        sig = np.sqrt(np.diag(C))
        assert np.all(np.abs(pm - p_ref) <= tol * sig), (i, (pm - p_ref) / sig)
        assert rf["chi2"][i] == pytest.approx(chi2_min, rel=0.3 * tol, abs=0.5 * tol)
        Cn = np.sqrt(np.outer(np.diag(Cm), np.diag(Cm)))
        assert np.all(np.abs(C - Cm) <= 0.5 * tol * Cn + 0.03 * Cn), (i, (C - Cm) / Cn)
        assert rf["n_upd"][i] == r["n_trk"][i]
        n_two += int(r["n_trk"][i] == 2)
    assert n_two > 0  # underdetermined by the tracklets alone: the prior decides
    assert np.all(rf["x"][sel] == 300.0)


def test_refit_recovers_noiseless_truth():
    p = G.default_params(material_on=0)
    tf = G.make_timeframe(300, seed=19, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p)
    r, rf = _follow_and_refit(tf, 100.0)
    full = np.nonzero((tf.truth_ids >= 0).all(1) & (rf["status"] == 0))[0]
    assert full.size > 150
    y, z, f, t, k, ok = G.truth_at_plane({key: v[full] for key, v in tf.truth.items()},
                                         rf["alpha"][full], 300.0)
    assert ok.all()
    sig = np.sqrt(rf["cov"][[0, 2, 5, 9, 14]][:, full])
    got = rf["par"][:, full]
    truth = np.stack([y, z, f, t, k])
    # inputs are FP32 (y ~ 50 cm rounded by ~4e-6 cm); anything else is a model error
    assert np.all(np.abs(got - truth) <= 2e-3 * sig), np.abs((got - truth) / sig).max(1)
    assert np.all(rf["chi2"][full] < 1e-4)


def test_refit_pulls_are_unit_normal():
    """An honest prior (the truth at the outermost layer smeared by a known
    sigma, whose variances divided by cov_scale are handed in as the input
    covariance) and the true tracklets: the refitted state at layer 0 must
    have unit-normal pulls against the truth in all five parameters, and the
    summed update chi2 must average 2 per update (independent innovations)."""
    p = G.default_params(material_on=0)
    tf = G.make_timeframe(3000, seed=23, noise=0.0, eff=1.0, params=p)
    full = np.nonzero((tf.truth_ids >= 0).all(1))[0]
    assert full.size > 1500
    n = full.size
    cov_scale = 100.0
    rng = np.random.default_rng(77)
    ch5 = tf.tracklets["chamber"][tf.truth_ids[full, 5]]
    a5 = ((ch5 // 30) + 0.5) * SECTOR
    tr = {key: v[full] for key, v in tf.truth.items()}
    y5, z5, f5, t5, k5, ok = G.truth_at_plane(tr, a5, _layer_x(5))
    assert ok.all()
    sig = np.stack([np.full(n, 0.3), np.full(n, 3.0), np.full(n, 0.01), np.full(n, 0.02), 0.1 * np.abs(k5)])
    prior = np.stack([y5, z5, f5, t5, k5]) + rng.normal(size=(5, n)) * sig
    cov = np.zeros((15, n), np.float32)
    cov[[0, 2, 5, 9, 14]] = (sig ** 2 / cov_scale).astype(np.float32)
    res = dict(alpha=a5.astype(np.float32), x=np.full(n, _layer_x(5), np.float32),
               par=prior.astype(np.float32), cov=cov, status=np.zeros(n, np.int32),
               tracklet_id=np.ascontiguousarray(tf.truth_ids[full].T))
    rf = O.refit(res, tf.tracklets, p, cov_scale=cov_scale)
    good = rf["status"] == 0
    assert good.mean() > 0.99
    y, z, f, t, k, ok0 = G.truth_at_plane({key: v[good] for key, v in tr.items()}, rf["alpha"][good], 300.0)
    truth = np.stack([y, z, f, t, k])
    pull = (rf["par"][:, good] - truth) / np.sqrt(rf["cov"][[0, 2, 5, 9, 14]][:, good])
    for c in range(5):
        assert abs(pull[c].mean()) < 0.1, (c, pull[c].mean())
        assert 0.9 < pull[c].std() < 1.1, (c, pull[c].std())
    assert np.all(rf["n_upd"][good] == 6)
    assert 11.0 < rf["chi2"][good].mean() < 13.0, rf["chi2"][good].mean()


def test_inward_material_gives_back_the_outward_loss():
    rng = np.random.default_rng(5)
    for _ in range(50):
        st = np.array([0.35, 300.0, rng.uniform(-30, 30), rng.uniform(-100, 100), rng.uniform(-0.5, 0.5),
                       rng.uniform(-0.8, 0.8), rng.choice([-1, 1]) * rng.uniform(0.1, 3.0)])
        c = np.diag([1e-2, 1e-2, 1e-6, 1e-6, 1e-4])[np.tril_indices(5)]
        ok1, s_out, c_out = O.material(st, c)
        ok2, s_in, c_in = O.material_inward(st, c)
        assert ok1 and ok2
        m = 0.13957039
        t2 = 1 + st[5] ** 2
        e = lambda s: math.sqrt(t2 / s[6] ** 2 + m * m)  # noqa: E731
        # the same loss, taken out going outward and given back going inward
        assert e(st) - e(s_out) == pytest.approx(e(s_in) - e(st), rel=1e-12)
        assert abs(s_in[6]) < abs(st[6]) < abs(s_out[6])
        assert np.sign(s_in[6]) == np.sign(st[6])
        # scattering widens the same terms by the same amounts in both directions
        for idx in (5, 9):
            assert c_out[idx] == pytest.approx(c_in[idx], rel=1e-12)
        # and once each direction's energy-loss Jacobian (finite differences of
        # its state map) is taken off, the added angular block is the same
        q = []
        for step in (O.material, O.material_inward):
            J = np.eye(5)
            for j in (2, 3, 4):
                h = 1e-6 * max(1.0, abs(st[2 + j]))
                sp, sm = st.copy(), st.copy()
                sp[2 + j] += h
                sm[2 + j] -= h
                J[:, j] = (step(sp, np.zeros(15))[1][2:7] - step(sm, np.zeros(15))[1][2:7]) / (2 * h)
            _, _, c0 = step(st, np.zeros(15))
            Ji = np.linalg.inv(J)
            q.append(Ji @ _full(c0) @ Ji.T)
        np.testing.assert_allclose(q[0][2:, 2:], q[1][2:, 2:], rtol=1e-5, atol=1e-9 * np.abs(q[0]).max())
        # positions and angles are untouched
        np.testing.assert_array_equal(s_in[:6], st[:6])


def test_refit_skips_unmatched_and_invalid_tracks():
    tf = G.make_timeframe(400, seed=29, noise=0.3)
    r = O.follow(tf.seeds, tf.tracklets, tf.params)
    rf = O.refit(r, tf.tracklets, tf.params)
    few = r["n_trk"] < 2
    assert few.any()
    assert np.all(rf["status"][few] == 8)
    assert np.all(rf["n_upd"][few] == 0)
    matched = ~few & ((r["status"] & 4) == 0)
    assert np.all(rf["status"][matched] != 8)
    assert np.mean(rf["status"][matched] == 0) > 0.99
    # a tracklet id outside the input, or a SEED_INVALID follower status, is skipped
    bad = {k: np.array(v, copy=True) for k, v in r.items()}
    i = int(np.nonzero(matched)[0][0])
    l = int(np.nonzero(bad["tracklet_id"][:, i] >= 0)[0][0])
    bad["tracklet_id"][l, i] = tf.n_tracklets
    i2 = int(np.nonzero(matched)[0][1])
    bad["status"][i2] = 4
    rb = O.refit(bad, tf.tracklets, tf.params)
    assert rb["status"][i] == 8 and rb["status"][i2] == 8
    others = np.ones(tf.n_seeds, bool)
    others[[i, i2]] = False
    np.testing.assert_array_equal(rb["par"][:, others], rf["par"][:, others])


def test_refit_output_frame_is_the_layer0_sector():
    tf = G.make_timeframe(600, seed=31, noise=0.2)
    r, rf = _follow_and_refit(tf)
    ok = np.nonzero(rf["status"] == 0)[0]
    secs = np.round(rf["alpha"][ok] / SECTOR - 0.5)
    assert np.allclose(rf["alpha"][ok], (secs + 0.5) * SECTOR, atol=1e-12)
    lim = 300.0 * math.tan(SECTOR / 2)
    has0 = r["tracklet_id"][0, ok] >= 0
    # where layer 0 has a tracklet, the refit ends in that tracklet's sector
    ch0 = tf.tracklets["chamber"][r["tracklet_id"][0, ok[has0]]]
    np.testing.assert_array_equal(secs[has0].astype(int), ch0 // 30)
    assert np.all(np.abs(rf["par"][0, ok]) < lim + 2.0)


def test_inward_refit_undoes_the_outward_material():
    """Carry a state outward over the six layers with material (the
    follower's step), then refit it inward with tracklets that carry no
    information (huge variances): the refit gives each layer's energy loss
    back, so q/pT at layer 0 returns to its value before layer 0's material
    up to second order in the loss (~1e-4 relative), where a loss taken
    with the wrong sign would miss by ~5 %."""
    p = G.default_params(material_on=1)
    rng = np.random.default_rng(9)
    n_ok = 0
    for _ in range(40):
        k0 = rng.choice([-1, 1]) * rng.uniform(0.4, 3.0)
        st = np.array([(3 + 0.5) * SECTOR, 299.0, rng.uniform(-20, 20), rng.uniform(-100, 100),
                       rng.uniform(-0.3, 0.3), rng.uniform(-0.8, 0.8), k0])
        c = np.diag([1e-2, 1e-2, 1e-6, 1e-6, 1e-4])[np.tril_indices(5)]
        ok, st0, c0 = O.propagate(st, c, 300.0, p["bz"])[:3]
        assert ok
        s, cc, sec, chambers, ok = st0.copy(), c0.copy(), 3, [], True
        for l in range(6):
            ok, s, cc, sec, ch = O.to_layer(s, cc, sec, l, p)
            if not ok or ch < 0:
                break
            chambers.append(ch)
        if not ok or len(chambers) < 6:
            continue
        n_ok += 1
        trk = dict(chamber=np.array(chambers, np.int32), y=np.zeros(6, np.float32), z=np.zeros(6, np.float32),
                   vyy=np.full(6, 1e10, np.float32), vzz=np.full(6, 1e10, np.float32),
                   vyz=np.zeros(6, np.float32))
        cdiag = np.zeros((15, 1), np.float32)
        cdiag[[0, 2, 5, 9, 14], 0] = [1e-4, 1e-4, 1e-8, 1e-8, 1e-8]
        res = dict(alpha=np.array([s[0]], np.float32), x=np.array([s[1]], np.float32),
                   par=s[2:7].astype(np.float32).reshape(5, 1), cov=cdiag, status=np.zeros(1, np.int32),
                   tracklet_id=np.arange(6, dtype=np.int32).reshape(6, 1))
        rf = O.refit(res, trk, p, cov_scale=1.0)
        assert rf["status"][0] == 0 and rf["n_upd"][0] == 6
        assert rf["x"][0] == 300.0
        k_out = s[6]
        assert abs(k_out) > abs(st0[6])  # the outward pass lost momentum
        assert rf["par"][4][0] == pytest.approx(st0[6], rel=3e-4)
        assert rf["par"][2][0] == pytest.approx(st0[4], abs=2e-4)
    assert n_ok > 20
