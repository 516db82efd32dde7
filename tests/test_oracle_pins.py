"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against a closed form, an invariant, an
independent formulation, brute force or a number the paper states, so that a
dropped term, a flipped sign, a wrong index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from synth import make_timeframe, make_workload, efficiency_purity
from synth import timeframe as G

HERE = os.path.dirname(os.path.abspath(__file__))
KAPPA = 2.99792458e-3
rng = np.random.default_rng(1234)


def _random_state(alpha=0.35, x=300.0):
    f = rng.uniform(-0.6, 0.6)
    t = rng.uniform(-1.0, 1.0)
    k = rng.choice([-1, 1]) * rng.uniform(0.05, 3.0)
    return np.array([alpha, x, rng.uniform(-40, 40), rng.uniform(-200, 200), f, t, k])


def _random_cov():
    A = rng.normal(size=(5, 5)) * np.array([0.1, 0.2, 2e-3, 2e-3, 0.02])[:, None]
    M = A @ A.T + np.diag([1e-2, 1e-2, 1e-6, 1e-6, 1e-4])
    return np.array([M[i, j] for i in range(5) for j in range(i + 1)])


def _full(c):
    M = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            M[i, j] = M[j, i] = c[k]
            k += 1
    return M


# ---------------------------------------------------------------- paper numbers
def test_geometry_matches_paper_constants():
    gold = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    c = O.constants()
    assert c["n_sectors"] == gold["n_sectors"]["value"]
    assert c["n_stacks"] == gold["n_stacks"]["value"]
    assert c["n_layers"] == gold["n_layers"]["value"]
    assert c["n_chambers"] == 18 * 5 * 6
    assert c["drift_length"] == gold["drift_length_cm"]["value"]
    assert c["tilt_deg"] == gold["pad_tilt_deg"]["value"]
    assert c["lorentz_deg"] == gold["lorentz_angle_deg"]["value"]
    p = G.default_params()
    assert p["dy_gate_sigma"] == gold["dy_gate_sigma"]["value"]
    assert p["bz"] == gold["bz_tesla"]["value"]


# ---------------------------------------------------------------- transport
def _circle_reference(st, x1, bz):
    """Independent circle geometry: centre + radius, intersection with x = x1,
    arc from the turning angle."""
    _, x0, y0, z0, f0, t, k = st
    rho = -KAPPA * bz * k
    phi0 = math.asin(f0)
    xc = x0 - math.sin(phi0) / rho
    yc = y0 + math.cos(phi0) / rho
    R = 1.0 / abs(rho)
    d = R * R - (x1 - xc) ** 2
    y1 = yc - math.copysign(1.0, rho) * math.sqrt(d)
    vx = -math.copysign(1.0, rho) * (y1 - yc) / R
    vy = math.copysign(1.0, rho) * (x1 - xc) / R
    phi1 = math.atan2(vy, vx)
    dphi = (phi1 - phi0 + math.pi) % (2 * math.pi) - math.pi
    s = dphi / rho
    return y1, z0 + t * s, math.sin(phi1)


@pytest.mark.parametrize("dx", [10.0, 12.6, 63.0, -25.0])
def test_helix_matches_circle_intersection(dx):
    for _ in range(50):
        st = _random_state()
        ok, out, _, _ = O.propagate(st, _random_cov(), st[1] + dx, 0.5)
        if not ok:
            continue
        y1, z1, f1 = _circle_reference(st, st[1] + dx, 0.5)
        assert out[2] == pytest.approx(y1, abs=1e-10, rel=1e-10)
        assert out[3] == pytest.approx(z1, abs=1e-9, rel=1e-10)
        assert out[4] == pytest.approx(f1, abs=1e-12)
        assert out[1] == st[1] + dx


def test_zero_field_is_a_straight_line():
    for _ in range(30):
        st = _random_state()
        dx = 37.0
        ok, out, _, _ = O.propagate(st, _random_cov(), st[1] + dx, 0.0)
        assert ok
        f = st[4]
        assert out[2] == pytest.approx(st[2] + dx * f / math.sqrt(1 - f * f), abs=1e-11)
        assert out[3] == pytest.approx(st[3] + st[5] * dx / math.sqrt(1 - f * f), abs=1e-11)
        assert out[4] == st[4]


def _fd_jacobian(fun, p, steps):
    J = np.zeros((5, 5))
    for j in range(5):
        h = steps[j]
        pp, pm = p.copy(), p.copy()
        pp[2 + j] += h
        pm[2 + j] -= h
        J[:, j] = (fun(pp)[2:7] - fun(pm)[2:7]) / (2 * h)
    return J


STEPS = np.array([1e-4, 1e-4, 1e-6, 1e-6, 1e-6])


@pytest.mark.parametrize("bz", [0.5, -0.5, 0.0])
def test_transport_jacobian_matches_finite_differences(bz):
    for _ in range(40):
        st = _random_state()
        x1 = st[1] + rng.choice([10.0, 12.6, 40.0, -12.6])

        def fun(p):
            ok, out, _, _ = O.propagate(p, np.eye(5)[np.tril_indices(5)], x1, bz)
            assert ok
            return out
        ok, _, _, J = O.propagate(st, _random_cov(), x1, bz)
        if not ok:
            continue
        Jfd = _fd_jacobian(fun, st, STEPS)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-7 * np.abs(Jfd).max())


def test_transport_jacobian_small_curvature_series_branch():
    # |w| < 1e-3 exercises the asin(w)/w series: very stiff track, short step
    st = np.array([0.0, 300.0, 1.0, 2.0, 0.1, 0.3, 0.02])
    x1 = 305.0

    def fun(p):
        return O.propagate(p, np.eye(5)[np.tril_indices(5)], x1, 0.5)[1]
    ok, _, _, J = O.propagate(st, _random_cov(), x1, 0.5)
    Jfd = _fd_jacobian(fun, st, np.array([1e-4, 1e-4, 1e-6, 1e-6, 1e-4]))
    np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-9)


def test_transport_is_reversible():
    for _ in range(30):
        st, c = _random_state(), _random_cov()
        ok1, a, ca, _ = O.propagate(st, c, st[1] + 62.0, 0.5)
        if not ok1:
            continue
        ok2, b, cb, _ = O.propagate(a, ca, st[1], 0.5)
        assert ok2
        np.testing.assert_allclose(b, st, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(cb, c, rtol=1e-9, atol=1e-14)


def test_transport_covariance_is_j_c_jt_and_stays_pd():
    for _ in range(20):
        st, c = _random_state(), _random_cov()
        ok, _, c1, J = O.propagate(st, c, st[1] + 12.6, 0.5)
        if not ok:
            continue
        M = J @ _full(c) @ J.T
        np.testing.assert_allclose(_full(c1), M, rtol=1e-12, atol=1e-16)
        assert O.cov_is_pd(c1)


def test_snp_limit_fails_transport():
    st = np.array([0.0, 300.0, 0.0, 0.0, 0.94, 0.1, 2.0])
    # rho < 0 for q2pt > 0 at +Bz: snp decreases outward; flip the field to increase it
    ok, _, _, _ = O.propagate(st, _random_cov(), 340.0, -0.5)
    assert not ok


def test_undefined_snp_fails_transport_and_rotation():
    """A sin(phi) that is not a number (a NaN q/pT after one step) cannot lie
    below the limit: the transport and the rotation fail, and a seed with a
    NaN q/pT ends with PROP_FAIL at its first layer, no tracklet attached."""
    st = np.array([0.0, 300.0, 0.0, 0.0, 0.2, 0.1, np.nan])
    ok, _, _, _ = O.propagate(st, _random_cov(), 310.0, 0.5)
    assert not ok
    st = np.array([0.0, 300.0, 0.0, 0.0, np.nan, 0.1, 1.0])
    ok, _, _, _ = O.rotate(st, _random_cov(), math.radians(20.0), 0.5)
    assert not ok
    tf = make_workload("tiny")
    s2 = {k: v.copy() for k, v in tf.seeds.items()}
    s2["q2pt"][:6] = np.nan
    r = O.follow(s2, tf.tracklets, tf.params, seed_index=np.arange(8))
    assert np.all(r["status"][:6] == O.STATUS_PROP_FAIL)
    assert np.all(r["tracklet_id"][:, :6] == -1) and np.all(r["n_trk"][:6] == 0)


# ---------------------------------------------------------------- rotation
def test_rotation_round_trip_is_identity():
    for _ in range(30):
        st, c = _random_state(alpha=0.5), _random_cov()
        ok, a, ca, J1 = O.rotate(st, c, 0.5 + math.radians(20.0), 0.5)
        if not ok:
            continue
        ok2, b, cb, J2 = O.rotate(a, ca, 0.5, 0.5)
        assert ok2
        np.testing.assert_allclose(b, st, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(cb, c, rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(J2 @ J1, np.eye(5), atol=1e-12)


def test_rotation_keeps_the_global_point_and_direction():
    for _ in range(20):
        st = _random_state(alpha=1.1)
        ok, a, _, _ = O.rotate(st, _random_cov(), 1.1 - 0.2, 0.5)
        assert ok
        g0 = (st[1] * math.cos(st[0]) - st[2] * math.sin(st[0]),
              st[1] * math.sin(st[0]) + st[2] * math.cos(st[0]))
        g1 = (a[1] * math.cos(a[0]) - a[2] * math.sin(a[0]),
              a[1] * math.sin(a[0]) + a[2] * math.cos(a[0]))
        np.testing.assert_allclose(g1, g0, atol=1e-10)
        assert math.asin(a[4]) + a[0] == pytest.approx(math.asin(st[4]) + st[0], abs=1e-12)


@pytest.mark.parametrize("bz", [0.5, 0.0])
def test_rotation_jacobian_matches_finite_differences(bz):
    """The first-order covariance transform equals the derivative of the exact
    map: rotate the point, then slide along the helix back to the new plane."""
    for _ in range(30):
        st = _random_state(alpha=0.2)
        a_new = 0.2 + rng.uniform(-0.3, 0.3)
        ok, nominal, _, J = O.rotate(st, _random_cov(), a_new, bz)
        if not ok:
            continue
        x_plane = nominal[1]

        def fun(p):
            ok1, r, _, _ = O.rotate(p, np.eye(5)[np.tril_indices(5)], a_new, bz)
            ok2, r2, _, _ = O.propagate(r, np.eye(5)[np.tril_indices(5)], x_plane, bz)
            assert ok1 and ok2
            return r2
        Jfd = _fd_jacobian(fun, st, STEPS)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-7 * np.abs(Jfd).max())


# ---------------------------------------------------------------- material
def test_bethe_minimum_ionising_near_betagamma_3_5():
    bg = np.exp(np.linspace(math.log(0.5), math.log(1000.0), 4000))
    v = np.array([O.bethe(b) for b in bg])
    i = int(np.argmin(v))
    assert 3.0 < bg[i] < 4.2
    assert 1.5 < v[i] < 2.2  # MeV cm^2/g for Z/A = 0.5
    assert v[0] > 3 * v[i]   # steep 1/beta^2 rise at low momentum
    assert v[-1] > v[i]      # relativistic rise


def test_highland_at_one_radiation_length():
    # at x/X0 = 1 the logarithmic term vanishes: theta0 = 13.6 MeV / (beta p)
    assert O.highland(1.0, 1.0, 1.0) == pytest.approx(0.0136 ** 2, rel=1e-14)
    assert O.highland(2.0, 1.0, 1.0) == pytest.approx((0.0136 / 2) ** 2, rel=1e-14)


def test_material_widens_angles_and_lowers_momentum():
    for _ in range(20):
        st, c = _random_state(), _random_cov()
        ok, s1, c1 = O.material(st, c)
        assert ok
        d = c1 - c
        # position block untouched, angle/curvature variances grow
        assert np.all(d[[0, 1, 2]] == 0)
        assert d[5] > 0 and d[9] > 0
        assert abs(s1[6]) > abs(st[6])  # |q/pT| grows as p drops
        assert s1[6] * st[6] > 0
        np.testing.assert_array_equal(s1[:6], st[:6])
        assert O.cov_is_pd(c1)



# The material reading's constants (not the paper's): one step per layer of
# x/X0 = 0.04 and 1 g/cm^2 at normal incidence, a pion.
MAT_X0 = 0.04
MAT_RHO = 1.0
M_PION = 0.13957039


def _direction(f, t):
    """Unit direction of a track with sin(phi) = f, tan(lambda) = t in the
    local frame (x along the layer normal)."""
    lam = math.atan(t)
    phi = math.asin(f)
    return np.array([math.cos(lam) * math.cos(phi), math.cos(lam) * math.sin(phi), math.sin(lam)])


def _path_through_layer(f, t):
    """Path length through a slab normal to x, per unit thickness: 1 over the
    direction's x component (geometry, not the oracle's expression)."""
    return 1.0 / _direction(f, t)[0]


def _material_states():
    # tgl away from 0: there the first-order q2pt variance (theta^2 tgl^2
    # q2pt^2) vanishes and the second-order term q2pt^2 theta^4 / 2, which a
    # linearised filter does not carry, would dominate the Monte-Carlo
    return [np.array([0.3, 300.0, 4.0, 20.0, f, t, k])
            for f, t, k in [(0.5, 0.8, 2.0), (-0.7, -0.4, -1.3), (0.1, 0.35, 3.0), (0.0, 1.1, -0.4),
                            (-0.3, 0.6, 0.25)]]


def test_bethe_slope_matches_finite_differences():
    for bg in [0.4, 1.0, 3.5, 10.0, 200.0]:
        h = 1e-5 * bg
        fd = (O.bethe(bg + h) - O.bethe(bg - h)) / (2 * h)
        assert O.bethe_dbg(bg) == pytest.approx(fd, rel=1e-7, abs=1e-9)


def _scatter_mc(f, t, k, theta2, n, seed):
    """Two independent projected angles of variance theta2 about the track
    direction, applied to the direction exactly; the momentum is unchanged.
    Returns samples of (snp, tgl, q2pt) after the deflection."""
    g = np.random.default_rng(seed)
    d = _direction(f, t)
    e1 = np.array([-d[1], d[0], 0.0]) / math.hypot(d[0], d[1])  # transverse, in the bending plane
    e2 = np.cross(d, e1)                                         # completes the right-handed triad
    a1 = g.normal(0.0, math.sqrt(theta2), n)
    a2 = g.normal(0.0, math.sqrt(theta2), n)
    dn = d[None, :] + np.tan(a1)[:, None] * e1[None, :] + np.tan(a2)[:, None] * e2[None, :]
    dn /= np.linalg.norm(dn, axis=1)[:, None]
    ct = np.hypot(dn[:, 0], dn[:, 1])           # cos(lambda')
    snp = dn[:, 1] / ct
    tgl = dn[:, 2] / ct
    q2pt = k * (d[0] ** 2 + d[1] ** 2) ** 0.5 / ct  # q/(p cos(lambda')), p fixed
    return np.stack([snp, tgl, q2pt], axis=1)


def _material_state_jacobian(st, inward=False):
    step = O.material_inward if inward else O.material
    J = np.eye(5)
    for j in (2, 3, 4):
        h = 1e-6 * max(1.0, abs(st[2 + j]))
        sp, sm = st.copy(), st.copy()
        sp[2 + j] += h
        sm[2 + j] -= h
        okp, op, _ = step(sp, np.zeros(15))
        okm, om, _ = step(sm, np.zeros(15))
        assert okp and okm
        J[:, j] = (op[2:7] - om[2:7]) / (2 * h)
    return J


@pytest.mark.parametrize("inward", [False, True])
def test_material_scattering_matches_monte_carlo_of_two_angles(inward):
    """The covariance the step adds, against the sample covariance of two
    projected scattering angles of the Highland variance (over the geometric
    path) carried through the exact direction geometry, then through the
    step's own energy-loss Jacobian (taken by finite differences)."""
    step = O.material_inward if inward else O.material
    for n_state, st in enumerate(_material_states()):
        f, t, k = st[4], st[5], st[6]
        p = math.sqrt(1 + t * t) / abs(k)
        beta = p / math.hypot(p, M_PION)
        theta2 = O.highland(p, beta, MAT_X0 * _path_through_layer(f, t))
        smp = _scatter_mc(f, t, k, theta2, 400_000, 100 + n_state)
        Q = np.zeros((5, 5))
        Q[2:, 2:] = np.cov(smp, rowvar=False)
        J = _material_state_jacobian(st, inward)
        want = J @ Q @ J.T
        ok, _, c1 = step(st, np.zeros(15))
        assert ok
        got = _full(c1)
        # diagonal within the Monte-Carlo error (~0.3 % at 400k samples)
        for i in (2, 3, 4):
            assert got[i, i] == pytest.approx(want[i, i], rel=0.015), (st, i)
        # the tgl-q2pt correlation (both come from the polar angle)
        assert got[4, 3] == pytest.approx(want[4, 3], rel=0.015, abs=0.01 * math.sqrt(want[3, 3] * want[4, 4]))
        # nothing outside the angular block; snp uncorrelated with the polar angle
        assert np.all(got[:2, :] == 0)
        for i, j in ((3, 2), (4, 2)):
            assert abs(got[i, j] - want[i, j]) < 0.01 * math.sqrt(want[i, i] * want[j, j]) + 1e-300


@pytest.mark.parametrize("inward", [False, True])
def test_material_energy_change_is_the_bethe_loss_over_the_path(inward):
    """E(p) - E(p') equals the Bethe mean loss at the entry momentum times the
    areal density along the geometric path (the reverse going inward); the
    angles and position do not change."""
    step = O.material_inward if inward else O.material
    sign = -1.0 if inward else 1.0
    for st in _material_states():
        f, t, k = st[4], st[5], st[6]
        ok, s1, _ = step(st, np.zeros(15))
        assert ok
        np.testing.assert_array_equal(s1[:6], st[:6])
        p0 = math.sqrt(1 + t * t) / abs(k)
        p1 = math.sqrt(1 + t * t) / abs(s1[6])
        assert s1[6] * k > 0
        de = math.hypot(p0, M_PION) - math.hypot(p1, M_PION)
        want = sign * O.bethe(p0 / M_PION) * MAT_RHO * _path_through_layer(f, t) * 1e-3
        assert de == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("inward", [False, True])
def test_material_covariance_transport_is_the_jacobian_of_the_state_map(inward):
    """Apart from the added scattering, the step carries the covariance by the
    Jacobian of its own state change: C'(C) - C'(0) = J C J^T, with J from
    finite differences of the step's (snp, tgl, q2pt) map."""
    step = O.material_inward if inward else O.material
    for st in _material_states():
        J = _material_state_jacobian(st, inward)
        # the loss depends on q2pt through p and the Bethe slope, and on the
        # path length through snp and tgl
        assert J[4, 4] != pytest.approx(st[6] / st[6], abs=1e-9)
        for _ in range(3):
            c = _random_cov()
            ok, _, c1 = step(st, c)
            ok0, _, c0 = step(st, np.zeros(15))
            assert ok and ok0
            got = _full(c1) - _full(c0)
            want = J @ _full(c) @ J.T
            scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-7 * scale.max())
            assert np.all(np.abs(got - want) <= 2e-6 * scale + 1e-300)

# ---------------------------------------------------------------- update
def _info_form(st, c, layer, meas):
    """Information-filter posterior (textbook alternative to the gain form)."""
    tt = G.pad_tilt_tan(layer)
    H = np.array([[1.0, -tt, 0, 0, 0], [0, 1.0, 0, 0, 0]])
    y_tl, z_tl, vyy, vzz, vyz = meas
    m_eff = np.array([y_tl - tt * z_tl, z_tl])
    V = np.array([[vyy, vyz], [vyz, vzz]])
    Ci = np.linalg.inv(_full(c))
    Vi = np.linalg.inv(V)
    Cp = np.linalg.inv(Ci + H.T @ Vi @ H)
    p = np.asarray(st[2:7])
    pp = Cp @ (Ci @ p + H.T @ Vi @ m_eff)
    d = pp - p
    e = m_eff - H @ pp
    chi2 = d @ Ci @ d + e @ Vi @ e
    return pp, Cp, chi2


@pytest.mark.parametrize("layer", [0, 1])
def test_kalman_update_equals_information_form(layer):
    for _ in range(30):
        st, c = _random_state(), _random_cov()
        meas = (st[2] + rng.normal(0, 0.2), st[3] + rng.normal(0, 3), 0.04 ** 2,
                64 / 12, rng.uniform(-0.01, 0.01))
        chi2, s1, c1 = O.update(st, c, layer, meas)
        pp, Cp, chi2_ref = _info_form(st, c, layer, meas)
        np.testing.assert_allclose(s1[2:7], pp, rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(_full(c1), Cp, rtol=1e-7, atol=1e-14)
        assert chi2 == pytest.approx(chi2_ref, rel=1e-8)
        assert chi2 == pytest.approx(O.chi2(st, c, layer, meas), rel=1e-14)


def test_joseph_form_equals_standard_and_stays_pd():
    for _ in range(30):
        st, c = _random_state(), _random_cov()
        meas = (st[2] + 0.05, st[3] - 1.0, 0.04 ** 2, 64 / 12, 0.0)
        _, a, ca = O.update(st, c, 2, meas, joseph=False)
        _, b, cb = O.update(st, c, 2, meas, joseph=True)
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(ca, cb, rtol=1e-9, atol=1e-12 * np.abs(ca).max())
        assert O.cov_is_pd(ca) and O.cov_is_pd(cb)
        M = _full(ca)
        assert np.all(np.diag(M) <= np.diag(_full(c)) + 1e-18)


def test_pad_tilt_sign_residual_vanishes_on_tilted_measurement():
    # A tracklet measured on a tilted pad at z_tl for a track at (y, z) reads
    # y - tan(tau) (z - z_tl) (generator's detector model): zero residual in y.
    for layer in range(6):
        st, c = _random_state(), _random_cov()
        z_tl = st[3] + 3.0
        y_tl = st[2] - G.pad_tilt_tan(layer) * (st[3] - z_tl)
        # a huge z variance removes the z residual from the chi2
        chi2 = O.chi2(st, c, layer, (y_tl, z_tl, 1e-4, 1e12, 0.0))
        assert chi2 < 1e-9
        wrong = st[2] + G.pad_tilt_tan(layer) * (st[3] - z_tl)
        assert O.chi2(st, c, layer, (wrong, z_tl, 1e-4, 1e12, 0.0)) > 1e-2


# ---------------------------------------------------------------- follower
def test_zero_noise_truth_is_recovered_exactly():
    """No smearing, no noise, every crossing measured at its true z, no
    material: the follower must pick every true tracklet with chi2 ~ 0."""
    p = G.default_params(material_on=0, n_sigma_road=3.0)
    tf = make_timeframe(400, seed=7, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p)
    r = O.follow(tf.seeds, tf.tracklets, tf.params)
    full = (tf.truth_ids >= 0).all(1)
    assert full.sum() > 200
    np.testing.assert_array_equal(r["tracklet_id"].T[full], tf.truth_ids[full])
    # inputs are FP32: y ~ 50 cm is rounded by ~4e-6 cm against sigma ~ 0.04 cm,
    # i.e. chi2 ~ 1e-8 per layer; any modelling error gives chi2 of order 1
    assert np.all(r["chi2"][full] < 1e-5)
    assert r["chi2"][full].mean() < 1e-6
    # every truth tracklet of every seed is found where the track reached the TRD
    got = (r["tracklet_id"].T == tf.truth_ids) | (tf.truth_ids < 0)
    assert got.mean() > 0.995


def test_zero_noise_with_pad_rows_assigns_truth():
    p = G.default_params(material_on=0)
    tf = make_timeframe(400, seed=8, noise=0.0, eff=1.0, smear=False, snap_z=True, params=p)
    r = O.follow(tf.seeds, tf.tracklets, tf.params)
    full = (tf.truth_ids >= 0).all(1)
    np.testing.assert_array_equal(r["tracklet_id"].T[full], tf.truth_ids[full])


def test_dy_gate_at_four_sigma():
    """Sec. 3: a tracklet whose deflection deviates by more than 4 sigma is
    excluded.  Shift the true tracklet's dy by 3.9 and 4.1 of the generator's
    own sigma and check acceptance."""
    p = G.default_params(material_on=0)
    tf = make_timeframe(200, seed=9, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p)
    ok = np.nonzero((tf.truth_ids[:, 0] >= 0))[0]
    j = tf.truth_ids[ok, 0]
    # generator's sigma at the true angle of the crossing (dy = 3 cm * (tan phi - tan psi))
    dy = tf.tracklets["dy"][j].astype(np.float64)
    u = dy / 3.0
    sig = np.sqrt(0.04 ** 2 + (0.1 * u) ** 2)
    for k, expect in ((3.9, True), (4.1, False)):
        t2 = {kk: v.copy() for kk, v in tf.tracklets.items()}
        t2["dy"][j] = (dy + k * sig).astype(np.float32)
        r = O.follow(tf.seeds, t2, tf.params, seed_index=ok)
        got = r["tracklet_id"][0] == j
        assert got.mean() > 0.97 if expect else got.mean() < 0.03


def test_brute_force_scan_equals_chamber_buckets():
    tf = make_workload("tiny", seed=3)
    a = O.follow(tf.seeds, tf.tracklets, tf.params)
    b = O.follow(tf.seeds, tf.tracklets, tf.params, brute=True)
    for k in ("tracklet_id", "n_trk", "status", "par", "cov", "chi2"):
        np.testing.assert_array_equal(a[k], b[k])


def test_event_rotated_by_one_sector_gives_identical_results():
    tf = make_workload("tiny", seed=4)
    a = O.follow(tf.seeds, tf.tracklets, tf.params)
    s2 = dict(tf.seeds)
    s2["alpha"] = (tf.seeds["alpha"].astype(np.float64) + math.radians(20.0)).astype(np.float32)
    t2 = dict(tf.tracklets)
    t2["chamber"] = ((tf.tracklets["chamber"] + 30) % 540).astype(np.int32)
    b = O.follow(s2, t2, tf.params)
    np.testing.assert_array_equal(a["tracklet_id"], b["tracklet_id"])
    np.testing.assert_array_equal(a["status"], b["status"])
    # alpha + 20 deg is rounded to FP32 (~2.4e-7 rad, ~7e-5 cm at 290 cm): compare
    # in units of each parameter's own sigma
    sig = np.sqrt(a["cov"][[0, 2, 5, 9, 14]])
    assert np.all(np.abs(a["par"] - b["par"]) <= 1e-2 * sig)
    # a y shift of ~4e-5 cm against sigma_y ~ 0.04 cm moves chi2 by ~2e-3
    np.testing.assert_allclose(a["chi2"], b["chi2"], atol=1e-2)


def test_tiny_efficiency_and_purity():
    tf = make_workload("tiny")
    r = O.follow(tf.seeds, tf.tracklets, tf.params)
    ep = efficiency_purity(r["tracklet_id"], tf.truth_ids)
    assert ep["efficiency_reachable"] > 0.97
    assert ep["purity"] > 0.98


def test_seed_validation():
    tf = make_workload("tiny")
    s2 = {k: v.copy() for k, v in tf.seeds.items()}
    s2["cov"][0, :5] = -1.0    # negative variance: not positive definite
    s2["snp"][5:10] = 0.97    # beyond the sin(phi) limit
    r = O.follow(s2, tf.tracklets, tf.params, seed_index=np.arange(12))
    assert np.all(r["status"][:10] == O.STATUS_SEED_INVALID)
    assert np.all(r["tracklet_id"][:, :10] == -1)


def _exhaustive_best(seed_st, seed_c, tracklets, params):
    """All paths through the layers under the cuts, by depth-first search
    over the oracle's per-layer steps (independent of its beam logic).
    Returns (ids, score) of the best path at the deepest layer reached."""
    phi = seed_st[0] + math.atan2(seed_st[2], seed_st[1])
    sec = int(math.floor((phi % (2 * math.pi)) / math.radians(20.0))) % 18
    ok, st, c, _ = O.rotate(seed_st, seed_c, math.radians(20.0 * (sec + 0.5)), params["bz"])
    assert ok
    best = {}

    def dfs(st, c, sec, l, score, nmiss, ids):
        if l == 6:
            best.setdefault(6, []).append((score, tuple(ids)))
            return
        okl, st1, c1, sec1, ch = O.to_layer(st, c, sec, l, params)
        if not okl:
            return
        exts = []
        if ch >= 0:
            cid, cchi = O.candidates(st1, c1, l, ch, tracklets, params)
            exts += [(score + x, j) for j, x in zip(cid, cchi)]
        if nmiss < params["max_missing"]:
            exts.append((score + params["p_miss"], -1))
        for sc, j in exts:
            best.setdefault(l + 1, []).append((sc, tuple(ids + [j])))
            if j >= 0:
                meas = (tracklets["y"][j], tracklets["z"][j], tracklets["vyy"][j],
                        tracklets["vzz"][j], tracklets["vyz"][j])
                _, st2, c2 = O.update(st1, c1, l, meas)
                dfs(st2, c2, sec1, l + 1, sc, nmiss, ids + [j])
            else:
                dfs(st1, c1, sec1, l + 1, sc, nmiss + 1, ids + [j])

    dfs(st, c, sec, 0, 0.0, 0, [])
    if not best:
        return None, None
    deepest = max(best)
    sc, ids = min(best[deepest])
    return list(ids) + [-1] * (6 - len(ids)), sc, len(best[deepest])


def test_beam_search_equals_exhaustive_enumeration():
    """With N at least the number of live paths, keeping the best N per layer
    is exhaustive search; the beam result must be the best deepest path."""
    p = G.default_params(n_sigma_road=5.0, n_hyp=4096, max_missing=2, chi2_cut=25.0)
    tf = make_timeframe(40, seed=11, noise=4.0, params=p)
    # crowd the roads: copy every truth tracklet twice with a small y offset
    sig = tf.truth_ids[tf.truth_ids >= 0]
    extra = {k: v[sig] for k, v in tf.tracklets.items()}
    extra["y"] = extra["y"] + np.float32(0.03)
    trk = {k: np.concatenate([tf.tracklets[k], extra[k]]) for k in tf.tracklets}
    r = O.follow(tf.seeds, trk, p)
    checked = 0
    for i in range(tf.n_seeds):
        st = np.array([tf.seeds[k][i] for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt")],
                      dtype=np.float64)
        c = tf.seeds["cov"][:, i].astype(np.float64)
        ids, sc, npaths = _exhaustive_best(st, c, trk, p)
        if ids is None or npaths > 4096:
            continue
        checked += 1
        assert list(r["tracklet_id"][:, i]) == ids, i
        total = r["chi2"][i] + p["p_miss"] * r["n_miss"][i]
        assert total == pytest.approx(sc, rel=1e-12, abs=1e-9)
    assert checked >= 30


def test_greedy_n1_takes_best_chi2_each_layer():
    """N = 1: each layer keeps the single best extension (Sec. 3 with
    N_candidates = 1), so each chosen tracklet has the lowest chi2 among the
    accepted candidates of its layer."""
    tf = make_workload("tiny", seed=5)
    p = tf.params
    r = O.follow(tf.seeds, tf.tracklets, p, seed_index=np.arange(150))
    for i in range(150):
        st = np.array([tf.seeds[k][i] for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt")],
                      dtype=np.float64)
        c = tf.seeds["cov"][:, i].astype(np.float64)
        phi = st[0] + math.atan2(st[2], st[1])
        sec = int(math.floor((phi % (2 * math.pi)) / math.radians(20.0))) % 18
        ok, st, c, _ = O.rotate(st, c, math.radians(20.0 * (sec + 0.5)), p["bz"])
        if not ok or r["status"][i] != 0:
            continue
        nmiss = 0
        for l in range(6):
            ok, st, c, sec, ch = O.to_layer(st, c, sec, l, p)
            assert ok
            cid, cchi = O.candidates(st, c, l, ch, tf.tracklets, p) if ch >= 0 else ([], [])
            got = r["tracklet_id"][l, i]
            if len(cid):
                assert got == cid[int(np.argmin(cchi))]
                j = got
                _, st, c = O.update(st, c, l, (tf.tracklets["y"][j], tf.tracklets["z"][j],
                                               tf.tracklets["vyy"][j], tf.tracklets["vzz"][j],
                                               tf.tracklets["vyz"][j]))
            else:
                assert got == -1
                nmiss += 1
        assert nmiss == r["n_miss"][i]


def test_road_boundary_at_n_sigma():
    """Sec. 3: tracklets inside a search road from the covariance.  Shift the
    true layer-0 tracklet by 2.9 and 3.1 of its residual's y sigma (3-sigma
    road; chi2 stays below the cut of 15 either way, so only the road
    decides)."""
    p = G.default_params(material_on=0, n_sigma_road=3.0, chi2_cut=15.0)
    tf = make_timeframe(150, seed=19, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p)
    ok = np.nonzero(tf.truth_ids[:, 0] >= 0)[0][:60]
    sig = []
    for i in ok:
        st = np.array([tf.seeds[k][i] for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt")], dtype=np.float64)
        c = tf.seeds["cov"][:, i].astype(np.float64)
        phi = st[0] + math.atan2(st[2], st[1])
        sec = int(math.floor((phi % (2 * math.pi)) / math.radians(20.0))) % 18
        _, st, c, _ = O.rotate(st, c, math.radians(20.0 * (sec + 0.5)), p["bz"])
        _, st, c, sec, ch = O.to_layer(st, c, sec, 0, p)
        tt = G.pad_tilt_tan(0)
        syy = c[0] - 2 * tt * c[1] + tt * tt * c[2] + tf.tracklets["vyy"][tf.truth_ids[i, 0]]
        sig.append(math.sqrt(syy))
    j = tf.truth_ids[ok, 0]
    for k, expect in ((2.9, True), (3.1, False)):
        t2 = {kk: v.copy() for kk, v in tf.tracklets.items()}
        t2["y"][j] = (t2["y"][j].astype(np.float64) + k * np.array(sig)).astype(np.float32)
        r = O.follow(tf.seeds, t2, p, seed_index=ok)
        got = r["tracklet_id"][0] == j
        assert got.mean() > 0.95 if expect else got.mean() < 0.05


# ---------------------------------------------------------------- association
def test_association_never_crosses_interactions():
    """Sec. 4: only tracklets of the track's own interaction are considered."""
    p = G.default_params()
    tf = make_timeframe(2000, seed=23, noise=0.5, params=p, n_interactions=40)
    r = O.follow(tf.seeds, tf.tracklets, p)
    ids = r["tracklet_id"]
    ok = ids >= 0
    seed_trig = np.broadcast_to(tf.seeds["trigger"], ids.shape)
    assert ok.sum() > 1000
    assert np.all(tf.tracklets["trigger"][ids[ok]] == seed_trig[ok])


def test_association_with_one_interaction_changes_nothing():
    tf = make_workload("tiny", seed=24)
    a = O.follow(tf.seeds, tf.tracklets, tf.params)
    s2 = dict(tf.seeds, trigger=np.full(tf.n_seeds, 3, np.int32))
    t2 = dict(tf.tracklets, trigger=np.full(tf.n_tracklets, 3, np.int32))
    b = O.follow(s2, t2, tf.params)
    untagged = dict(tf.tracklets, trigger=np.full(tf.n_tracklets, -1, np.int32))
    c = O.follow(s2, untagged, tf.params)  # tracklets without an id stay candidates for every seed
    for k in ("tracklet_id", "par", "cov", "chi2", "status"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])


def test_association_improves_purity_at_timeframe_density():
    """With Run-3 time frames of many collisions (Sec. 3.1), restricting the
    candidates to the track's interaction removes the other collisions' fakes."""
    base = make_workload("timeframe", seed=2, n_seeds=40_000)
    p = base.params
    assoc = make_timeframe(40_000, seed=2, noise=0.3, params=p, name="timeframe", n_interactions=600)
    sel = np.arange(0, 40_000, 8)
    ep0 = efficiency_purity(O.follow(base.seeds, base.tracklets, p, seed_index=sel)["tracklet_id"],
                            base.truth_ids[sel])
    ep1 = efficiency_purity(O.follow(assoc.seeds, assoc.tracklets, p, seed_index=sel)["tracklet_id"],
                            assoc.truth_ids[sel])
    assert ep1["purity"] > ep0["purity"] + 0.02
    assert ep1["efficiency_reachable"] >= ep0["efficiency_reachable"] - 0.005
