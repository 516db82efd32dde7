"""Pins of the oracle's residual collection and distortion extraction
(Sec. 2, steps 4 and 5) against facts that do not come from the oracle.

* Voxel assignment: hand-placed clusters land in the voxel their position
  names (side, sector, row, y/x bin, |z|/x bin), and a brute-force FP32
  recount of random clusters agrees.
* Undistorted clusters on the truth helix, exact refits: every residual
  vanishes (the transports and the combination add no bias).
* Distorted clusters, exact refits: each residual equals the first-order
  effect of the generator's own field, dy = Dy - Dx tan(phi), dz = Dz - Dx
  tan(lambda)/cos(phi), up to second order in Dx.
* Honest smeared refits, exact clusters: the combined (y, z) deviates from
  the truth by unit-normal pulls of the combined covariance.
* The per-voxel solve equals numpy's least squares on the raw clusters and
  recovers noiseless linear data exactly; on a densely filled sector the
  extracted map reproduces the generator's field.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth import timeframe as G
from synth import tpc

TAN10 = math.tan(math.radians(10.0))


def _voxel(side, sector, row, iy, iz):
    return (((side * 18 + sector) * 152 + row) * 15 + iy) * 5 + iz


def test_voxel_of_hand_placed_clusters():
    xr = tpc.row_x()
    # centre of a row, z just above 0: middle y bin, first z bin, side A
    assert O.voxel_of(0.0, 0.5, 3, 10) == _voxel(0, 3, 10, 7, 0)
    # z < 0 is side C
    assert O.voxel_of(0.0, -0.5, 3, 10) == _voxel(1, 3, 10, 7, 0)
    # y at the low sector edge -> bin 0; beyond the high edge -> clamped to 14
    x = float(xr[50])
    assert O.voxel_of(-x * TAN10 * 0.999, 10.0, 0, 50) == _voxel(0, 0, 50, 0, 0)
    assert O.voxel_of(x * TAN10 * 1.2, 10.0, 0, 50) == _voxel(0, 0, 50, 14, 0)
    # |z|/x = 0.5 -> bin 2 of 5; |z|/x = 3 -> clamped to bin 4
    assert O.voxel_of(0.0, -0.5 * x, 17, 50) == _voxel(1, 17, 50, 7, 2)
    assert O.voxel_of(0.0, 3.0 * x, 17, 50) == _voxel(0, 17, 50, 7, 4)
    # y/x one bin width above the low edge, and the last row and sector
    w = 2 * TAN10 / 15
    assert O.voxel_of((-TAN10 + 1.5 * w) * float(xr[151]), 1.0, 17, 151) == _voxel(0, 17, 151, 1, 0)
    assert O.voxel_of(0.0, 0.0, 18, 0) == -1 and O.voxel_of(0.0, 0.0, 0, 152) == -1


def test_voxel_of_matches_fp32_brute_force():
    rng = np.random.default_rng(3)
    n = 20000
    row = rng.integers(0, 152, n)
    xr = tpc.row_x()[row]
    y = (rng.uniform(-1.1, 1.1, n) * TAN10 * xr).astype(np.float32)
    z = rng.uniform(-260, 260, n).astype(np.float32)
    sec = rng.integers(0, 18, n)
    f = np.float32
    T = f(0.17632698070846498)
    ys = f(15) / (f(2) * T)
    iy = np.floor(((y / xr).astype(f) + T).astype(f) * ys).astype(np.int64).clip(0, 14)
    iz = np.floor((np.abs(z) / xr).astype(f) * f(5)).astype(np.int64).clip(0, 4)
    want = _voxel((z < 0).astype(np.int64), sec, row, iy, iz)
    got = np.array([O.voxel_of(float(a), float(b), int(c), int(d)) for a, b, c, d in zip(y, z, sec, row)])
    np.testing.assert_array_equal(got, want)


def test_no_distortion_exact_refits_give_zero_residuals():
    w = tpc.make_residual_workload(1500, seed=11, distorted=False, smear=0.0, refit_smear=False, fail_frac=0.0)
    r = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    ok = r["vox"] >= 0
    assert ok.sum() > 150_000
    # inputs are FP32: a half-ulp of sin(phi) (3e-8) carried over 215 cm at
    # cos(phi) = 0.5 moves y by 5e-5 cm; a modelling error gives 1e-3 or more
    assert np.abs(r["res"][0][ok]).max() < 2e-4
    assert np.abs(r["res"][1][ok]).max() < 2e-4
    assert np.abs(r["res"][0][ok]).mean() < 2e-5
    # every present cluster of a usable track was used
    np.testing.assert_array_equal(ok, w.clusters["sector"] >= 0)


def test_residuals_follow_the_injected_field():
    w = tpc.make_residual_workload(1500, seed=12, distorted=True, smear=0.0, refit_smear=False, fail_frac=0.0)
    r = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    ok = r["vox"] >= 0
    rows = np.nonzero(ok)
    dx, dy, dz = (w.applied[k][rows].astype(np.float64) for k in ("dx", "dy", "dz"))
    t, u = r["res"][2][rows], r["res"][3][rows]
    ey = r["res"][0][rows] - (dy - dx * t)
    ez = r["res"][1][rows] - (dz - dx * u)
    # second order in dx (<= 1.8 cm): half dx^2 times the track's change of
    # slope, d(tan phi)/dx = rho / cos^3(phi), up to ~0.03 cm
    assert np.abs(ey).max() < 0.03, np.abs(ey).max()
    assert np.abs(ez).max() < 0.03, np.abs(ez).max()
    assert np.abs(ey).mean() < 2e-3 and np.abs(ez).mean() < 2e-3
    assert np.abs(dy - dx * t).max() > 0.5  # the field is not negligible


def test_combined_estimate_has_unit_pulls():
    w = tpc.make_residual_workload(3000, seed=13, distorted=False, smear=0.0, refit_smear=True, fail_frac=0.0)
    r = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    ok = r["vox"] >= 0
    # the clusters are the truth, so -residual is the combination's error;
    # over all rows, and over the outer rows alone, where the TRD refit
    # weighs as much as the ITS one
    outer = ok.copy()
    outer[:120] = False
    for sel in (ok, outer):
        for k in range(2):
            pull = r["res"][k][sel] / np.sqrt(r["var"][k][sel])
            assert abs(pull.mean()) < 0.05, (k, pull.mean())
            assert 0.93 < pull.std() < 1.07, (k, pull.std())
    # and tracks whose refits failed contribute nothing
    w2 = tpc.make_residual_workload(500, seed=14, fail_frac=0.3)
    r2 = O.residuals(w2.its, w2.trd, w2.clusters, w2.bz, with_clusters=True)
    bad = (w2.its["status"] != 0) | (w2.trd["status"] != 0)
    assert bad.any()
    assert np.all(r2["vox"][:, bad] == -1)


def _sums_from(t, u, dy, dz):
    return np.array([len(t), t.sum(), u.sum(), (t * t).sum(), (u * u).sum(), dy.sum(), dz.sum(),
                     (t * dy).sum(), (u * dz).sum(), (dy * dy).sum(), (dz * dz).sum()])


def test_voxel_solve_equals_least_squares():
    rng = np.random.default_rng(21)
    S, want = [], []
    for _ in range(50):
        m = rng.integers(5, 400)
        t, u = rng.normal(0.1, 0.4, m), rng.normal(-0.2, 0.6, m)
        D = rng.normal(0, 1, 3)
        dy = D[1] - D[0] * t + rng.normal(0, 0.1, m)
        dz = D[2] - D[0] * u + rng.normal(0, 0.1, m)
        A = np.zeros((2 * m, 3))
        A[:m, 0], A[:m, 1] = -t, 1.0
        A[m:, 0], A[m:, 2] = -u, 1.0
        want.append(np.linalg.lstsq(A, np.concatenate([dy, dz]), rcond=None)[0])
        S.append(_sums_from(t, u, dy, dz))
    out = O.voxel_solve(np.array(S), 1)
    np.testing.assert_allclose(out[:, :3], np.array(want), rtol=1e-9, atol=1e-10)
    # noiseless linear data: exact; too few clusters or no angular spread: undetermined
    t = np.linspace(-0.5, 0.5, 9)
    u = np.linspace(0.3, -0.2, 9)
    out = O.voxel_solve(np.array([_sums_from(t, u, 0.7 + 0.4 * t, -0.2 + 0.4 * u),
                                  _sums_from(t[:3], u[:3], t[:3], u[:3]),
                                  _sums_from(np.zeros(9), np.zeros(9), np.ones(9), np.ones(9))]), 5)
    np.testing.assert_allclose(out[0, :3], [-0.4, 0.7, -0.2], atol=1e-12)
    assert np.isnan(out[1, :3]).all() and out[1, 3] == 3
    assert np.isnan(out[2, 0]) and out[2, 3] == 9


def test_map_recovers_a_uniform_displacement():
    """All tracks in one sector and a narrow eta band, every cluster moved by
    the same (dx, dy, dz) and smeared by 0.1 cm, exact refits: the linear
    model of the voxel solve is then exact up to second order and the only
    noise is the clusters', so each filled voxel's (Dx, Dy, Dz) must scatter
    about the displacement with unit pulls of the least-squares errors (the
    inverse normal matrix times 0.1^2).  With smeared refits the reference's
    own slope and position errors, correlated within a track, bias Dx over
    the narrow angular spread of a voxel (an errors-in-variables effect of
    the method, not tested here)."""
    D = (-0.8, 0.5, 0.3)
    w = tpc.make_residual_workload(6000, seed=15, distorted=True, smear=0.1, refit_smear=False, fail_frac=0.0,
                                   phi_range=(math.radians(62.0), math.radians(78.0)), eta_range=(0.2, 0.3),
                                   uniform=D)
    r = O.residuals(w.its, w.trd, w.clusters, w.bz)
    m = O.voxel_solve(r["sums"], 100)
    good = np.nonzero(~np.isnan(m[:, 0]))[0]
    assert good.size > 2000
    S = r["sums"][good]
    side = (good // (18 * 152 * 75)).astype(np.float64)
    want = np.stack([np.full(good.size, D[0]), np.full(good.size, D[1]), D[2] * (1.0 - 2.0 * side)])
    for j, v in enumerate(good):
        n, St, Su, Stt, Suu = S[j, :5]
        M = np.array([[Stt + Suu, -St, -Su], [-St, n, 0.0], [-Su, 0.0, n]])
        sig = 0.1 * np.sqrt(np.diag(np.linalg.inv(M)))
        if j == 0:
            sigs = np.zeros((3, good.size))
        sigs[:, j] = sig
    pull = (m[good, :3].T - want) / sigs
    for k in range(3):
        assert abs(pull[k].mean()) < 0.15, (k, pull[k].mean())
        assert 0.85 < pull[k].std() < 1.2, (k, pull[k].std())
    assert m[good, 3].min() >= 100
