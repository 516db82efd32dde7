"""Parity of the CUDA residual collection and distortion solve (trd_residuals,
trd_voxel_solve, through the C ABI) with the FP64 oracle.

Tolerances, from the arithmetic: each refit reaches a row in one FP32
transport of up to 215 cm from its last rotation point, which moves y by up
to ~100 cm (y carried as a double-float, but the step dx * tan(phi) is one
FP32 product: a few 1e-6 relative) and z by up to 250 cm (a float whose
spacing there is 1.5e-5 cm, plus the arc's rounding), so per cluster
|d dy| <= 1e-4 max(|dy|, sigma_y) + 4e-5 cm and |d dz| <= 1e-4 max(|dz|,
sigma_z) + 1e-4 cm (sigma the combination's error; measured maxima 2.9e-5
and 6.5e-5 cm); the slopes t, u within 1e-5 relative + 1e-6.  Which
clusters contribute and which voxel each falls in are decided identically
(the voxel in FP32 on both sides), so voxel counts are equal exactly; every
other voxel sum within 1e-4 of the sum of its terms' magnitudes plus the
per-cluster floor times the count.
"""
import numpy as np
import pytest

from oracle import oracle as O
from parity import to_numpy
from synth import tpc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCALE = float(1 << 24)


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


def _dev(w):
    from paper_2003_03174_b300 import trd
    return trd.to_device(w.its), trd.to_device(w.trd), trd.to_device(w.clusters)


def _gpu(ctx, w, cluster_res=True):
    its, tr, cl = _dev(w)
    out = ctx.residuals(its, tr, cl, w.bz, cluster_res=cluster_res)
    torch.cuda.synchronize()
    if cluster_res:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy(), None


def _check_clusters(g_res, o):
    ok_o = o["vox"] >= 0
    ok_g = ~np.isnan(g_res[0])
    # presence decided by the same rules; a track near the |snp| limit may differ
    diff = ok_o != ok_g
    near = (o["slack"] < 1e-3)[None, :].repeat(ok_o.shape[0], 0)
    assert not (diff & ~near).any(), int((diff & ~near).sum())
    both = ok_o & ok_g & ~near
    sy, sz = np.sqrt(o["var"][0][both]), np.sqrt(o["var"][1][both])
    e = {}
    for k, (sig, floor) in enumerate(((sy, 4e-5), (sz, 1e-4))):
        ov, gv = o["res"][k][both].astype(np.float64), g_res[k][both].astype(np.float64)
        err = np.abs(gv - ov)
        tol = 1e-4 * np.maximum(np.abs(ov), sig) + floor
        assert np.all(err <= tol), (k, float((err / tol).max()))
        e[k] = float(err.max())
    for k in (2, 3):
        ov, gv = o["res"][k][both].astype(np.float64), g_res[k][both].astype(np.float64)
        assert np.all(np.abs(gv - ov) <= 1e-5 * np.abs(ov) + 1e-6), k
    return both.sum(), e


def _check_sums(g_sums, o):
    n_g, n_o = g_sums[:, 0], o["sums"][:, 0]
    np.testing.assert_array_equal(n_g, n_o.astype(np.int64))
    n = n_o
    G = g_sums[:, 1:].astype(np.float64) / SCALE
    Ov, A = o["sums"][:, 1:], o["abs_sums"][:, 1:]
    # per-term floors: t, u, t^2, u^2 (relative only); dy, dz and products
    floor = np.array([0, 0, 0, 0, 4e-5, 1e-4, 4e-5 * 3, 1e-4 * 3, 4e-5 * 10, 1e-4 * 10])
    tol = 1e-4 * A + (floor[None, :] + 1.0 / SCALE) * n[:, None]
    bad = np.abs(G - Ov) > tol
    assert not bad.any(), np.argwhere(bad)[:5]


def test_cluster_residuals_and_voxel_sums_match_oracle(ctx):
    w = tpc.make_residual_workload(3001, seed=41)
    g_sums, g_res = _gpu(ctx, w)
    o = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    n, _ = _check_clusters(g_res, o)
    assert n > 300_000
    _check_sums(g_sums, o)


@pytest.mark.parametrize("kw", [dict(distorted=False, smear=0.0, refit_smear=False),
                                dict(uniform=(-0.8, 0.5, 0.3), bz=-0.5),
                                dict(fail_frac=0.4, eff=0.5)])
def test_residual_parity_variants(ctx, kw):
    w = tpc.make_residual_workload(1500, seed=42, **kw)
    g_sums, g_res = _gpu(ctx, w)
    o = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    _check_clusters(g_res, o)
    _check_sums(g_sums, o)


def test_non_finite_clusters_and_failed_refits_contribute_nothing(ctx):
    w = tpc.make_residual_workload(800, seed=43, fail_frac=0.2)
    w.clusters["y"][5, :100] = np.nan
    w.clusters["z"][90, 100:200] = np.inf
    w.clusters["sector"][30, 200:300] = 40  # not a sector
    g_sums, g_res = _gpu(ctx, w)
    o = O.residuals(w.its, w.trd, w.clusters, w.bz, with_clusters=True)
    _check_clusters(g_res, o)
    _check_sums(g_sums, o)
    assert np.isnan(g_res[0][5, :100]).all() and np.isnan(g_res[0][90, 100:200]).all()
    bad = (w.its["status"] != 0) | (w.trd["status"] != 0)
    assert np.isnan(g_res[0][:, bad]).all()


def test_sums_accumulate_across_calls(ctx):
    from paper_2003_03174_b300 import trd
    a = tpc.make_residual_workload(700, seed=44)
    b = tpc.make_residual_workload(900, seed=45)
    ia, ta, ca = _dev(a)
    ib, tb, cb = _dev(b)
    s = ctx.residuals(ia, ta, ca, a.bz)
    ctx.residuals(ib, tb, cb, b.bz, sums=s)
    torch.cuda.synchronize()
    o = O.residuals(a.its, a.trd, a.clusters, a.bz)
    O.residuals(b.its, b.trd, b.clusters, b.bz, sums=o["sums"])
    np.testing.assert_array_equal(s[:, 0].cpu().numpy(), o["sums"][:, 0].astype(np.int64))
    # integer sums: the order of accumulation cannot change them
    s2 = ctx.residuals(ib, tb, cb, b.bz)
    ctx.residuals(ia, ta, ca, a.bz, sums=s2)
    torch.cuda.synchronize()
    assert torch.equal(s, s2)
    assert trd.N_VOXELS == O.N_VOXELS


def _quantized_sums(rng, n_vox):
    """Voxel sums built in numpy from random FP32 terms, quantized the way the
    library stores them; returned as int64 (for the library) and float64
    (the same values, for the oracle)."""
    S = np.zeros((n_vox, 11), np.int64)
    for v in range(n_vox):
        m = int(rng.integers(0, 300))
        t = rng.normal(0.1, 0.3, m).astype(np.float32)
        u = rng.normal(-0.2, 0.5, m).astype(np.float32)
        D = rng.normal(0, 1, 3)
        dy = (D[1] - D[0] * t + rng.normal(0, 0.1, m)).astype(np.float32)
        dz = (D[2] - D[0] * u + rng.normal(0, 0.1, m)).astype(np.float32)
        terms = [t, u, t * t, u * u, dy, dz, t * dy, u * dz, dy * dy, dz * dz]
        S[v, 0] = m
        for k, x in enumerate(terms):
            S[v, k + 1] = np.rint(x.astype(np.float32).astype(np.float64) * SCALE).astype(np.int64).sum()
    Sf = S.astype(np.float64)
    Sf[:, 1:] /= SCALE
    return S, Sf


def test_voxel_solve_matches_oracle(ctx):
    from paper_2003_03174_b300 import trd
    rng = np.random.default_rng(46)
    n_vox = 3000
    S, Sf = _quantized_sums(rng, n_vox)
    full = np.zeros((trd.N_VOXELS, 11), np.int64)
    idx = rng.choice(trd.N_VOXELS, n_vox, replace=False)
    full[idx] = S
    m = ctx.voxel_solve(torch.from_numpy(full).cuda(), min_count=20)
    torch.cuda.synchronize()
    g = m.cpu().numpy()[idx]
    o = O.voxel_solve(Sf, 20)
    np.testing.assert_array_equal(np.isnan(g[:, 0]), np.isnan(o[:, 0]))
    np.testing.assert_array_equal(g[:, 3], o[:, 3])
    ok = ~np.isnan(o[:, 0])
    assert ok.sum() > 2000
    for k in range(3):
        assert np.all(np.abs(g[ok, k] - o[ok, k]) <= 1e-5 * np.maximum(np.abs(o[ok, k]), 0.1)), k
    for k in (4, 5):
        assert np.all(np.abs(g[ok, k] - o[ok, k]) <= 1e-4 * o[ok, k] + 1e-6), k
    # empty voxels: n = 0 and NaN
    rest = np.setdiff1d(np.arange(trd.N_VOXELS), idx)[:1000]
    assert np.all(m.cpu().numpy()[rest, 3] == 0) and np.isnan(m.cpu().numpy()[rest, 0]).all()


def test_full_map_at_scale(ctx):
    """The map workload (450,000 tracks, ~61 M clusters): voxel counts
    identical, every voxel sum and every solved voxel within tolerance of
    the oracle's."""
    w = tpc.make_map_workload(450_000, seed=0)
    g_sums, _ = _gpu(ctx, w, cluster_res=False)
    o = O.residuals(w.its, w.trd, w.clusters, w.bz)
    _check_sums(g_sums, o)
    m = ctx.voxel_solve(torch.from_numpy(g_sums).cuda(), min_count=50).cpu().numpy()
    om = O.voxel_solve(o["sums"], 50)
    ok = ~np.isnan(om[:, 0]) & ~np.isnan(m[:, 0])
    assert ok.sum() > 0.5 * (om[:, 3] >= 50).sum()
    # the solve amplifies the sums' tolerance by the voxel's conditioning:
    # compare against the statistical error of each voxel instead
    for k in (1, 2):
        assert np.percentile(np.abs(m[ok, k] - om[ok, k]), 99) < 1e-3, k
    assert np.percentile(np.abs(m[ok, 0] - om[ok, 0]), 99) < 1e-2
