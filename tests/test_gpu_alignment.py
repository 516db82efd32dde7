"""Parity of the CUDA follower's misalignment and field-map path
(trd_follow_aligned, per-tracklet radii in the index) with the FP64 oracle,
through the C ABI, with the follower's tolerances: per-tracklet radii and
chamber radii (N = 1 and the group scan), a non-uniform Bz map, both
together; the refit at the tracklet radii; radii carried through the serving
path; and nominal radii against the aligned kernels."""
import numpy as np
import pytest

from oracle import oracle as O
from parity import compare, compare_refit, to_numpy
from synth import make_timeframe, make_workload
from synth import timeframe as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


def _field_map():
    rs, zs = np.linspace(250.0, 420.0, 18), np.linspace(-400.0, 400.0, 41)
    R, Z = np.meshgrid(rs, zs)
    bz = (0.5 * (1.0 - 0.15 * (Z / 400.0) ** 2) * (1.0 + 0.05 * (R - 300.0) / 100.0)).astype(np.float32)
    return dict(bz=bz, r_min=250.0, r_max=420.0, z_min=-400.0, z_max=400.0)


def _gpu(ctx, tf, params, chamber_x=None, field=None, lanes=0):
    from paper_2003_03174_b300 import trd
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t)
    dcx = torch.from_numpy(chamber_x).cuda() if chamber_x is not None else None
    dfield = dict(field, bz=torch.from_numpy(field["bz"]).cuda()) if field is not None else None
    if dcx is None and dfield is None:
        r = ctx.follow(s, idx, params, lanes_per_track=lanes)
    else:
        r = ctx.follow(s, idx, params, lanes_per_track=lanes, chamber_x=dcx, field=dfield)
    torch.cuda.synchronize()
    return to_numpy(r)


@pytest.mark.parametrize("n_hyp", [1, 3])
def test_misaligned_parity(ctx, n_hyp):
    p = G.default_params(n_hyp=n_hyp)
    tf = make_timeframe(4000, seed=71 + n_hyp, noise=0.3, params=p, misalign=0.5, x_jitter=0.1)
    g = _gpu(ctx, tf, p, chamber_x=tf.chamber_x)
    o = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x)
    rep = compare(g, o)
    assert rep["same_path"] >= 0.98 * tf.n_seeds


def test_misaligned_noiseless_truth_on_the_gpu(ctx):
    p = G.default_params(material_on=0)
    tf = make_timeframe(2000, seed=73, noise=0.0, eff=1.0, smear=False, snap_z=False, params=p,
                        misalign=0.5, x_jitter=0.1)
    g = _gpu(ctx, tf, p, chamber_x=tf.chamber_x)
    full = (tf.truth_ids >= 0).all(1)
    np.testing.assert_array_equal(g["tracklet_id"].T[full], tf.truth_ids[full])
    assert g["chi2"][full].max() < 0.05


@pytest.mark.parametrize("misaligned", [False, True])
def test_field_map_parity(ctx, misaligned):
    p = G.default_params()
    kw = dict(misalign=0.5, x_jitter=0.1) if misaligned else {}
    tf = make_timeframe(4000, seed=75, noise=0.3, params=p, **kw)
    fm = _field_map()
    g = _gpu(ctx, tf, p, chamber_x=tf.chamber_x, field=fm)
    o = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x, field=fm)
    compare(g, o)


def test_nominal_radii_match_the_default_kernels(ctx):
    tf = make_workload("tiny", seed=76)
    nominal = np.array([300.0 + 12.6 * l for l in range(6)], np.float32)
    trk = dict(tf.tracklets, x=nominal[tf.tracklets["chamber"] % 6])
    base = _gpu(ctx, tf, tf.params)
    tf2 = type(tf)(name=tf.name, seeds=tf.seeds, tracklets=trk, params=tf.params, truth_ids=tf.truth_ids)
    ext = _gpu(ctx, tf2, tf.params, chamber_x=np.tile(nominal, 90))
    np.testing.assert_array_equal(base["tracklet_id"], ext["tracklet_id"])
    np.testing.assert_allclose(ext["par"], base["par"], rtol=2e-5, atol=3e-4)


def test_refit_at_tracklet_radii_parity(ctx):
    from paper_2003_03174_b300 import trd
    p = G.default_params()
    tf = make_timeframe(3000, seed=77, noise=0.3, params=p, misalign=0.5, x_jitter=0.1)
    of = O.follow(tf.seeds, tf.tracklets, p, chamber_x=tf.chamber_x)
    tracks = {k: np.ascontiguousarray(of[k].astype(np.float32)) for k in ("alpha", "x", "par", "cov", "chi2")}
    tracks.update({k: np.ascontiguousarray(of[k].astype(np.int32))
                   for k in ("n_trk", "n_miss", "status", "tracklet_id")})
    g = to_numpy(ctx.refit(trd.to_device(tracks), trd.to_device(tf.tracklets), p))
    torch.cuda.synchronize()
    o = O.refit(tracks, tf.tracklets, p)
    rep = compare_refit(g, o)
    assert rep["refitted"] > 1500


def test_served_misaligned_equals_plain(ctx):
    """The server copies the radii with the tracklets; without an alignment
    table its results equal trd_follow on the same index (radii only)."""
    from paper_2003_03174_b300 import trd
    p = G.default_params()
    tf = make_timeframe(3000, seed=78, noise=0.3, params=p, misalign=0.5, x_jitter=0.1)
    srv = trd.Server(ctx, p, max_slots=2)
    out = trd.host_results(tf.n_seeds)
    assert srv.wait(srv.submit(tf.seeds, tf.tracklets, out), 60_000) is not None
    srv.close()
    plain = _gpu(ctx, tf, p)
    for k in plain:
        np.testing.assert_array_equal(out[k], plain[k], err_msg=k)
    o = O.follow(tf.seeds, tf.tracklets, p)
    compare(plain, o)


def test_full_aligned_timeframe_parity_every_seed(ctx):
    """The benchmark's misaligned timeframe (200k seeds, chambers shifted by up
    to 0.5 cm, tracklets by 0.1 cm more, the Bz(r, z) map): every seed against
    the oracle (it holds a stack-boundary near tie that moves one track's state
    without changing its tracklets)."""
    from synth.timeframe import field_map
    tf = make_workload("timeframe", misalign=0.5, x_jitter=0.1)
    fm = field_map(tf.params["bz"])
    g = _gpu(ctx, tf, tf.params, chamber_x=tf.chamber_x, field=fm, lanes=1)
    o = O.follow(tf.seeds, tf.tracklets, tf.params, chamber_x=tf.chamber_x, field=fm)
    rep = compare(g, o)
    assert rep["same_path"] >= 0.995 * tf.n_seeds
