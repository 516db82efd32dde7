"""Parity of the CUDA TRD-only refit (trd_refit, through the C ABI) with the
FP64 oracle's refit.

Both sides refit the same input: the oracle follower's results stored as the
FP32 arrays the library reads, against the same tracklets.  At full size the
chain is checked end to end: the CUDA follower then the CUDA refit against
the oracle follower then the oracle refit, on a sample of tracks whose
follower paths agree.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from parity import compare_refit, to_numpy
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


def _f32_tracks(r):
    """Oracle follower results as the FP32/int32 arrays of the library's layout."""
    out = {k: np.ascontiguousarray(r[k].astype(np.float32)) for k in ("alpha", "x", "par", "cov", "chi2")}
    for k in ("n_trk", "n_miss", "status", "tracklet_id"):
        out[k] = np.ascontiguousarray(r[k].astype(np.int32))
    return out


def _gpu_refit(ctx, tracks, tracklets, params, cov_scale=100.0):
    from paper_2003_03174_b300 import trd
    out = ctx.refit(trd.to_device(tracks), trd.to_device(tracklets), params, cov_scale)
    torch.cuda.synchronize()
    return to_numpy(out)


def _parity(ctx, tf, params=None, cov_scale=100.0):
    p = params or tf.params
    tracks = _f32_tracks(O.follow(tf.seeds, tf.tracklets, p))
    g = _gpu_refit(ctx, tracks, tf.tracklets, p, cov_scale)
    o = O.refit(tracks, tf.tracklets, p, cov_scale=cov_scale)
    return compare_refit(g, o), tracks, g, o


def test_refit_parity_tiny(ctx):
    tf = make_workload("tiny")
    rep, tracks, g, o = _parity(ctx, tf)
    assert rep["refitted"] > 0.5 * tf.n_seeds
    # skipped tracks carry their input state and a zero covariance
    sk = o["status"] == 8
    assert sk.any()
    np.testing.assert_array_equal(g["par"][:, sk], tracks["par"][:, sk])
    assert not g["cov"][:, sk].any()


# cov_scale up to 1e3 (prior errors x31.6): the first update against a prior
# R times wider than the tracklet error cancels ~log10(R) digits in
# (I - K H) ~ V / (C + V); at 1e4 the FP32 refit reaches 2e-4 relative (tgl)
# and 2e-3 in chi2, outside the parity tolerance.
@pytest.mark.parametrize("material,res_mode,bz,cov_scale", [
    (1, 0, 0.5, 100.0), (0, 0, 0.5, 100.0), (1, 1, 0.5, 100.0), (1, 0, -0.5, 100.0), (1, 0, 0.5, 1e3),
    (0, 1, -0.5, 1.0)])
def test_refit_parity_modes(ctx, material, res_mode, bz, cov_scale):
    p = G.default_params(bz=bz, material_on=material, res_mode=res_mode)
    tf = make_timeframe(3001, seed=61, noise=0.3, bz=bz, params=p)
    rep, *_ = _parity(ctx, tf, p, cov_scale)
    assert rep["refitted"] > 1500


def test_refit_parity_spans_tiles_and_ragged_tail(ctx):
    tf = make_workload("timeframe", seed=62, n_seeds=20_000 + 37)
    rep, *_ = _parity(ctx, tf)
    assert rep["refitted"] > 10_000


def test_refit_parity_after_multi_hypothesis_follow(ctx):
    p = G.default_params(n_hyp=6, n_sigma_road=5.0)
    tf = make_timeframe(2500, seed=63, noise=0.5, params=p)
    _parity(ctx, tf, p)


def test_refit_chain_at_full_size(ctx):
    """Timeframe workload (200k seeds): the CUDA follower + refit against the
    oracle follower + refit on a sample of 2,000 tracks; where the follower
    paths agree the refits must agree within the same tolerances."""
    from paper_2003_03174_b300 import trd
    tf = make_workload("timeframe")
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t)
    res = ctx.follow(s, idx, tf.params)
    rf = ctx.refit(res, t, tf.params)
    torch.cuda.synchronize()
    gf, g = to_numpy(res), to_numpy(rf)
    sel = np.arange(0, tf.n_seeds, 100)
    of = O.follow(tf.seeds, tf.tracklets, tf.params, seed_index=sel)
    same = (gf["tracklet_id"][:, sel] == of["tracklet_id"]).all(0) & (gf["status"][sel] == of["status"])
    assert same.mean() > 0.99
    o = O.refit(_f32_tracks(of), tf.tracklets, tf.params)
    keep = np.nonzero(same)[0]
    o_keep = {k: v[..., keep] for k, v in o.items()}
    rep = compare_refit(g, o_keep, sel=sel[keep])
    assert rep["refitted"] > 1000
    # the whole launch: every matched track was refitted or skipped for a reason
    matched = gf["n_trk"] >= 2
    assert np.mean(g["status"][matched] == 0) > 0.99
    assert np.all(g["status"][~matched] == 8)


def test_refit_edge_cases(ctx):
    from paper_2003_03174_b300 import trd
    tf = make_workload("tiny", seed=3)
    tracks = _f32_tracks(O.follow(tf.seeds, tf.tracklets, tf.params))
    # n = 0: nothing to do, no launch
    empty = {k: v[..., :0].copy() for k, v in tracks.items()}
    out = ctx.refit(trd.to_device(empty), trd.to_device(tf.tracklets), tf.params)
    assert out["alpha"].numel() == 0
    # ids past the tracklet arrays, negative ids other than -1, invalid seeds, chambers out of range
    bad = {k: v.copy() for k, v in tracks.items()}
    m = np.nonzero(tracks["n_trk"] >= 2)[0]
    bad["tracklet_id"][0, m[0]] = tf.n_tracklets + 5
    bad["tracklet_id"][0, m[1]] = -7
    bad["status"][m[2]] = 4
    trk = {k: v.copy() for k, v in tf.tracklets.items()}
    l3 = int(np.nonzero(tracks["tracklet_id"][:, m[3]] >= 0)[0][0])
    trk["chamber"][tracks["tracklet_id"][l3, m[3]]] = 777
    g = _gpu_refit(ctx, bad, trk, tf.params)
    o = O.refit(bad, trk, tf.params)
    compare_refit(g, o)
    assert g["status"][m[0]] == 8 and g["status"][m[2]] == 8 and g["status"][m[3]] == 8
    # every track unmatched: all skipped
    none = {k: v.copy() for k, v in tracks.items()}
    none["tracklet_id"][:] = -1
    g = _gpu_refit(ctx, none, tf.tracklets, tf.params)
    assert np.all(g["status"] == 8) and np.all(g["n_upd"] == 0)


def test_refit_rejects_bad_arguments(ctx):
    from paper_2003_03174_b300 import trd
    tf = make_workload("tiny", seed=4)
    tracks = trd.to_device(_f32_tracks(O.follow(tf.seeds, tf.tracklets, tf.params)))
    t = trd.to_device(tf.tracklets)
    for cs in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(trd.TrdError) as e:
            ctx.refit(tracks, t, tf.params, cov_scale=cs)
        assert e.value.code == trd.TRD_EINVAL
    L = trd.lib()
    rs, ts, ps = trd.results_struct(tracks), trd.tracklets_struct(t), trd.params_struct(tf.params)
    out = trd.alloc_refit(tf.n_seeds)
    os_ = trd.RefitOut(*[trd._ptr(out[k]) for k in ("alpha", "x", "par", "cov", "chi2", "n_upd", "status")])
    assert L.trd_refit(ctx.handle, C.byref(rs), -1, C.byref(ts), C.byref(ps), 100.0, C.byref(os_), None) \
        == trd.TRD_EINVAL
    assert L.trd_refit(None, C.byref(rs), 5, C.byref(ts), C.byref(ps), 100.0, C.byref(os_), None) == trd.TRD_EINVAL
    os_.status = None
    assert L.trd_refit(ctx.handle, C.byref(rs), 5, C.byref(ts), C.byref(ps), 100.0, C.byref(os_), None) \
        == trd.TRD_EINVAL
