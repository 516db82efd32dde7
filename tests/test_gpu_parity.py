"""Parity of the CUDA follower (through the C ABI) with the FP64 oracle.

Element-by-element comparison on the same seeded inputs at sizes the oracle
finishes in seconds, every seed of the full timeframe (and every 20th seed of
the calibration pass) in the launch configuration the benchmark times, and
the edge cases (empty and invalid inputs, ragged tails, every hypothesis count
and mode).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from parity import compare, to_numpy
from synth import make_timeframe, make_workload, efficiency_purity
from synth import timeframe as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


def run_gpu(ctx, tf, params=None, lanes=0, bin_width=0.0, seeds=None, tracklets=None):
    from paper_2003_03174_b300 import trd
    s = trd.to_device(tf.seeds if seeds is None else seeds)
    t = trd.to_device(tf.tracklets if tracklets is None else tracklets)
    idx = ctx.index_build(t, bin_width)
    r = ctx.follow(s, idx, params or tf.params, lanes_per_track=lanes)
    torch.cuda.synchronize()
    return to_numpy(r), idx


def test_tiny_parity(ctx):
    tf = make_workload("tiny")
    g, _ = run_gpu(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, tf.params)
    rep = compare(g, o)
    assert rep["same_path"] >= 0.98 * tf.n_seeds


def test_medium_parity_spans_tiles_and_ragged_tail(ctx):
    tf = make_workload("timeframe", seed=5, n_seeds=20_000 + 37)
    g, _ = run_gpu(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, tf.params)
    compare(g, o)


@pytest.mark.parametrize("n_hyp", [2, 3, 6, 8])
def test_multi_hypothesis_parity(ctx, n_hyp):
    p = G.default_params(n_hyp=n_hyp, n_sigma_road=5.0)
    tf = make_timeframe(3000 + n_hyp, seed=20 + n_hyp, noise=0.5, params=p)
    g, _ = run_gpu(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, p)
    compare(g, o)


def test_calibration_distribution_parity(ctx):
    tf = make_workload("calibration", seed=3, n_seeds=4000)
    g, _ = run_gpu(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, tf.params)
    compare(g, o)


@pytest.mark.parametrize("over", [dict(res_mode=1), dict(material_on=0), dict(bz=-0.5),
                                  dict(bz=0.0), dict(max_missing=0), dict(max_missing=6),
                                  dict(chi2_cut=4.0, p_miss=6.0)])
def test_mode_parity(ctx, over):
    p = G.default_params(**over)
    tf = make_timeframe(3000, seed=41, noise=0.3, bz=p["bz"], params=p)
    g, _ = run_gpu(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, p)
    compare(g, o)


def test_lanes_per_track_do_not_change_results(ctx):
    tf = make_workload("timeframe", seed=8, n_seeds=5000)
    base, _ = run_gpu(ctx, tf, lanes=1)
    for lanes in (2, 4, 8):
        g, _ = run_gpu(ctx, tf, lanes=lanes)
        for k in base:
            np.testing.assert_array_equal(g[k], base[k], err_msg=f"{k} lanes={lanes}")


def test_bin_width_does_not_change_results(ctx):
    tf = make_workload("timeframe", seed=9, n_seeds=5000)
    base, _ = run_gpu(ctx, tf)
    for w in (0.5, 8.0, 132.0):
        g, _ = run_gpu(ctx, tf, bin_width=w)
        for k in base:
            np.testing.assert_array_equal(g[k], base[k], err_msg=f"{k} w={w}")


def test_results_are_deterministic(ctx):
    tf = make_workload("timeframe", seed=10, n_seeds=8000)
    a, _ = run_gpu(ctx, tf)
    b, _ = run_gpu(ctx, tf)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _bucket_reference(trk, w):
    """Numpy counting sort with the index's FP32 bucketing expressions."""
    f32 = np.float32
    ch = trk["chamber"].astype(np.int64)
    stack = (ch // 6) % 5
    zlo = (f32(-360.0) + f32(144.0) * stack.astype(f32)).astype(f32)
    row = np.floor((trk["z"] - zlo).astype(f32) * f32(0.125)).astype(f32)
    row = np.clip(row, 0, 17).astype(np.int64)
    inv_w = f32(1.0) / f32(w)
    nb = int(math.ceil(np.float32(132.0) / np.float32(w)))
    yb = np.clip(np.floor((trk["y"] + f32(66.0)).astype(f32) * inv_w), 0, nb - 1).astype(np.int64)
    return (ch * 18 + row) * nb + yb, nb


@pytest.mark.parametrize("w", [2.0, 0.7, 0.25, 0.05])
def test_index_buckets_are_exact(ctx, w):
    # 0.25 and 0.05 cm make more scan tiles than the apply kernel adds up
    # itself (1,253 and 6,265), so their tile sums go through the one-block
    # scan (two passes of it at 0.05 cm)
    tf = make_workload("timeframe", seed=11, n_seeds=30_000)
    from paper_2003_03174_b300 import trd
    idx = ctx.index_build(trd.to_device(tf.tracklets), w)
    off, ids = idx.copy_out()
    bk, nb = _bucket_reference(tf.tracklets, w)
    counts = np.bincount(bk, minlength=540 * 18 * nb)
    ref_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    np.testing.assert_array_equal(off, ref_off)
    # every bucket holds exactly its tracklets (order inside a bucket is free)
    assert np.array_equal(np.sort(ids), np.arange(tf.n_tracklets))
    got_bucket = np.repeat(np.arange(counts.shape[0]), counts)
    np.testing.assert_array_equal(bk[ids], got_bucket)


def test_empty_inputs(ctx):
    from paper_2003_03174_b300 import trd
    tf = make_workload("tiny", seed=12)
    empty_t = {k: v[:0] for k, v in tf.tracklets.items()}
    g, idx = run_gpu(ctx, tf, tracklets=empty_t)
    assert idx.info()["n_indexed"] == 0
    o = O.follow(tf.seeds, empty_t, tf.params)
    compare(g, o)
    assert np.all(g["n_trk"] == 0)
    # no seeds at all: nothing launched, nothing written
    s0 = trd.to_device({k: v[..., :0] if k != "cov" else v[:, :0] for k, v in tf.seeds.items()})
    r = ctx.follow(s0, idx, tf.params)
    torch.cuda.synchronize()
    assert r["chi2"].numel() == 0


def test_invalid_tracklets_are_left_out(ctx):
    tf = make_workload("tiny", seed=13)
    m = 40
    bad = {k: v[:m].copy() for k, v in tf.tracklets.items()}
    bad["chamber"][:10] = 540
    bad["chamber"][10:20] = -3
    bad["y"][20:30] = np.nan
    bad["vyy"][30:40] = -1.0
    trk = {k: np.concatenate([tf.tracklets[k], bad[k]]) for k in tf.tracklets}
    g, idx = run_gpu(ctx, tf, tracklets=trk)
    info = idx.info()
    assert info["n_rejected"] == m and info["n_indexed"] == tf.n_tracklets
    o = O.follow(tf.seeds, tf.tracklets, tf.params)
    compare(g, o)


def test_invalid_seeds(ctx):
    tf = make_workload("tiny", seed=14)
    s = {k: v.copy() for k, v in tf.seeds.items()}
    s["snp"][:5] = 0.97
    s["cov"][0, 5:10] = -1.0
    s["cov"][1, 10:15] = 1.0  # |c10| > sqrt(c00 c11): not positive definite
    g, _ = run_gpu(ctx, tf, seeds=s)
    assert np.all(g["status"][:15] == O.STATUS_SEED_INVALID)
    assert np.all(g["tracklet_id"][:, :15] == -1)
    o = O.follow(s, tf.tracklets, tf.params)
    compare(g, o)


def test_event_rotated_by_one_sector(ctx):
    tf = make_workload("tiny", seed=15)
    s2 = dict(tf.seeds)
    s2["alpha"] = (tf.seeds["alpha"].astype(np.float64) + math.radians(20.0)).astype(np.float32)
    t2 = dict(tf.tracklets)
    t2["chamber"] = ((tf.tracklets["chamber"] + 30) % 540).astype(np.int32)
    g, _ = run_gpu(ctx, tf, seeds=s2, tracklets=t2)
    o = O.follow(s2, t2, tf.params)
    compare(g, o)


def _bench_step_results(ctx, tf):
    """The benchmark's step on a workload: the autotuned launch shape and bin
    width, one CUDA-graph replay of index rebuild + follow (the library's
    single-timeframe batch)."""
    from paper_2003_03174_b300 import autotune, trd
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    tuned = autotune.tune(ctx, s, t, tf.params, cache=None, reps=3)
    shape = {k: tuned[k] for k in ("lanes_per_track", "block_threads", "min_blocks_per_sm")}
    res = trd.alloc_results(tf.n_seeds)
    batch = ctx.batch_create(s, t, [0, tf.n_seeds], [0, tf.n_tracklets], tf.params, res,
                             y_bin_width=tuned["y_bin_width"], **shape)
    stream = torch.cuda.Stream()
    for _ in range(2):  # a replay over the previous replay's buffers too
        batch.run(stream)
    torch.cuda.synchronize()
    out = to_numpy(res)
    batch.free()
    return out


def test_full_timeframe_parity_every_seed(ctx):
    """200k seeds, ~1M tracklets, N = 1, 3 sigma road: every seed of the
    benchmark's timed step against the oracle following all of them."""
    tf = make_workload("timeframe")
    g = _bench_step_results(ctx, tf)
    o = O.follow(tf.seeds, tf.tracklets, tf.params)
    rep = compare(g, o)
    assert rep["same_path"] >= 0.995 * tf.n_seeds
    # Sec. 3.1: purity ~1 in pp, falling to ~0.9 for low-momentum tracks at
    # Pb-Pb density; this timeframe is Pb-Pb-like (1M tracklets, 30% noise)
    ep = efficiency_purity(g["tracklet_id"], tf.truth_ids)
    assert ep["efficiency_reachable"] > 0.95 and ep["purity"] > 0.85


def test_full_calibration_parity(ctx):
    """450k seeds with the coherent y distortion, 5 sigma road, N = 6, in the
    benchmark's step; the oracle follows 22,500 of them (every 20th) against
    all tracklets."""
    tf = make_workload("calibration")
    g = _bench_step_results(ctx, tf)
    sel = np.arange(0, tf.n_seeds, 20)
    o = O.follow(tf.seeds, tf.tracklets, tf.params, seed_index=sel)
    rep = compare(g, o, sel=sel)
    assert rep["same_path"] >= 0.99 * sel.size


@pytest.mark.parametrize("n_hyp,shapes", [(6, ((8, 3), (32, 3), (32, 4), (8, 4), (8, 5), (8, 6))),
                                          (3, ((4, 3), (4, 4), (4, 5), (4, 6), (8, 3), (8, 5), (32, 4))),
                                          (2, ((2, 3), (2, 4), (2, 5), (2, 6), (4, 6)))])
def test_lane_groups_do_not_change_multi_hypothesis_results(ctx, n_hyp, shapes):
    """N hypotheses with 2, 4 or 8 lanes per seed (lists sized to N or to the
    group), and with a whole warp per seed, scanning by shuffled roads (3 or 4
    blocks per SM) or by the road table with the lanes' states parked (groups
    of 8, or 5 and 6 blocks per SM): the same candidates, arithmetic and
    order, so identical results."""
    from paper_2003_03174_b300 import trd
    tf = make_workload("calibration", seed=9, n_seeds=4000)
    params = dict(tf.params, n_hyp=n_hyp)
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t)
    outs = []
    for lanes, mb in shapes:
        outs.append(to_numpy(ctx.follow(s, idx, params, lanes_per_track=lanes, min_blocks_per_sm=mb)))
    torch.cuda.synchronize()
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)


@pytest.mark.parametrize("n_hyp", [1, 3])
def test_association_parity(ctx, n_hyp):
    """Per-interaction association (Sec. 4) on the GPU against the oracle."""
    p = G.default_params(n_hyp=n_hyp)
    tf = make_timeframe(20_000, seed=31 + n_hyp, noise=0.3, params=p, n_interactions=100)
    g, _ = run_gpu(ctx, tf, params=p)
    o = O.follow(tf.seeds, tf.tracklets, p)
    compare(g, o)
    ids = g["tracklet_id"]
    ok = ids >= 0
    assert np.all(tf.tracklets["trigger"][ids[ok]] == np.broadcast_to(tf.seeds["trigger"], ids.shape)[ok])


@pytest.mark.parametrize("n_hyp", [1, 3])
def test_seed_order_does_not_change_results(ctx, n_hyp):
    """The follower takes seeds in order of |q/pT|; a seed's result does not
    depend on where it sits in the input: permuted seeds give the permuted
    results, bit for bit."""
    p = G.default_params(n_hyp=n_hyp)
    tf = make_timeframe(6000, seed=41 + n_hyp, noise=0.3, params=p)
    base, _ = run_gpu(ctx, tf, params=p)
    perm = np.random.default_rng(7).permutation(tf.n_seeds)
    s = {k: np.ascontiguousarray(v[..., perm]) for k, v in tf.seeds.items()}
    g, _ = run_gpu(ctx, tf, params=p, seeds=s)
    for k in base:
        np.testing.assert_array_equal(g[k], base[k][..., perm], err_msg=k)


def test_momentum_order_edge_cases(ctx):
    """Seeds at the ends of the |q/pT| order against the oracle: NaN q/pT
    (first bin; the transport fails), |q/pT| = 40 c/GeV (first bin; the
    helix cannot reach the layers), q/pT = 0 (last bin; a straight line)."""
    tf = make_workload("tiny", seed=16)
    s = {k: v.copy() for k, v in tf.seeds.items()}
    s["q2pt"][:4] = np.nan
    s["q2pt"][4:8] = 0.0
    s["q2pt"][8:12] = 40.0
    s["q2pt"][12:16] = -40.0
    g, _ = run_gpu(ctx, tf, seeds=s)
    o = O.follow(s, tf.tracklets, tf.params)
    np.testing.assert_array_equal(g["status"][:16], o["status"][:16])
    np.testing.assert_array_equal(g["tracklet_id"][:, :16], o["tracklet_id"][:, :16])
    assert np.all(g["status"][:4] == O.STATUS_PROP_FAIL) and np.all(g["status"][8:16] == O.STATUS_PROP_FAIL)
    fin = np.arange(4, tf.n_seeds)
    compare(g, {k: v[..., fin] for k, v in o.items()}, sel=fin)


@pytest.mark.parametrize("n", [1, 2049])
def test_one_momentum_bin(ctx, n):
    """Every seed with the same q/pT: one bin holds them all (the key kernel's
    atomics all on one counter), a single seed, and a ragged second block."""
    tf = make_timeframe(n, seed=17 + n, noise=0.3)
    s = {k: v.copy() for k, v in tf.seeds.items()}
    s["q2pt"][:] = np.float32(0.8)
    g, _ = run_gpu(ctx, tf, seeds=s)
    o = O.follow(s, tf.tracklets, tf.params)
    compare(g, o)


@pytest.mark.parametrize("n", [31, 32, 33, 95])
def test_ragged_warps_of_seeds(ctx, n):
    """One hypothesis: a warp carries 32 consecutive sorted seeds through the
    layers together; seed counts around a warp's size leave the last warp
    partly empty."""
    tf = make_timeframe(n, seed=40 + n, noise=0.3)
    g, _ = run_gpu(ctx, tf)
    compare(g, O.follow(tf.seeds, tf.tracklets, tf.params))


def test_a_warp_of_seeds_that_all_end_early(ctx):
    """40 seeds with |q/pT| = 40 c/GeV (the helix cannot reach the layers)
    sort into the first momentum bin, so one warp holds only seeds that end
    at the first layer while the other warps follow ordinary seeds; seeds
    that run out of their missing-layer budget early (no tracklets at all in
    their chambers) end at layer 2 beside seeds that reach layer 5."""
    tf = make_timeframe(600, seed=44, noise=0.3)
    s = {k: v.copy() for k, v in tf.seeds.items()}
    s["q2pt"][:40] = np.where(np.arange(40) % 2 == 0, 40.0, -40.0).astype(np.float32)
    t = {k: v.copy() for k, v in tf.tracklets.items()}
    # no tracklets in the sectors of seeds 100..299's frames: most of them
    # spend their two missing layers and stop
    sec = (((s["alpha"][100:300].astype(np.float64) + math.pi) % (2 * math.pi)) / (2 * math.pi / 18)).astype(int)
    drop = np.isin(t["chamber"] // 30, np.unique(sec)[:3])
    t = {k: v[~drop] for k, v in t.items()}
    g, _ = run_gpu(ctx, tf, seeds=s, tracklets=t)
    o = O.follow(s, t, tf.params)
    assert np.all(g["status"][:40] == O.STATUS_PROP_FAIL)
    assert (o["n_miss"] == 2).sum() > 20 and (o["status"] != 0).sum() > 40
    compare(g, o)


def test_launch_shapes_do_not_change_one_hypothesis_results(ctx):
    """Block sizes and register budgets of the layer-synchronous follower
    (and so the number of warps resident per SM) change nothing."""
    tf = make_workload("timeframe", seed=45, n_seeds=6000)
    from paper_2003_03174_b300 import trd
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t)
    outs = [to_numpy(ctx.follow(s, idx, tf.params, lanes_per_track=1, block_threads=b, min_blocks_per_sm=m))
            for b, m in ((64, 4), (64, 6), (128, 5), (128, 8))]
    torch.cuda.synchronize()
    for o in outs[1:]:
        for k in outs[0]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)


def test_resident_index_rebuilds_stay_exact(ctx):
    """A resident index rebuilt with different tracklet sets in turn (the
    bucket counters return to zero after every build): each build's offsets
    and bucket contents equal the counting-sort reference of its own set."""
    from paper_2003_03174_b300 import trd
    a = make_workload("timeframe", seed=12, n_seeds=30_000).tracklets
    b = make_workload("timeframe", seed=13, n_seeds=20_000).tracklets
    w = 2.0
    idx = ctx.index_create(max(len(a["chamber"]), len(b["chamber"])), w)
    for trk in (a, b, a, b):
        idx.rebuild(trd.to_device(trk))
        torch.cuda.synchronize()
        off, ids = idx.copy_out()
        bk, nb = _bucket_reference(trk, w)
        counts = np.bincount(bk, minlength=540 * 18 * nb)
        np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
        n = len(trk["chamber"])
        assert np.array_equal(np.sort(ids[:n]), np.arange(n))
        np.testing.assert_array_equal(bk[ids[:n]], np.repeat(np.arange(counts.shape[0]), counts))


@pytest.mark.parametrize("n_hyp,lanes", [(1, 1), (3, 4)])
def test_timed_follow_gives_the_same_results_and_times_the_kernel_alone(ctx, n_hyp, lanes):
    # trd_follow_timed: the results of trd_follow_tuned, and its events bracket
    # the follower kernel inside the whole call
    from paper_2003_03174_b300 import trd
    tf = make_workload("timeframe", seed=17, n_seeds=20_000)
    params = dict(tf.params, n_hyp=n_hyp)
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t, 1.0)
    plain = to_numpy(ctx.follow(s, idx, params, lanes_per_track=lanes))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record()
    ev[0].record()
    timed = ctx.follow(s, idx, params, lanes_per_track=lanes, kernel_events=(ev[1], ev[2]))
    ev[3].record()
    torch.cuda.synchronize()
    for k, v in to_numpy(timed).items():
        np.testing.assert_array_equal(v, plain[k], err_msg=k)
    kernel, call = ev[1].elapsed_time(ev[2]), ev[0].elapsed_time(ev[3])
    assert 0 < kernel < call
    # no seeds: both events recorded at once
    none = {k: v[..., :0] for k, v in tf.seeds.items()}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    e1.record()
    ctx.follow(trd.to_device(none), idx, params, lanes_per_track=lanes, kernel_events=(e0, e1))
    torch.cuda.synchronize()
    assert 0 <= e0.elapsed_time(e1) < 0.05
    idx.free()
