"""Batches of timeframes in one graph replay: every timeframe's result must be
the same as when it is followed alone (the per-seed arithmetic is identical),
and must agree with the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from parity import compare, to_numpy
from synth.timeframe import concat, make_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

COUNTS = [3000, 0, 500, 8000, 1, 2000, 12_000]


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


def _plain(ctx, tf):
    from paper_2003_03174_b300 import trd
    idx = ctx.index_build(trd.to_device(tf.tracklets))
    r = ctx.follow(trd.to_device(tf.seeds), idx, tf.params)
    torch.cuda.synchronize()
    return to_numpy(r)


def _slice(res, a, b):
    return {k: v[..., a:b] for k, v in res.items()}


def _run_batch(ctx, tfs, **shape):
    from paper_2003_03174_b300 import trd
    seeds, trk, so, to = concat(tfs)
    s, t = trd.to_device(seeds), trd.to_device(trk)
    res = trd.alloc_results(int(so[-1]))
    b = ctx.batch_create(s, t, so, to, tfs[0].params, res, **shape)
    b.run()
    torch.cuda.synchronize()
    return b, s, t, res, so


def test_batch_equals_each_timeframe_alone(ctx):
    tfs = make_batch(COUNTS, seed=3)
    b, s, t, res, so = _run_batch(ctx, tfs)
    got = to_numpy(res)
    for k, tf in enumerate(tfs):
        alone = _plain(ctx, tf)
        part = _slice(got, so[k], so[k + 1])
        for key in alone:
            np.testing.assert_array_equal(part[key], alone[key], err_msg=f"tf {k} {key}")
    b.free()


def test_batch_matches_oracle(ctx):
    tfs = make_batch(COUNTS, seed=4)
    b, s, t, res, so = _run_batch(ctx, tfs)
    got = to_numpy(res)
    for k in (0, 3, 6):
        tf = tfs[k]
        o = O.follow(tf.seeds, tf.tracklets, tf.params)
        compare(_slice(got, so[k], so[k + 1]), o)
    b.free()


def test_graph_replay_sees_refilled_inputs(ctx):
    """Refill the bound seed buffers in place (same sizes, new draw) and replay:
    each timeframe's result must equal the plain path on the new seeds."""
    from paper_2003_03174_b300 import trd
    first = make_batch(COUNTS, seed=5)
    b, s, t, res, so = _run_batch(ctx, first)
    a1 = to_numpy(res)
    second = make_batch(COUNTS, seed=6)
    seeds2 = concat(second)[0]
    for k, v in trd.to_device(seeds2).items():
        s[k].copy_(v)
    b.run()
    torch.cuda.synchronize()
    a2 = to_numpy(res)
    assert not np.array_equal(a1["par"], a2["par"])
    for k, (tf_old, tf_new) in enumerate(zip(first, second)):
        idx = ctx.index_build(trd.to_device(tf_old.tracklets))
        alone = to_numpy(ctx.follow(trd.to_device(tf_new.seeds), idx, tf_old.params))
        part = _slice(a2, so[k], so[k + 1])
        for key in alone:
            np.testing.assert_array_equal(part[key], alone[key], err_msg=f"tf {k} {key}")
    b.run()  # replaying again gives the same answer
    torch.cuda.synchronize()
    a3 = to_numpy(res)
    for key in a2:
        np.testing.assert_array_equal(a2[key], a3[key])
    b.free()


def test_batch_launch_shapes_agree(ctx):
    tfs = make_batch([4000, 700, 2500], seed=7)
    base = to_numpy(_run_batch(ctx, tfs)[3])
    for shape in (dict(lanes_per_track=8, min_blocks_per_sm=3), dict(block_threads=64)):
        got = to_numpy(_run_batch(ctx, tfs, **shape)[3])
        for key in base:
            np.testing.assert_array_equal(got[key], base[key], err_msg=f"{shape} {key}")


def test_batch_rejects_bad_offsets(ctx):
    from paper_2003_03174_b300 import trd
    tfs = make_batch([300, 200], seed=8)
    seeds, trk, so, to = concat(tfs)
    s, t = trd.to_device(seeds), trd.to_device(trk)
    res = trd.alloc_results(int(so[-1]))
    for bad_so, bad_to in ((so + 1, to), (so, to[::-1].copy()), (so[:-1], to)):
        with pytest.raises(trd.TrdError):
            ctx.batch_create(s, t, bad_so, bad_to if len(bad_to) == len(bad_so) else to[:len(bad_so)],
                             tfs[0].params, res)


def test_batch_with_association_equals_alone(ctx):
    from synth.timeframe import default_params, make_timeframe
    p = default_params(n_hyp=3)
    tfs = [make_timeframe(n, seed=40 + k, noise=0.3, params=p, n_interactions=30) for k, n in
           enumerate([2000, 0, 700, 3500])]
    b, s, t, res, so = _run_batch(ctx, tfs)
    got = to_numpy(res)
    for k, tf in enumerate(tfs):
        alone = _plain(ctx, tf)
        part = _slice(got, so[k], so[k + 1])
        for key in alone:
            np.testing.assert_array_equal(part[key], alone[key], err_msg=f"tf {k} {key}")
    b.free()
