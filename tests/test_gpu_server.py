"""The serving loop: each request's result is the same alone and in the mix;
admission follows the device-memory budget; every failure is reported on the
host without any device-side wait."""
import numpy as np
import pytest

from parity import to_numpy
from synth.timeframe import make_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [6000, 0, 1500, 20_000, 1, 9000, 3000, 15_000]


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


@pytest.fixture(scope="module")
def tfs():
    return make_batch(SIZES, seed=21)


def _alone(ctx, tf):
    from paper_2003_03174_b300 import trd
    idx = ctx.index_build(trd.to_device(tf.tracklets))
    r = ctx.follow(trd.to_device(tf.seeds), idx, tf.params)
    torch.cuda.synchronize()
    return to_numpy(r)


@pytest.mark.parametrize("slots,pinned", [(3, False), (4, True)])
def test_served_results_equal_alone_and_requests_overlap(ctx, tfs, slots, pinned):
    from paper_2003_03174_b300 import trd
    srv = trd.Server(ctx, tfs[0].params, max_slots=slots)
    if pinned:
        inputs = [({k: torch.from_numpy(v).pin_memory() for k, v in tf.seeds.items()},
                   {k: torch.from_numpy(v).pin_memory() for k, v in tf.tracklets.items()}) for tf in tfs]
    else:
        inputs = [(tf.seeds, tf.tracklets) for tf in tfs]
    outs = [trd.host_results(tf.n_seeds, pinned=pinned) for tf in tfs]
    tickets = [srv.submit(s, t, o) for (s, t), o in zip(inputs, outs)]
    timings = [srv.wait(t, 60_000) for t in tickets]
    assert all(tm is not None for tm in timings)
    for tf, o, tm in zip(tfs, outs, timings):
        alone = _alone(ctx, tf)
        got = {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in o.items()}
        for k in alone:
            np.testing.assert_array_equal(got[k], alone[k], err_msg=k)
        assert tm["submit_s"] <= tm["admit_s"] <= tm["done_s"]
        assert 0 <= tm["slot"] < slots
        # the device-clock stage marks: copies in, kernels, copies out in order,
        # spanning the request's GPU time (event resolution ~0.5 us)
        assert 0 <= tm["start_ms"] <= tm["inputs_ms"] <= tm["kernels_ms"] <= tm["results_ms"]
        assert abs((tm["results_ms"] - tm["start_ms"]) - tm["gpu_ms"]) < 0.01 + 1e-3 * tm["gpu_ms"]
    # continuous batching: some requests were in flight at the same time
    # (whether their device work overlapped depends on their sizes and the
    # host's timing; the served bench line measures that from these marks)
    iv = sorted((tm["admit_s"], tm["done_s"]) for tm in timings)
    assert any(b[0] < a[1] for a, b in zip(iv, iv[1:]))
    # requests on one slot run one after another on the device clock
    for sl in range(slots):
        dv = sorted((tm["start_ms"], tm["results_ms"]) for tm in timings if tm["slot"] == sl)
        assert all(b[0] >= a[1] - 1e-3 for a, b in zip(dv, dv[1:]))
    st = srv.stats()
    assert st["queued"] == 0 and st["in_flight"] == 0
    srv.close()


def test_budget_admits_one_request_at_a_time(ctx, tfs):
    from paper_2003_03174_b300 import trd
    big = max(tfs, key=lambda t: t.n_seeds)
    # the server charges a request's inputs and results plus its stream's index:
    # leave room for the index and one and a half requests, never for two
    # (with the follower's scratch: 136 B per seed + 528 B)
    io = 220 * big.n_seeds + 36 * big.n_tracklets + 7 * 256 + 136 * big.n_seeds + 528 + 256
    index = 40 * big.n_tracklets + 8 * 540 * 18 * 66 + 4096
    one = index + io + io // 2
    srv = trd.Server(ctx, big.params, max_slots=4, mem_budget_bytes=one)
    outs = [trd.host_results(big.n_seeds) for _ in range(3)]
    tickets = [srv.submit(big.seeds, big.tracklets, o) for o in outs]
    tms = [srv.wait(t, 60_000) for t in tickets]
    iv = sorted((tm["admit_s"], tm["done_s"]) for tm in tms)
    assert all(b[0] >= a[1] for a, b in zip(iv, iv[1:])), iv  # never two in flight
    alone = _alone(ctx, big)
    for o in outs:
        np.testing.assert_array_equal(o["tracklet_id"], alone["tracklet_id"])
    # a request larger than the whole budget is refused at submission
    tiny = trd.Server(ctx, big.params, mem_budget_bytes=1 << 20)
    with pytest.raises(trd.TrdError) as e:
        tiny.submit(big.seeds, big.tracklets, trd.host_results(big.n_seeds))
    assert e.value.code == trd.TRD_ENOMEM
    tiny.close()
    srv.close()


def test_queue_full_timeouts_and_unknown_tickets(ctx, tfs):
    from paper_2003_03174_b300 import trd
    big = max(tfs, key=lambda t: t.n_seeds)
    srv = trd.Server(ctx, big.params, max_slots=1, max_queue=1)
    outs, tickets, refused = [], [], 0
    for _ in range(12):
        o = trd.host_results(big.n_seeds)
        try:
            tickets.append(srv.submit(big.seeds, big.tracklets, o))
            outs.append(o)
        except trd.TrdError as e:
            assert e.code == trd.TRD_EAGAIN
            refused += 1
    assert refused > 0  # one slot, one queue place: later submissions bounce
    assert srv.wait(tickets[-1], 0) is None  # a zero-length bounded wait runs out
    for t in tickets:
        assert srv.wait(t, 60_000) is not None
    with pytest.raises(trd.TrdError) as e:
        srv.poll(tickets[0])  # already released
    assert e.value.code == trd.TRD_EINVAL
    with pytest.raises(trd.TrdError):
        srv.poll(987654321)
    srv.close()


def test_destroy_finishes_pending_work(ctx, tfs):
    from paper_2003_03174_b300 import trd
    srv = trd.Server(ctx, tfs[0].params, max_slots=2)
    outs = [trd.host_results(tf.n_seeds) for tf in tfs]
    for tf, o in zip(tfs, outs):
        srv.submit(tf.seeds, tf.tracklets, o)
    srv.close()  # returns once queued and running requests are done
    for tf, o in zip(tfs, outs):
        if tf.n_seeds:
            np.testing.assert_array_equal(o["tracklet_id"], _alone(ctx, tf)["tracklet_id"])


def test_served_association_equals_alone(ctx):
    from paper_2003_03174_b300 import trd
    from synth.timeframe import default_params, make_timeframe
    p = default_params(n_hyp=3)
    tfs = [make_timeframe(n, seed=50 + k, noise=0.3, params=p, n_interactions=25) for k, n in
           enumerate([3000, 800, 5000])]
    srv = trd.Server(ctx, p, max_slots=2)
    outs = [trd.host_results(tf.n_seeds) for tf in tfs]
    tickets = [srv.submit(tf.seeds, tf.tracklets, o) for tf, o in zip(tfs, outs)]
    for t in tickets:
        assert srv.wait(t, 60_000) is not None
    for tf, o in zip(tfs, outs):
        alone = _alone(ctx, tf)
        for k in alone:
            np.testing.assert_array_equal(o[k], alone[k], err_msg=k)
    srv.close()
