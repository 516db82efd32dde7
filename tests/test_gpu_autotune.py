"""The autotuner's search runs every launch shape on the GPU, checks each one
gives bit-identical results, re-times its best few as whole steps (index
rebuild + follower call, L2 flushed) and returns the fastest of those."""
import pytest

from synth import make_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name,n", [("timeframe", 20_000), ("calibration", 3000)])
def test_autotune_picks_a_shape_from_its_table(name, n, tmp_path):
    from paper_2003_03174_b300 import autotune, trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tf = make_workload(name, n_seeds=n)
    ctx = trd.Context(0)
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(ctx, trd.to_device(tf.seeds), trd.to_device(tf.tracklets), tf.params,
                      bin_widths=(2.0, 4.0), reps=3, cache=cache)
    top = sorted(r["table"], key=lambda row: row["ms"])[:4]
    assert all("step_ms" in row for row in top)
    assert r["step_ms"] == min(row["step_ms"] for row in top)
    assert any(row["ms"] == r["ms"] and row["min_blocks_per_sm"] == r["min_blocks_per_sm"] for row in top)
    assert r["lanes_per_track"] >= tf.params["n_hyp"]
    again = autotune.tune(ctx, trd.to_device(tf.seeds), trd.to_device(tf.tracklets), tf.params,
                          cache=cache)
    assert again["key"] == r["key"] and again["ms"] == r["ms"]  # served from the cache
