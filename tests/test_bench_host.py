"""Host-side parts of bench.py that run without a GPU: the oracle baselines
it reports beside the GPU numbers (all cores and one thread, the refit's,
the residual collection's)."""
import numpy as np

import bench
from synth import make_workload
from synth import tpc


def test_follower_cpu_baseline_reports_all_cores_one_thread_and_refit():
    tf = make_workload("tiny", seed=2)
    cb = bench.cpu_baseline(tf, tf.n_seeds)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["value"] > 0
    assert cb["sample"].startswith(f"all {tf.n_seeds} seeds")
    assert cb["seeds"] == tf.n_seeds and 0 < cb["matched"] <= tf.n_seeds
    one = cb["one_thread"]
    assert one["cores"] == 1 and one["kind"] == "oracle" and one["value"] > 0
    rf = cb["refit"]
    assert rf["unit"] == "refitted tracks/s" and rf["value"] > 0 and "repeats" in rf["sample"]


def test_residual_cpu_baseline_counts_the_sample_clusters():
    w = tpc.make_map_workload(2_000, seed=3, chunk=1_000, workers=1)
    cb = bench.residual_cpu_baseline(w, 500)
    assert cb["unit"] == "clusters/s" and cb["value"] > 0 and cb["kind"] == "oracle"
    assert cb["sample"].startswith("first 500 of 2000 tracks")
    n_cl = int(cb["sample"].split("(")[1].split()[0])
    sec = np.asarray(w.clusters["sector"])[:, :500]
    assert 0 < n_cl <= int(((sec >= 0) & (sec < 18)).sum())
