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


def test_served_timeline_summary_measures_copies_under_other_requests_kernels():
    # three requests: (start, inputs in, kernels done, results out), ms
    marks = [(0, 1, 5, 6), (1, 2, 7, 8), (5, 6, 9, 10)]
    tl = bench.timeline_summary(marks)
    # copies: A [0,1] none, [5,6] under B; B [1,2] under A, [7,8] under C;
    # C [5,6] under B, [9,10] none -> 4 of 6 ms
    assert abs(tl["copy_time_under_other_kernels"] - 4 / 6) < 1e-12
    assert abs(tl["kernels_busy_share_of_span"] - 0.8) < 1e-12  # kernels cover [1, 9] of [0, 10]
    assert tl["inputs_ms_p50"] == 1 and tl["kernels_ms_p50"] == 4 and tl["results_ms_p50"] == 1
    # one request alone: its copies never run under another's kernels
    assert bench.timeline_summary([(0, 1, 3, 4)])["copy_time_under_other_kernels"] == 0.0
    assert bench._covered(0, 10, [(2, 4), (3, 6), (8, 12), (-5, -1)]) == 6
