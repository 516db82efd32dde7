"""Per-parameter error of the CUDA follower against the FP64 oracle.

  python tests/parity_report.py [--workload calibration] [--stride 1500]

Runs the full workload on the GPU (the benchmark's launch) and the oracle on
every `stride`-th seed, and prints one JSON line: for each track parameter the
maximum and 99th percentile of |gpu - oracle| / max(|oracle|, sigma), the
chi2 error, the covariance error, and the near-tie exemptions.
"""
import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="calibration")
    ap.add_argument("--stride", type=int, default=1500)
    ap.add_argument("--association", type=int, default=0, help="interactions per timeframe")
    a = ap.parse_args()
    import torch
    from oracle import oracle as O
    from paper_2003_03174_b300 import trd
    from parity import compare, to_numpy
    from synth import make_workload, efficiency_purity
    tf = make_workload(a.workload, n_interactions=a.association)
    ctx = trd.Context(0)
    idx = ctx.index_build(trd.to_device(tf.tracklets))
    g = to_numpy(ctx.follow(trd.to_device(tf.seeds), idx, tf.params))
    torch.cuda.synchronize()
    sel = np.arange(0, tf.n_seeds, a.stride)
    o = O.follow(tf.seeds, tf.tracklets, tf.params, seed_index=sel)
    rep = compare(g, o, sel=sel)
    names = ["y", "z", "snp", "tgl", "q2pt"]
    out = {"workload": a.workload, "interactions": a.association, "seeds": tf.n_seeds,
           "tracklets": tf.n_tracklets,
           "params": {k: tf.params[k] for k in ("n_hyp", "n_sigma_road", "chi2_cut", "max_missing")},
           "sample": len(sel), "same_path": rep["same_path"], "exempt_near_ties": rep["exempt"],
           "param_rel_err": {nm: {"max": rep["max_par_rel_each"][i], "p99": rep["p99_par_rel"][i]}
                             for i, nm in enumerate(names)},
           "chi2_abs_err": {"max": rep["max_chi2_abs"], "p99": rep["p99_chi2_abs"]},
           "cov_rel_err_max": rep["max_cov_rel"],
           "efficiency_purity": efficiency_purity(g["tracklet_id"], tf.truth_ids)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
