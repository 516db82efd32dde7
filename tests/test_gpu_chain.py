"""The calibration chain of Sec. 2 end to end on one set of tracks: the TRD
follower matches the seeds to tracklets, the TRD-only refit refits the
matched tracks, and the residuals of the same tracks' TPC clusters to the
combination of that refit with an ITS refit are collected per voxel.  The
CUDA chain (trd_follow -> trd_refit -> trd_residuals) against the oracle's
chain (follow -> refit -> residuals), each stage fed by its own side's
previous stage.

Tracks whose follower path or refit status differ between the two chains
(near-tie decisions of the follower) are left out of the comparison by
removing their clusters on both sides.  On the others the differences of the
three FP32 stages compound: each cluster residual within 1e-4 max(|dy|,
sigma) + 1e-3 cm (10^-2 of the 0.1 cm cluster resolution), the voxel counts
identical.
"""
import numpy as np
import pytest

from oracle import oracle as O
from parity import to_numpy
from synth import make_workload
from synth import tpc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2003_03174_b300 import trd
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return trd.Context(0)


def _f32(d, keys_f, keys_i):
    out = {k: np.ascontiguousarray(np.asarray(d[k], dtype=np.float32)) for k in keys_f}
    out.update({k: np.ascontiguousarray(np.asarray(d[k], dtype=np.int32)) for k in keys_i})
    return out


def test_calibration_chain_matches_the_oracle_chain(ctx):
    from paper_2003_03174_b300 import trd
    tf = make_workload("timeframe", seed=91, n_seeds=20_000)
    its, cl, _ = tpc.clusters_for_truth(tf.truth, bz=tf.params["bz"], seed=91)
    p = tf.params

    # the CUDA chain
    s, t = trd.to_device(tf.seeds), trd.to_device(tf.tracklets)
    idx = ctx.index_build(t)
    res = ctx.follow(s, idx, p)
    rf = ctx.refit(res, t, p)
    torch.cuda.synchronize()
    g_f, g_rf = to_numpy(res), to_numpy(rf)

    # the oracle chain
    o_f = O.follow(tf.seeds, tf.tracklets, p)
    o_rf = O.refit(_f32(o_f, ("alpha", "x", "par", "cov", "chi2"), ("n_trk", "n_miss", "status", "tracklet_id")),
                   tf.tracklets, p)

    same = ((g_f["tracklet_id"] == o_f["tracklet_id"]).all(0) & (g_f["status"] == o_f["status"]) &
            (g_rf["status"] == o_rf["status"]))
    assert same.mean() > 0.98
    assert (same & (g_rf["status"] == 0)).sum() > 10_000
    # the clusters of the other tracks are removed on both sides
    cl_cmp = {k: v.copy() for k, v in cl.items()}
    cl_cmp["sector"][:, ~same] = -1

    g_states = {k: g_rf[k] for k in ("alpha", "x", "par", "cov", "status")}
    sums, cres = ctx.residuals(trd.to_device(its), trd.to_device(g_states), trd.to_device(cl_cmp), p["bz"],
                               cluster_res=True)
    torch.cuda.synchronize()
    sums, cres = sums.cpu().numpy(), cres.cpu().numpy()
    o_states = _f32(o_rf, ("alpha", "x", "par", "cov"), ("status",))
    o = O.residuals(its, o_states, cl_cmp, p["bz"], with_clusters=True)

    ok_o, ok_g = o["vox"] >= 0, ~np.isnan(cres[0])
    near = (o["slack"] < 1e-3)[None, :].repeat(ok_o.shape[0], 0)
    assert not ((ok_o != ok_g) & ~near).any()
    both = ok_o & ok_g & ~near
    assert both.sum() > 1_000_000
    for k in (0, 1):
        sig = np.sqrt(o["var"][k][both])
        err = np.abs(cres[k][both].astype(np.float64) - o["res"][k][both])
        tol = 1e-4 * np.maximum(np.abs(o["res"][k][both]), sig) + 1e-3
        assert np.all(err <= tol), (k, float((err / tol).max()), float(err.max()))
    np.testing.assert_array_equal(sums[:, 0], o["sums"][:, 0].astype(np.int64))
