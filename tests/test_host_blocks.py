"""Host-side packing of a timeframe's inputs and results into one block in
the server's copy order (no GPU: the block is not pinned here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_03174_b300 import trd  # noqa: E402
from synth import make_workload  # noqa: E402


@pytest.mark.parametrize("kw", [{}, dict(n_interactions=40), dict(misalign=0.5, x_jitter=0.1)])
def test_inputs_are_packed_in_copy_order(kw):
    tf = make_workload("tiny", seed=3, **kw)
    hs, ht = trd.pinned_inputs(tf.seeds, tf.tracklets, pin=False)
    assert ("trigger" in ht) == ("n_interactions" in kw) and ("x" in ht) == ("misalign" in kw)
    for src, dst in ((tf.seeds, hs), (tf.tracklets, ht)):
        assert set(dst) == set(src)
        for k in src:
            np.testing.assert_array_equal(dst[k].numpy(), src[k], err_msg=k)
    n, m = tf.n_seeds, tf.n_tracklets
    order = [(hs, k) for k in ("alpha", "x", "y", "z", "snp", "tgl", "q2pt", "cov")] + \
            [(ht, k) for k in ("chamber", "y", "z", "dy", "vyy", "vzz", "vyz")]
    if "trigger" in hs:
        order.append((hs, "trigger"))
    if "trigger" in ht:
        order.append((ht, "trigger"))
    if "x" in ht:
        order.append((ht, "x"))
    # every array starts where the previous one ends: the server merges them
    # into one copy
    p = order[0][0][order[0][1]].data_ptr()
    for d, k in order:
        assert d[k].data_ptr() == p, k
        p += d[k].numel() * 4
    assert p - hs["alpha"].data_ptr() == 4 * (22 * n + 7 * m + (n if "trigger" in hs else 0) +
                                            (m if "trigger" in ht else 0) + (m if "x" in ht else 0))


def test_result_views_follow_the_device_order():
    import paper_2003_03174_b300.trd as T
    block = torch.zeros(32 * 5, dtype=torch.int32)
    v = T._pinned_views(block, T._RESULT_ROWS, 5)
    assert v["par"].shape == (5, 5) and v["cov"].shape == (15, 5) and v["tracklet_id"].shape == (6, 5)
    assert v["par"].dtype == torch.float32 and v["status"].dtype == torch.int32
    base = block.data_ptr()
    assert v["alpha"].data_ptr() == base and v["chi2"].data_ptr() == base + 4 * 22 * 5
    assert v["n_trk"].data_ptr() == base + 4 * 23 * 5 and v["tracklet_id"].data_ptr() == base + 4 * 26 * 5
