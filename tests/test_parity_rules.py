"""The parity comparison's own rules, on hand-made results (no GPU): a track
on the oracle's path is held to the tolerances; a near tie of a decision
(the oracle's margin below 1e-3) exempts a track whose path or state differs;
without a near tie any difference fails."""
import numpy as np
import pytest

from parity import compare


def _oracle(n=3):
    rng = np.random.default_rng(4)
    cov = np.zeros((15, n))
    for i, k in enumerate((0, 2, 5, 9, 14)):
        cov[k] = 10.0 ** -(i + 1)
    return dict(
        tracklet_id=np.tile(np.array([[7], [-1], [9], [11], [-1], [-1]]), (1, n)).astype(np.int32),
        status=np.full(n, 2, np.int32), n_trk=np.full(n, 3, np.int32), n_miss=np.full(n, 2, np.int32),
        margin=np.full((6, n), 0.5), par=rng.normal(size=(5, n)) + 3.0, cov=cov,
        chi2=np.full(n, 7.25), x=np.full(n, 350.4), alpha=np.full(n, 2.2689))


def _gpu_like(ora):
    return {k: (v.astype(np.float32) if v.dtype.kind == "f" else v.copy()) for k, v in ora.items() if k != "margin"}


def test_identical_results_are_on_the_oracles_path():
    ora = _oracle()
    rep = compare(_gpu_like(ora), ora)
    assert rep["same_path"] == 3 and rep["exempt"] == 0


def test_a_near_tie_exempts_a_state_that_moved_with_the_same_ids():
    # a stack-boundary near tie (4e-5 cm) at layer 4: the GPU carried the
    # hypothesis on to the chamber's radius, the oracle did not; same ids
    ora = _oracle()
    ora["margin"][4, 1] = 4e-5
    g = _gpu_like(ora)
    g["par"][0, 1] += 0.1
    g["x"][1] = 350.0
    rep = compare(g, ora)
    assert rep["exempt"] == 1 and rep["same_path"] == 2


def test_without_a_near_tie_a_moved_state_fails():
    ora = _oracle()
    g = _gpu_like(ora)
    g["par"][0, 1] += 0.1
    with pytest.raises(AssertionError, match="par: 1 tracks"):
        compare(g, ora)


def test_a_near_tie_exempts_a_different_path_and_a_late_tie_does_not():
    ora = _oracle()
    g = _gpu_like(ora)
    g["tracklet_id"][2, 0] = 12  # differs at layer 2
    ora["margin"][1, 0] = 1e-4   # a near tie before it: exempt
    rep = compare(g, ora)
    assert rep["exempt"] == 1
    ora2 = _oracle()
    ora2["margin"][4, 0] = 1e-4  # the near tie comes after the first difference
    with pytest.raises(AssertionError, match="path: 1 tracks"):
        compare(g, ora2)
