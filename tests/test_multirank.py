"""Host logic of the multi-rank benchmark, on CPU with gloo (world size 2):
each rank follows its own timeframe, and the only collective reduces the
timing scalars (max over ranks) and the matched counts (sum)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total, matched = bench.reduce_over_ranks(1.5 + rank, 1000 * (rank + 1))
    out[rank] = (total, matched, bench.rank_workload_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_timing_and_sum_matched():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.5        # slowest rank's time
    assert out[0][1] == out[1][1] == 3000.0     # matched tracks of all ranks
    assert out[0][2] != out[1][2]               # different timeframes per rank


def test_single_process_needs_no_collective():
    import bench
    assert bench.reduce_over_ranks(0.25, 7) == (0.25, 7.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=1, warmup=3, gpus=2, ref_sample=10)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
