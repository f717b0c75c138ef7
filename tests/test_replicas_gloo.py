"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank runs an independent replica, so the only cross-rank step is the
max-over-ranks reduction of the step time; the whole-job value is every rank's
points over the slowest rank's time.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [100.0 + 50.0 * rank, 2.0 + rank]          # rank 1 is the slower one
        got = bench.reduce_max_over_ranks(local)
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_aggregate():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == [150.0, 3.0]
    import bench
    # 4 metrics x 1M points per rank, 2 ranks, slowest rank 150 ms
    assert bench.replica_throughput(4_000_000, 2, 150.0) == pytest.approx(8e6 / 0.150)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_max_over_ranks([1.5, 2.5]) == [1.5, 2.5]


def test_reference_arm_on_other_ranks_exits_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1"])
    bench.main()
    assert capsys.readouterr().out == ""
