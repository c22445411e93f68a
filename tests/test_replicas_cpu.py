"""The bench's multi-GPU path is replicas only (no data-path collective): each
rank runs its own copy of the workload; the job's time is the slowest rank's
and the job's rate counts every rank's units.  Checked with two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    local_ms = 10.0 * (rank + 1)
    ms = bench.max_over_ranks(local_ms, ws, "cpu")
    rate = bench.job_rate(100.0, 4, ws, ms)
    out[rank] = (ms, rate)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
        res = dict(out)
    for r in range(ws):
        ms, rate = res[r]
        assert ms == 20.0  # the slowest rank
        assert abs(rate - ws * 4 * 100.0 / 0.020) < 1e-9


def test_one_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(10.0, 2, 1, 1000.0) == 20.0
