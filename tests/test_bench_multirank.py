"""The bench's whole-job aggregation under two ranks (gloo on CPU): units are summed over
ranks and the time is the maximum over ranks, for the device-timed value and for e2e."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = [1.0e9, 3.0e9][rank]
        secs = [0.5, 0.8][rank]
        solves = [5.0, 5.0][rank]
        e2e = [[2.0e9, 1.0, 840, 100], [4.0e9, 1.5, 840, 100]][rank]
        vals, e2 = bench.aggregate([units, secs, solves], e2e, dist, "cpu")
        out[rank] = (vals, e2)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        vals, e2 = res[rank]
        assert vals == [4.0e9, 0.8, 10.0]          # units summed, time = max, solves summed
        assert e2[:2] == [6.0e9, 1.5] and e2[2:] == [840, 100]
    # the whole-job rate is the sum of units over the slowest rank's time
    assert res[0][0][0] / res[0][0][1] == pytest.approx(5.0e9)


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    vals, e2 = bench.aggregate([1.0, 2.0, 3.0], None, None, "cpu")
    assert vals == [1.0, 2.0, 3.0] and e2 is None
