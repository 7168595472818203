"""The multi-GPU form is replicas only (one independent H-LU per rank); the
only communication is the scalar reduction of timing and work.  Exercised
here with two gloo ranks on the CPU: barrier, max of the times, sum of the
work, and the whole-job throughput bench.py reports from them."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ops = bench.RankOps(world, "cpu")
    ops.barrier()
    t_max = ops.max(100.0 + 50.0 * rank)       # rank 1 is the slower replica
    work = ops.sum(1e9 * (rank + 1))            # 1 and 2 GFLOP
    out[rank] = (t_max, work, bench.aggregate(t_max, work))
    ops.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_time_and_work():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t_max, work, value = out[r]
        assert t_max == 150.0 and work == 3e9
        assert value == pytest.approx(3e9 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    ops = bench.RankOps(1, "cpu")
    ops.barrier()
    assert ops.max(7.0) == 7.0 and ops.sum(7.0) == 7.0
