"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1, the way torchrun runs
the bench with one replica a rank.  Each rank times its own replica; the job's time is the
slowest rank's, its work the sum over the ranks, and its rate their ratio (weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t_ms = 10.0 + 5.0 * rank               # rank 1 is the slower replica
        units = 1000.0 * (rank + 1)            # replicas need not do equal work
        t_max = bench.over_ranks(t_ms, dist, "cpu", "max")
        u_sum = bench.over_ranks(units, dist, "cpu", "sum")
        out[rank] = (t_max, u_sum, bench.replicas_rate(u_sum, t_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        t_max, u_sum, rate = out[r]
        assert t_max == 15.0 and u_sum == 3000.0
        assert rate == pytest.approx(3000.0 / 15e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(12.5, None, "cpu", "max") == 12.5
    assert bench.replicas_rate(2.0e9, 4.0) == pytest.approx(5.0e11)
