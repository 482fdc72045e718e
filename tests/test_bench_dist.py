"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
rank times are combined by a max all-reduce and the throughput counts every
rank's work over the slowest rank's time (weak scaling, no data collective)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [2.0, 3.0][rank]
    ms, value, edges_per_s = bench.aggregate_ranks(ms_local, 1.0e9, 2.0e6, world, dist, "cpu")
    out[rank] = (ms, value, edges_per_s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_work():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value, eps = out[r]
        assert ms == pytest.approx(3.0)
        assert value == pytest.approx(2 * 1.0e9 / 3e-3)
        assert eps == pytest.approx(2 * 2.0e6 / 3e-3)


def test_single_rank_uses_local_time():
    import bench

    ms, value, eps = bench.aggregate_ranks(4.0, 1e9, 1e6, 1)
    assert ms == 4.0 and value == pytest.approx(1e9 / 4e-3)
