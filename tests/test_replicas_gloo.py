"""The multi-GPU form of the benchmark runs independent replicas (the step has
no exchange between independent domains): each rank times its own replica,
the job's time is the slowest rank's, and the throughput counts every rank's
cells.  This checks that host-side logic with two gloo ranks on the CPU."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [12.5, 20.0][rank]
    ms_max = bench.reduce_max(ms_local, world, "cpu")
    out[rank] = (ms_max, bench.replica_mlups(1000, 10, ms_max, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_cells():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        ms_max, mlups = out[r]
        assert ms_max == 20.0
        # 2 ranks x 1000 cells x 10 steps in 20 ms
        assert mlups == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.0, 1, "cpu") == 3.0
    assert bench.replica_mlups(100, 2, 1.0, 1) == pytest.approx(100 * 2 / 1e-3 / 1e6)
