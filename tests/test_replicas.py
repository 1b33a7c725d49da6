"""Multi-GPU runs are independent replicas: two gloo ranks on the CPU check
the slowest-rank timing and the whole-job throughput, and that each rank gets
its own stimulus location (no data-path exchange to test)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank
    ms, value = bench.replica_time(ms_local, world, dist, torch.device("cpu"))
    geom, grid, cfg, V0, w0 = bench.workload(16, rank)
    centre = np.argwhere(V0 > 0).mean(axis=0)
    out[rank] = (ms, value, tuple(centre))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_and_stimuli():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == out[1][1] == pytest.approx(world * 1000.0 / 15.0)
    assert out[0][2] != out[1][2]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_time(20.0, 1) == (20.0, 50.0)
