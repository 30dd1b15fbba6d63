"""The N > 1 bench path (replicas, no data-path collective) on CPU with gloo:
the whole-job time is the slowest rank's and the converged pairs add up."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, c = bench.aggregate(1.0 + rank, 64 - rank, dist, "cpu")
    out[rank] = (t, c)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_world2_gloo():
    import torch.multiprocessing as mp

    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0] == (2.0, 127) and out[1] == (2.0, 127)


def test_aggregate_single_rank_passthrough():
    import bench

    assert bench.aggregate(0.5, 64) == (0.5, 64)
