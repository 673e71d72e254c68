"""The multi-GPU form is replicas only (requests and benchmark replicas are
independent; no collective on the data path).  The bench's whole-job
aggregation (max time over ranks, summed throughput) is checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    t = bench.job_time(ms, dist)
    v = bench.job_mlups(1000, 10, world, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_job_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 150.0
        assert v == pytest.approx(world * 1000 * 10 / 0.150 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.job_time(12.5, None) == 12.5
