"""Multi-GPU mode of the benchmark is replicas only (the method is not
sharded): each rank runs its own copy and rank 0 reports the slowest rank's
time and the sum of all ranks' work.  The host-side reduction runs here as two
gloo processes on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = (10.0, 1.0e9) if rank == 0 else (12.5, 3.0e9)
    out[rank] = bench.aggregate_ranks(ms, units, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (12.5, 4.0e9)  # max time, summed work, on every rank


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(7.0, 5) == (7.0, 5.0)
