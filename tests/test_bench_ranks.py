"""The benchmark's multi-rank path (replicas, one box per rank) on CPU with gloo:
the reported time is the slowest rank's and the particle count is all ranks' sum."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, n = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 + rank)
    # the reference arm prints only on rank 0 and the others return without work
    import argparse
    ran = bench.run_reference(argparse.Namespace(steps=0, warmup=0, workload="c512")) if rank else None
    q.put((rank, ms, n, ran))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, n, ran in res:
        assert ms == 20.0 and n == 2001.0
        assert ran is None


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(3.5, 7) == (3.5, 7.0)
