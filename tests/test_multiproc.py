"""The N > 1 path of bench.py (one process per GPU, replicas of the solve,
no data-path collective) on two gloo ranks on the CPU: the timing barrier,
the maximum of the per-rank times and the sum of the per-rank work, and the
reference arm, which only rank 0 runs."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        mx = bench.max_over_ranks(1.5 + rank, world)
        sm = bench.sum_over_ranks(10.0 * (rank + 1), world)

        class A:
            steps, warmup, gpus = 1, 0, world
        # rank != 0 leaves the reference arm at once, without work or output
        ran = None
        if rank != 0:
            ran = bench.run_reference(A, world, rank)
        out.put((rank, mx, sm, ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, ran in res:
        assert mx == 2.5 and sm == 30.0
        if rank != 0:
            assert ran is None
