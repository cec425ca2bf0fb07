"""N > 1 path of the benchmark on CPU: two gloo ranks each render their own frame (weak
scaling); the job value is the rays of all ranks over the slowest rank's step time."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [40.0, 55.0][rank]
    rays = [1000.0, 3000.0][rank]
    q.put((rank, bench.reduce_ranks(ms, rays, torch.device("cpu"))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (55.0, 4000.0)
