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


# ----------------------------------------------------------------------------- one frame on several ranks
# The plumbing of paper_2607_22780_b300.shard on gloo ranks: pixel shards, the image gather
# and the gradient all-reduce, with a stand-in per-pixel "shader" (a fixed function of the
# pixel index) and a stand-in adjoint, so that nothing here needs a GPU.

def _fake_shade(pixels):
    import torch
    p = pixels.double()
    return [torch.stack([p, 2 * p + 1, torch.sin(p)], 1), (p % 7) / 7.0]


def _fake_adjoint(grads):
    def run(pixels):
        import torch
        g = grads[0]
        # every pixel adds its index to surfel (pixel mod 13), and 1 to a second buffer
        g.index_add_(0, (pixels.long() % g.shape[0]), pixels.double())
        grads[1] += pixels.numel()
    return run


def _frame_valid(P=997, seed=0):
    import torch
    gen = torch.Generator().manual_seed(seed)
    return (torch.rand(P, generator=gen) > 0.3).to(torch.int32)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    from paper_2607_22780_b300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    valid = _frame_valid()
    outs, pixels = shard.shade_frame(_fake_shade, valid)
    grads = [torch.zeros(13, dtype=torch.float64), torch.zeros(1, dtype=torch.float64)]
    shard.backward_frame(_fake_adjoint(grads), grads, valid)
    q.put((rank, [o.numpy() for o in outs], pixels.numpy(), [g.numpy() for g in grads]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_frame_shards_gather_and_gradient_reduce_on_gloo(world):
    import numpy as np
    import torch
    from paper_2607_22780_b300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + world + os.getpid() % 500
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (o, px, g)) for r, o, px, g in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the single-process result of the same frame
    valid = _frame_valid()
    full = shard.partition(valid, 0, 1)
    ref_rows = _fake_shade(full)
    ref = [torch.zeros((valid.numel(),) + tuple(t.shape[1:]), dtype=t.dtype) for t in ref_rows]
    for r_, t in zip(ref, ref_rows):
        r_[full.long()] = t
    g_ref = [torch.zeros(13, dtype=torch.float64), torch.zeros(1, dtype=torch.float64)]
    _fake_adjoint(g_ref)(full)
    # shares are disjoint, cover every valid pixel, and differ in size by at most one
    shares = [res[r][1] for r in range(world)]
    allp = np.concatenate(shares)
    assert len(allp) == len(set(allp.tolist())) == int(valid.sum())
    assert max(map(len, shares)) - min(map(len, shares)) <= 1
    for r in range(world):
        outs, _, grads = res[r]
        for a, b in zip(outs, ref):
            assert np.array_equal(a, b.numpy())        # the gathered image, on every rank
        for a, b in zip(grads, g_ref):
            assert np.array_equal(a, b.numpy())        # the all-reduced gradient, on every rank
