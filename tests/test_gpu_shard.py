"""One frame split by pixels across ranks on the CUDA path (paper_2607_22780_b300.shard):
the gathered image equals the single-rank image bit for bit, and the all-reduced
gradient equals the single-rank gradient up to the order of float atomic additions.

The two-rank case runs two processes on the one GPU of the box, exchanging over gloo on
the host (no kernel of one rank waits on the other's)."""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2607_22780_b300 import api, shard, workloads as wl

pytestmark = pytest.mark.gpu

ALLOC = (8, 4, 4)
SEED = 17


def _setup():
    sc = wl.scene_objects(20_000, seed=5)
    S = api.Scene.from_workload(sc)
    cam = wl.camera_orbit(5, 64, 64, 3.0)
    G = api.gbuffer_primary(S, cam)
    E = api.Environment(torch.from_numpy(wl.envmap_hdr(5, 64, 32)).cuda())
    tgt = torch.from_numpy(wl.target_image(5, 64, 64).reshape(-1, 3)).cuda()
    return S, G, E, tgt


def _frame(S, G, E, tgt, host=False):
    """(image outputs, gradients) of the whole frame, one rank or sharded."""
    def shade(px):
        out = api.shade_pixels(S, G, E, *ALLOC, seed=SEED, pixels=px.cuda())
        return [t.cpu() for t in out] if host else list(out)

    outs, _ = shard.shade_frame(shade, G.valid.cpu() if host else G.valid)
    col = outs[0].cuda()
    dl_full = ((col - tgt) * G.valid.unsqueeze(1).float()).contiguous()
    g = api.SurfelGrads.zeros(S)

    def adjoint(px):
        api.shade_backward(S, G, E, *ALLOC, SEED, dl_full[px.long().cuda()].contiguous(), pixels=px.cuda(), grads=g)

    bufs = [g.mu, g.quat, g.scale, g.opacity, g.color]
    if not host:
        shard.backward_frame(adjoint, bufs, G.valid)
        return [o.cpu() for o in outs], [b.cpu() for b in bufs]
    # gloo ranks: this rank's share on the GPU, the sum over ranks on host copies
    adjoint(shard.partition(G.valid.cpu(), *shard.rank_world()))
    hbufs = [b.cpu() for b in bufs]
    shard.reduce_grads(hbufs)
    return [o.cpu() for o in outs], hbufs


def _close(a, b):
    for x, y in zip(a, b):
        tol = 1e-4 * float(y.abs().max()) + 1e-12
        assert float((x - y).abs().max()) <= tol


def test_single_rank_frame_equals_whole_frame_calls():
    S, G, E, tgt = _setup()
    outs, grads = _frame(S, G, E, tgt)
    ref = api.shade_pixels(S, G, E, *ALLOC, seed=SEED)
    for a, b in zip(outs, ref):
        assert torch.equal(a, b.cpu())
    dl = ((ref[0] - tgt) * G.valid.unsqueeze(1).float()).contiguous()
    g = api.shade_backward(S, G, E, *ALLOC, SEED, dl)
    _close(grads, [t.cpu() for t in (g.mu, g.quat, g.scale, g.opacity, g.color)])
    assert S.status() == 0


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S, G, E, tgt = _setup()
        outs, grads = _frame(S, G, E, tgt, host=True)
        # the same frame on this rank alone, for comparison
        ref = api.shade_pixels(S, G, E, *ALLOC, seed=SEED)
        dl = ((ref[0] - tgt) * G.valid.unsqueeze(1).float()).contiguous()
        g = api.shade_backward(S, G, E, *ALLOC, SEED, dl)
        same_image = all(torch.equal(a, b.cpu()) for a, b in zip(outs, ref))
        _close(grads, [t.cpu() for t in (g.mu, g.quat, g.scale, g.opacity, g.color)])
        q.put((rank, same_image, S.status()))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e), -1))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_gloo_match_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 500
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, same, status in res:
        assert same is True, (rank, same)
        assert status == 0
