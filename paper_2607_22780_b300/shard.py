"""One frame on several GPUs: pixel shards, an image gather and a gradient all-reduce.

Every pixel's secondary rays are independent given the resident surfels and their tree
(the paper optimises on a pixel subset per iteration, Sec. III-F), so a frame splits
across ranks by pixels with nothing exchanged while it is traced:

* forward: every rank holds the whole scene and BVH, shades its own contiguous share of
  the frame's valid pixels (`pixel_list`), and an all-gather assembles the image;
* backward: each rank runs the adjoint over its share only, into a full per-surfel
  gradient buffer, and one all-reduce (sum) of the 58 floats per surfel (mu 3, quat 4,
  scale 2, opacity 1, SH 48) gives every rank the gradient of the whole frame.

A pixel's result depends only on its own samples, so the sharded image equals the
single-GPU image bit for bit, and the reduced gradient equals the single-GPU gradient up
to the order of float additions.  The collectives are torch.distributed calls (NCCL on
GPUs, gloo on CPU); the shading itself is whatever `shade` / `adjoint` callable the caller
passes (the CUDA library's shade_pixels / shade_backward in use).
"""
from __future__ import annotations

from typing import Callable, Sequence, Tuple

import torch
import torch.distributed as dist


def rank_world(group=None) -> Tuple[int, int]:
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def partition(valid: torch.Tensor, rank: int, world: int) -> torch.Tensor:
    """This rank's share of the valid pixels: int32 raster indices, contiguous in raster
    order, shares differing in size by at most one pixel."""
    idx = torch.nonzero(valid.reshape(-1) != 0).reshape(-1).to(torch.int32)
    n = idx.numel()
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return idx[lo:hi].contiguous()


def gather_rows(local: torch.Tensor, pixels: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """Rows local[i] belong to pixel pixels[i] of this rank; returns the [n_total, ...]
    array of every rank's rows in place (zeros where no rank shaded a pixel)."""
    rank, world = rank_world(group)
    out = torch.zeros((n_total,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    if world == 1:
        out[pixels.long()] = local
        return out
    counts = torch.tensor([pixels.numel()], device=local.device, dtype=torch.int64)
    all_counts = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    m = int(max(int(c.item()) for c in all_counts))
    # all_gather wants equal shapes: pad every share to the largest
    pad_rows = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad_rows[:local.shape[0]] = local
    pad_pix = torch.full((m,), -1, dtype=torch.int64, device=local.device)
    pad_pix[:pixels.numel()] = pixels.long()
    rows = [torch.empty_like(pad_rows) for _ in range(world)]
    pix = [torch.empty_like(pad_pix) for _ in range(world)]
    dist.all_gather(rows, pad_rows, group=group)
    dist.all_gather(pix, pad_pix, group=group)
    for r, p in zip(rows, pix):
        keep = p >= 0
        out[p[keep]] = r[keep]
    return out


def shade_frame(shade: Callable[[torch.Tensor], Sequence[torch.Tensor]], valid: torch.Tensor, group=None):
    """Forward of one frame split across the ranks: shade(pixels) -> per-pixel outputs of
    this rank's pixels (colour [n,3], visibility [n], indirect [n,3], ...); returns the
    full-frame outputs, the same on every rank, and this rank's pixel list."""
    rank, world = rank_world(group)
    pixels = partition(valid, rank, world)
    local = shade(pixels)
    P = valid.numel()
    return [gather_rows(t, pixels, P, group) for t in local], pixels


def reduce_grads(tensors: Sequence[torch.Tensor], group=None) -> None:
    """Sum every rank's per-surfel gradient buffers in place (one all-reduce over one flat
    buffer of all of them)."""
    rank, world = rank_world(group)
    if world == 1 or not tensors:
        return
    flat = torch.cat([t.reshape(-1) for t in tensors])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for t in tensors:
        n = t.numel()
        t.copy_(flat[off:off + n].view_as(t))
        off += n


def backward_frame(adjoint: Callable[[torch.Tensor], None], grads: Sequence[torch.Tensor], valid: torch.Tensor,
                   group=None) -> torch.Tensor:
    """Adjoint of one frame split across the ranks: adjoint(pixels) accumulates this rank's
    share into `grads` (zeroed by the caller on every rank), then one all-reduce sums the
    shares.  Returns this rank's pixel list."""
    rank, world = rank_world(group)
    pixels = partition(valid, rank, world)
    adjoint(pixels)
    reduce_grads(grads, group)
    return pixels
