"""torch.autograd wrappers: forward and backward are libgrt kernels (Sec. III-B: gradients
flow through the secondary-ray trace into the surfel parameters)."""
from __future__ import annotations

import torch

from . import api


class TraceFunction(torch.autograd.Function):
    """(c_rt, o_rt) = Trace(ray_o, ray_d) as a function of the scene's surfel tensors.

    The scene's BVH must have been built or refit from the same mu/quat/scale/opacity.
    Gradients flow to mu, quat, scale, opacity and color (not to the rays).
    """

    @staticmethod
    def forward(ctx, scene: api.Scene, ray_o, ray_d, mu, quat, scale, opacity, color):
        rgb, op = api.trace_forward(scene, ray_o, ray_d)
        ctx.scene = scene
        ctx.save_for_backward(ray_o, ray_d)
        return rgb, op

    @staticmethod
    def backward(ctx, g_rgb, g_op):
        ray_o, ray_d = ctx.saved_tensors
        g = api.trace_backward(ctx.scene, ray_o, ray_d, g_rgb.contiguous(),
                               None if g_op is None else g_op.contiguous())
        return None, None, None, g.mu, g.quat, g.scale, g.opacity, g.color


class ShadeFunction(torch.autograd.Function):
    """(colour, visibility, indirect) = shade_pixels(...) as a function of the surfels.

    With store_hits = L the forward keeps each ray's first L composited hits and the
    backward replays them (rays with more hits are traced again); with store_hits = None
    the backward recomputes every hit list (no per-ray memory kept between the passes)."""

    @staticmethod
    def forward(ctx, scene, gb, env, alloc, seed, brdf, pixels, store_hits, mu, quat, scale, opacity, color):
        if store_hits is None:
            col, vis, ind = api.shade_pixels(scene, gb, env, *alloc, seed, brdf=brdf, pixels=pixels)
            saved = None
        else:
            col, vis, ind, saved = api.shade_pixels_save(scene, gb, env, *alloc, seed, brdf=brdf, pixels=pixels,
                                                         max_hits=store_hits)
        ctx.args = (scene, gb, env, alloc, seed, brdf, pixels, saved)
        return col, vis, ind

    @staticmethod
    def backward(ctx, g_col, g_vis, g_ind):
        scene, gb, env, alloc, seed, brdf, pixels, saved = ctx.args
        ctx.args = None
        n = gb.W * gb.H if pixels is None else int(pixels.shape[0])
        dev = gb.pos.device
        g_col = g_col.contiguous() if g_col is not None else torch.zeros((n, 3), device=dev)
        g = api.shade_backward(scene, gb, env, *alloc, seed, g_col,
                               None if g_vis is None else g_vis.contiguous(),
                               None if g_ind is None else g_ind.contiguous(), brdf=brdf, pixels=pixels, saved=saved)
        return (None,) * 8 + (g.mu, g.quat, g.scale, g.opacity, g.color)


def trace(scene, ray_o, ray_d):
    return TraceFunction.apply(scene, ray_o, ray_d, scene.mu, scene.quat, scene.scale, scene.opacity, scene.color)


def shade(scene, gb, env, alloc, seed, brdf=1, pixels=None, store_hits=64):
    return ShadeFunction.apply(scene, gb, env, tuple(alloc), seed, brdf, pixels, store_hits, scene.mu, scene.quat,
                               scene.scale, scene.opacity, scene.color)
