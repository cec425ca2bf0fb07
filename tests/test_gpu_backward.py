"""GPU parity of the adjoint kernels against the oracle's FP64 gradient.

Tolerance: |g_gpu - g_ref| <= 2e-3 |g_ref| + 1e-5 max|g_ref| per parameter block (FP32
atomics and FP32 geometry against FP64)."""
import numpy as np
import pytest
import torch

import oracle
from tests._gpu import check_grads, random_rays, scene_gpu, t
from tests._handmade import random_gbuffer
from paper_2607_22780_b300 import api, autograd, workloads as wl

pytestmark = pytest.mark.gpu

_check = check_grads


@pytest.mark.parametrize("color_dim", [3, 48])
def test_ray_backward_matches_oracle(color_dim):
    sc = wl.scene_random_soup(400, seed=7, extent=0.6, scale_lo=0.05, scale_hi=0.2, color_dim=color_dim)
    rng = np.random.default_rng(8)
    o, d = random_rays(rng, 4000, -1.5, 1.5, 0.5)
    wr = rng.normal(size=(4000, 3)).astype(np.float32)
    wo = rng.normal(size=4000).astype(np.float32)
    ref = oracle.backward_rays(sc, o, d, wr, wo)
    keep = ref["flags"] == 0
    o, d, wr, wo = o[keep], d[keep], wr[keep], wo[keep]
    ref = oracle.backward_rays(sc, o, d, wr, wo)
    S = scene_gpu(sc)
    g = api.trace_backward(S, t(o), t(d), t(wr), t(wo))
    _check(g, ref)


def test_autograd_trace_function():
    sc = wl.scene_random_soup(200, seed=9, extent=0.5, scale_lo=0.05, scale_hi=0.2, color_dim=48)
    rng = np.random.default_rng(10)
    o, d = random_rays(rng, 1000, -1.5, 1.5, 0.4)
    S = scene_gpu(sc)
    for p in (S.mu, S.quat, S.scale, S.opacity, S.color):
        p.requires_grad_(True)
    rgb, op = autograd.trace(S, t(o), t(d))
    loss = (rgb ** 2).sum() + op.sum()
    loss.backward()
    ref_rgb = oracle.trace_rays(sc, o, d)
    g = oracle.backward_rays(sc, o, d, 2 * ref_rgb["rgb"], np.ones(len(o)))
    got = api.SurfelGrads(S.mu.grad, S.quat.grad, S.scale.grad, S.opacity.grad, S.color.grad)
    _check(got, g, rel=5e-3, absf=5e-5)


def test_shade_backward_matches_oracle():
    sc = wl.scene_random_soup(300, seed=12, extent=0.6, scale_lo=0.05, scale_hi=0.25, color_dim=48)
    rng = np.random.default_rng(13)
    gb = random_gbuffer(rng, 256, eye=(0.0, 0.0, 3.0))
    env = wl.envmap_hdr(4, 64, 32, sun_gain=20.0, sun_width=0.05)
    dc = rng.normal(size=(256, 3)).astype(np.float32)
    dv = rng.normal(size=256).astype(np.float32)
    di = rng.normal(size=(256, 3)).astype(np.float32)
    ref = oracle.backward_pixels(sc, gb, env, 8, 4, 4, seed=21, dL_dcolor=dc, dL_dvis=dv, dL_dind=di)
    assert (ref["flags"] == 0).mean() > 0.97
    keep = np.nonzero(ref["flags"] == 0)[0].astype(np.int32)
    ref = oracle.backward_pixels(sc, gb, env, 8, 4, 4, seed=21, dL_dcolor=dc[keep], dL_dvis=dv[keep],
                                 dL_dind=di[keep], pixels=keep)
    S = scene_gpu(sc)
    G = api.GBuffer.from_arrays(gb)
    E = api.Environment(t(env))
    g = api.shade_backward(S, G, E, 8, 4, 4, 21, t(dc[keep]), t(dv[keep]), t(di[keep]),
                           pixels=t(keep, torch.int32))
    _check(g, ref)


def _objects_gb(n=20000, W=40, H=32, seed=51):
    sc = wl.scene_objects(n, seed=seed)
    cam = wl.camera_orbit(seed, W, H, 3.0)
    gb32 = oracle.gbuffer_f32(oracle.gbuffer(sc, cam))
    return sc, gb32, wl.envmap_hdr(seed, 128, 64)


def _close(g, h):
    for f in ("mu", "quat", "scale", "opacity", "color"):
        x, y = getattr(g, f), getattr(h, f)
        assert torch.allclose(x, y, rtol=1e-4, atol=1e-6 * float(y.abs().max())), f


@pytest.mark.parametrize("max_hits", [16, 2, 0])
def test_saved_record_replay_equals_recompute(max_hits):
    # the same hits in the same order: replayed (rays with <= max_hits hits) or traced again
    sc, gb32, env = _objects_gb()
    S = scene_gpu(sc)
    G = api.GBuffer.from_arrays(gb32)
    E = api.Environment(t(env))
    a = api.shade_pixels(S, G, E, 8, 4, 4, seed=3)
    col, vis, ind, saved = api.shade_pixels_save(S, G, E, 8, 4, 4, seed=3, max_hits=max_hits)
    for x, y in zip(a, (col, vis, ind)):
        assert torch.equal(x, y)
    rng = np.random.default_rng(max_hits)
    n = gb32["W"] * gb32["H"]
    dc, dv, di = (t(rng.normal(size=sh).astype(np.float32)) for sh in ((n, 3), (n,), (n, 3)))
    g0 = api.shade_backward(S, G, E, 8, 4, 4, 3, dc, dv, di)
    g1 = api.shade_backward(S, G, E, 8, 4, 4, 3, dc, dv, di, saved=saved)
    _close(g1, g0)
    assert S.status() == 0


def test_saved_record_backward_matches_oracle():
    sc = wl.scene_random_soup(300, seed=12, extent=0.6, scale_lo=0.05, scale_hi=0.25, color_dim=48)
    rng = np.random.default_rng(14)
    gb = random_gbuffer(rng, 256, eye=(0.0, 0.0, 3.0))
    env = wl.envmap_hdr(4, 64, 32, sun_gain=20.0, sun_width=0.05)
    pre = oracle.backward_pixels(sc, gb, env, 8, 4, 4, seed=22, dL_dcolor=np.ones((256, 3)))
    keep = np.nonzero(pre["flags"] == 0)[0].astype(np.int32)
    dc = rng.normal(size=(len(keep), 3)).astype(np.float32)
    ref = oracle.backward_pixels(sc, gb, env, 8, 4, 4, seed=22, dL_dcolor=dc, pixels=keep)
    S = scene_gpu(sc)
    G = api.GBuffer.from_arrays(gb)
    E = api.Environment(t(env))
    pk = t(keep, torch.int32)
    _, _, _, saved = api.shade_pixels_save(S, G, E, 8, 4, 4, seed=22, pixels=pk, max_hits=4)
    g = api.shade_backward(S, G, E, 8, 4, 4, 22, t(dc), pixels=pk, saved=saved)
    _check(g, ref)


def test_autograd_shade_store_and_recompute_agree():
    sc, gb32, env = _objects_gb(n=15000, W=24, H=20, seed=52)
    tgt = t(wl.target_image(52, 20, 24).reshape(-1, 3))
    out = []
    for store in (16, None):
        S = scene_gpu(sc)
        for p in (S.mu, S.quat, S.scale, S.opacity, S.color):
            p.requires_grad_(True)
        G = api.GBuffer.from_arrays(gb32)
        E = api.Environment(t(env))
        col, vis, ind = autograd.shade(S, G, E, (8, 4, 4), 9, store_hits=store)
        loss = 0.5 * ((col - tgt) ** 2).sum() + vis.sum()
        loss.backward()
        out.append(api.SurfelGrads(S.mu.grad, S.quat.grad, S.scale.grad, S.opacity.grad, S.color.grad))
    _close(out[0], out[1])
    assert float(out[0].opacity.abs().sum()) > 0
