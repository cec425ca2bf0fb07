"""Pins of the oracle's adjoint into the environment map and the per-pixel materials
(directions and proposal density held fixed): closed forms under a white furnace, and
FP64 central differences of the oracle's own shading for every parameter kind, in
allocations whose proposal does not depend on the perturbed parameter."""
import numpy as np
import pytest

import oracle
from tests._handmade import gbuffer, random_gbuffer, scene
from paper_2607_22780_b300 import workloads as wl


def test_white_furnace_gradients_closed_form():
    # Lambert, cosine samples, no occluder, constant map L: colour = a L and light = L per
    # pixel, so dc/da = L, and the map gradient summed over texels is a (colour) or 1 (light)
    P = 6
    rng = np.random.default_rng(0)
    alb = rng.uniform(0.1, 0.9, (P, 3))
    gb = gbuffer(np.zeros((P, 3)), np.tile([0, 0, 1.0], (P, 1)), alb, np.full(P, 0.5), np.zeros(P), eye=(0, 0, 3))
    L = 1.5
    env = wl.envmap_constant(L, 32, 16)
    empty = scene([])
    fwd = oracle.shade_pixels(empty, gb, env, 16, 0, 0, seed=1, brdf=0)
    np.testing.assert_allclose(fwd["light"], L, rtol=1e-12)
    dc = rng.normal(size=(P, 3))
    g = oracle.backward_material(empty, gb, env, 16, 0, 0, seed=1, dL_dcolor=dc, brdf=0)
    np.testing.assert_allclose(g["albedo"], dc * L, rtol=1e-12)
    a32 = np.asarray(gb["albedo"], np.float64)
    np.testing.assert_allclose(g["env"].sum((0, 1)), (dc * a32).sum(0), rtol=1e-12)
    assert not g["rough"].any() and not g["metal"].any()
    dl = rng.normal(size=(P, 3))
    g2 = oracle.backward_material(empty, gb, env, 16, 0, 0, seed=1, dL_dcolor=np.zeros((P, 3)), dL_dlight=dl,
                                  brdf=0)
    np.testing.assert_allclose(g2["env"].sum((0, 1)), dl.sum(0), rtol=1e-12)


def _setup(alloc, seed=5, P=24):
    sc = wl.scene_random_soup(60, seed=seed, extent=0.5, scale_lo=0.1, scale_hi=0.3, color_dim=48)
    rng = np.random.default_rng(seed)
    gb = random_gbuffer(rng, P, eye=(0.0, 0.0, 3.0))
    gb["metal"] = rng.uniform(0.1, 0.9, P).astype(np.float32)
    gb["rough"] = rng.uniform(0.3, 0.9, P).astype(np.float32)
    env = wl.envmap_hdr(seed, 32, 16, sun_gain=20.0, sun_width=0.05)
    wc = rng.normal(size=(P, 3)); wl_ = rng.normal(size=(P, 3))
    return sc, gb, env, wc, wl_


def _loss(sc, gb, env, alloc, wc, wl_):
    r = oracle.shade_pixels(sc, gb, env, *alloc, seed=11)
    return float((wc * r["color"]).sum() + (wl_ * r["light"]).sum()), r["flags"]


def _fd(sc, gb, env, alloc, wc, wl_, key, idx, h, grad):
    arr = gb[key] if key != "env" else env
    x = float(arr.flat[idx])
    xp, xm = np.float32(x + h), np.float32(x - h)
    arr.flat[idx] = xp
    lp, fp = _loss(sc, gb, env, alloc, wc, wl_)
    arr.flat[idx] = xm
    lm, fm = _loss(sc, gb, env, alloc, wc, wl_)
    arr.flat[idx] = x
    fd = (lp - lm) / (float(xp) - float(xm))
    assert fd == pytest.approx(grad, rel=2e-4, abs=1e-7), (key, idx, fd, grad)


@pytest.mark.parametrize("key,alloc", [("albedo", (4, 2, 2)), ("metal", (4, 2, 2)), ("rough", (4, 0, 2))])
def test_material_gradients_vs_fd(key, alloc):
    # albedo and metal do not enter the proposal; roughness does through the GGX pdf and
    # samples, so its check uses no GGX proposals
    sc, gb, env, wc, wl_ = _setup(alloc)
    g = oracle.backward_material(sc, gb, env, *alloc, seed=11, dL_dcolor=wc, dL_dlight=wl_)
    assert np.all(g["flags"] == 0)
    grad = g[key].reshape(-1)
    rng = np.random.default_rng(1)
    for idx in rng.choice(grad.size, 8, replace=False):
        _fd(sc, gb, env, alloc, wc, wl_, key, int(idx), 1e-3, grad[idx])


def test_map_gradients_vs_fd():
    # without environment proposals the map enters the estimate linearly
    alloc = (4, 2, 0)
    sc, gb, env, wc, wl_ = _setup(alloc)
    g = oracle.backward_material(sc, gb, env, *alloc, seed=11, dL_dcolor=wc, dL_dlight=wl_)
    ge = g["env"].reshape(-1)
    hit = np.nonzero(ge)[0]
    assert len(hit) > 20
    rng = np.random.default_rng(2)
    for idx in rng.choice(hit, 10, replace=False):
        _fd(sc, gb, env, alloc, wc, wl_, "env", int(idx), 1e-2 * max(1.0, abs(float(env.flat[idx]))), ge[idx])


def test_roughness_clamp_has_no_gradient():
    sc, gb, env, wc, wl_ = _setup((4, 0, 2))
    gb["rough"][:] = 0.005   # r^2 < 1e-4: alpha is clamped
    g = oracle.backward_material(sc, gb, env, 4, 0, 2, seed=11, dL_dcolor=wc)
    assert not g["rough"].any()
