"""Pins of the oracle's analytic adjoint of Eq. 8 (and of the shaded outputs) by FP64
central finite differences of the oracle's own forward pass, plus closed forms."""
import math

import numpy as np
import pytest

import oracle
from tests._handmade import Q_NZ, random_gbuffer, scene
from paper_2607_22780_b300 import workloads as wl

FIELDS = ("mu", "quat", "scale", "opacity", "color")


def _f64(sc):
    return wl.Scene(**{k: np.array(v, np.float64) for k, v in sc.arrays().items()})


def _perturbed(sc, field, idx, h):
    s2 = wl.Scene(**{k: v.copy() for k, v in sc.arrays().items()})
    getattr(s2, field).reshape(-1)[idx] += h
    return s2


def _fd_check(sc, loss, grads, rng, n_params=40, rel=1e-5):
    """Central differences on random parameters; skips parameters whose hit sets change."""
    checked = 0
    for _ in range(n_params * 3):
        f = FIELDS[rng.integers(len(FIELDS))]
        arr = getattr(sc, f).reshape(-1)
        i = int(rng.integers(arr.size))
        g = grads[f].reshape(-1)[i]
        h = 1e-6 * max(1.0, abs(arr[i]))
        lp, kp = loss(_perturbed(sc, f, i, h))
        lm, km = loss(_perturbed(sc, f, i, -h))
        if kp != km:
            continue
        fd = (lp - lm) / (2 * h)
        scale = max(abs(fd), abs(g), 1e-6)
        assert abs(fd - g) <= rel * scale + 1e-9, (f, i, fd, g)
        checked += 1
        if checked == n_params:
            break
    assert checked >= n_params // 2


@pytest.mark.parametrize("color_dim", [3, 48])
def test_ray_mode_gradient_vs_fd(color_dim):
    rng = np.random.default_rng(10 + color_dim)
    sc = _f64(wl.scene_random_soup(40, seed=4, extent=0.4, scale_lo=0.1, scale_hi=0.3, color_dim=color_dim))
    R = 300
    o = rng.uniform(-1.2, 1.2, size=(R, 3)).astype(np.float32)
    tgt = rng.uniform(-0.2, 0.2, size=(R, 3))
    d = (tgt - o); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    wr = rng.normal(size=(R, 3)); wo = rng.normal(size=R)

    def loss(s):
        r = oracle.trace_rays(s, o, d)
        return float(np.sum(wr * r["rgb"]) + np.sum(wo * r["opacity"])), \
            (r["hits"].tobytes(), r["nhits"].tobytes())

    grads = oracle.backward_rays(sc, o, d, wr, wo)
    assert np.all(grads["flags"] == 0)
    _fd_check(sc, loss, grads, rng)


def test_pixel_mode_gradient_vs_fd():
    rng = np.random.default_rng(21)
    sc = _f64(wl.scene_random_soup(40, seed=6, extent=0.5, scale_lo=0.1, scale_hi=0.3, color_dim=48))
    gb = random_gbuffer(rng, 24, eye=(0.0, 0.0, 3.0))
    env = wl.envmap_hdr(2, 32, 16, sun_gain=30.0, sun_width=0.05)
    alloc = (4, 2, 2)
    wc = rng.normal(size=(24, 3)); wv = rng.normal(size=24); wi = rng.normal(size=(24, 3))

    def loss(s):
        r = oracle.shade_pixels(s, gb, env, *alloc, seed=123)
        return float(np.sum(wc * r["color"]) + np.sum(wv * r["vis"]) + np.sum(wi * r["ind"])), None

    grads = oracle.backward_pixels(sc, gb, env, *alloc, seed=123, dL_dcolor=wc, dL_dvis=wv, dL_dind=wi)
    _fd_check(sc, loss, grads, rng, n_params=30)


def test_opacity_gradient_closed_form():
    # d o_rt / d a_k = T_final / (1 - a_k); with G = 1, d o_rt / d o_k is the same.
    sc = scene([dict(mu=(0, 0, 0), opacity=0.3), dict(mu=(0, 0, 1), opacity=0.6), dict(mu=(0, 0, 2), opacity=0.5)])
    o = np.array([[0, 0, -1]], np.float32); d = np.array([[0, 0, 1]], np.float32)
    g = oracle.backward_rays(sc, o, d, np.zeros((1, 3)), np.ones(1))
    a = sc.opacity.astype(np.float64)
    Tf = np.prod(1 - a)
    np.testing.assert_allclose(g["opacity"], Tf / (1 - a), rtol=1e-12)
    # colour gradient of c_rt is T_k a_k
    g = oracle.backward_rays(sc, o, d, np.ones((1, 3)), np.zeros(1))
    T = np.array([1, 1 - a[0], (1 - a[0]) * (1 - a[1])])
    np.testing.assert_allclose(g["color"][:, 0], T * a, rtol=1e-12)


def test_clamped_alpha_has_no_opacity_gradient():
    sc = scene([dict(mu=(0, 0, 0), opacity=1.0)])
    g = oracle.backward_rays(sc, np.array([[0, 0, -1]], np.float32), np.array([[0, 0, 1]], np.float32),
                             np.ones((1, 3)), np.ones(1))
    assert g["opacity"][0] == 0 and np.all(g["mu"] == 0)
