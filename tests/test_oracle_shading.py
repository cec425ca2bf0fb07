"""Pins of the oracle's MIS shading (Eq. 10-13) and primary G-buffer (Eq. 9)."""
import math

import numpy as np
import pytest

import oracle
from tests._handmade import Q_NZ, gbuffer, random_gbuffer, scene
from paper_2607_22780_b300 import workloads as wl


def test_white_furnace_cosine_lambert_is_exact():
    # Cosine sampling with f = a/pi gives g/q = a L_i per sample; no occluders and
    # constant L give colour = a L, visibility 1, indirect 0 (Eq. 12).
    rng = np.random.default_rng(0)
    gb = random_gbuffer(rng, 64)
    L = 1.75
    r = oracle.shade_pixels(scene([]), gb, wl.envmap_constant(L), 4, 0, 0, seed=9, brdf=0)
    np.testing.assert_allclose(r["color"], gb["albedo"].astype(np.float64) * L, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["vis"], 1.0, atol=0)
    assert np.all(r["ind"] == 0) and np.all(r["flags"] == 0)


def test_uniform_occluder_closed_form():
    # A huge surfel of opacity o above every shading point: every sample sees V = 1-o and
    # L_ind = o c, so colour = a ((1-o) L + o c) exactly for cosine + Lambert.
    o, c, L = 0.6, np.array([0.2, 0.5, 0.7]), 1.25
    sc = scene([dict(mu=(0, 0, 1.0), quat=Q_NZ, scale=(1e6, 1e6), opacity=o, color=c)])
    P = 16
    rng = np.random.default_rng(1)
    pos = np.c_[rng.uniform(-0.3, 0.3, (P, 2)), np.zeros(P)]
    gb = gbuffer(pos, np.tile([0, 0, 1.0], (P, 1)), rng.uniform(0.1, 1, (P, 3)), np.full(P, 0.5),
                 np.zeros(P), eye=(0, 0, 0.5))
    r = oracle.shade_pixels(sc, gb, wl.envmap_constant(L), 8, 0, 0, seed=3, brdf=0)
    o32, c32 = float(np.float32(o)), c.astype(np.float32).astype(np.float64)
    exp = gb["albedo"].astype(np.float64) * ((1 - o32) * L + o32 * c32)
    np.testing.assert_allclose(r["color"], exp, rtol=1e-6)
    np.testing.assert_allclose(r["vis"], 1 - o32, rtol=1e-6)
    np.testing.assert_allclose(r["ind"], np.tile(o32 * c32, (P, 1)), rtol=1e-6)


def _shade_mean(gb, env, alloc, brdf, seed=5):
    r = oracle.shade_pixels(scene([]), gb, env, *alloc, seed=seed, brdf=brdf)
    c = r["color"]
    return c.mean(0), c.std(0) / math.sqrt(c.shape[0])


@pytest.mark.parametrize("alloc", [(128, 64, 64), (0, 0, 256), (0, 256, 0)])
def test_mis_unbiased_lambert(alloc):
    # Balance-heuristic MIS (Eq. 13) under a constant map on an empty scene: E[colour] = a L.
    P = 128
    gb = gbuffer(np.zeros((P, 3)), np.tile([0.3, 0.8, 0.2], (P, 1)), np.tile([0.7, 0.4, 0.2], (P, 1)),
                 np.full(P, 0.4), np.zeros(P), eye=(1.0, 3.0, 0.5))
    m, se = _shade_mean(gb, wl.envmap_constant(2.0), alloc, brdf=0)
    exp = np.array([0.7, 0.4, 0.2], np.float32).astype(np.float64) * 2.0
    assert np.all(np.abs(m - exp) < 5 * se + 1e-9), (m, exp, se)


@pytest.mark.parametrize("rough,metal", [(0.3, 1.0), (0.6, 0.0), (0.15, 1.0)])
def test_mis_matches_quadrature_ggx(rough, metal):
    # E[colour] = L Int f cos dw, with the integral by independent quadrature of the BRDF.
    n = np.array([0.0, 1.0, 0.0]); wo = np.array([0.4, 0.9, 0.1]); wo /= np.linalg.norm(wo)
    alb = np.array([0.9, 0.6, 0.3], np.float32).astype(np.float64)
    nt, nph = 600, 300
    th = (np.arange(nt) + 0.5) * (math.pi / 2) / nt
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    acc = np.zeros(3)
    for t in th:
        st, ct = math.sin(t), math.cos(t)
        for p in ph:
            w = np.array([st * math.sin(p), ct, st * math.cos(p)])
            acc += oracle.brdf(wo, w, n, alb, rough, metal) * ct * st
    R = acc * (math.pi / 2 / nt) * (2 * math.pi / nph)
    P = 256
    eye = wo * 3.0
    gb = gbuffer(np.zeros((P, 3)), np.tile(n, (P, 1)), np.tile(alb, (P, 1)), np.full(P, rough),
                 np.full(P, metal), eye=eye)
    m, se = _shade_mean(gb, wl.envmap_constant(1.0), (64, 32, 32), brdf=1)
    assert np.all(np.abs(m - R) < 5 * se + 2e-3 * R), (m, R, se)


def test_pixel_alone_equals_in_list():
    sc = wl.scene_random_soup(60, seed=2, extent=0.6, scale_lo=0.05, scale_hi=0.2)
    gb = random_gbuffer(np.random.default_rng(3), 40)
    env = wl.envmap_hdr(1, 32, 16)
    full = oracle.shade_pixels(sc, gb, env, 4, 2, 2, seed=77)
    for p in (0, 17, 39):
        one = oracle.shade_pixels(sc, gb, env, 4, 2, 2, seed=77, pixels=[p])
        assert np.array_equal(one["color"][0], full["color"][p])
        assert one["vis"][0] == full["vis"][p]


# ------------------------------------------------------------------ G-buffer

def _cam(eye, W=5, H=5):
    return wl.Camera(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0),
                     tan_half_fovy=math.tan(math.radians(30)), width=W, height=H)


def test_camera_centre_ray_and_unit_directions():
    cam = _cam((0.0, 0.0, 3.0))
    o, d = oracle.camera_ray(cam, 2, 2)
    np.testing.assert_allclose(d, (0, 0, -1), atol=1e-7)
    np.testing.assert_allclose(o, (0, 0, 3))
    oo, dd = oracle.camera_rays(_cam((1.0, 2.0, 3.0), 7, 4))
    np.testing.assert_allclose(np.linalg.norm(dd, axis=1), 1, atol=2e-7)
    # top-left pixel looks up and to the left of the forward axis
    o0, d0 = oracle.camera_ray(cam, 0, 0)
    assert d0[0] < 0 and d0[1] > 0


def test_gbuffer_single_surfel():
    alb = (0.2, 0.4, 0.6)
    for q, flip in ((Q_NZ, False), ((0.0, 1.0, 0.0, 0.0), True)):
        sc = scene([dict(mu=(0, 0, 0), quat=q, scale=(0.5, 0.5), opacity=0.7, albedo=alb,
                         rough=0.3, metal=1.0)])
        g = oracle.gbuffer(sc, _cam((0.0, 0.0, 3.0)))
        c = 2 * 5 + 2
        assert g["valid"][c] == 1
        assert g["depth"][c] == pytest.approx(3.0, abs=1e-6)
        np.testing.assert_allclose(g["pos"][c], 0, atol=1e-6)
        np.testing.assert_allclose(g["normal"][c], (0, 0, 1), atol=1e-7)
        np.testing.assert_allclose(g["albedo"][c], np.array(alb, np.float32), atol=1e-7)
        assert g["rough"][c] == pytest.approx(0.3, abs=1e-7) and g["metal"][c] == 1.0
        assert g["alpha"][c] == pytest.approx(0.7, abs=1e-7)


def test_gbuffer_two_layers_normalised_weights():
    # w1 = a1, w2 = (1-a1) a2; normalised: 0.6/0.8 and 0.2/0.8.
    sc = scene([dict(mu=(0, 0, 0), scale=(1, 1), opacity=0.5, albedo=(0, 0, 1), rough=0.2),
                dict(mu=(0, 0, 0.5), scale=(1, 1), opacity=0.6, albedo=(1, 0, 0), rough=0.8)])
    g = oracle.gbuffer(sc, _cam((0.0, 0.0, 3.0)))
    c = 12
    a1, a2 = float(np.float32(0.6)), float(np.float32(0.5))
    w1, w2 = a1, (1 - a1) * a2
    s = w1 + w2
    assert g["alpha"][c] == pytest.approx(s, abs=1e-12)
    np.testing.assert_allclose(g["albedo"][c], [w1 / s, 0, w2 / s], atol=1e-12)
    assert g["depth"][c] == pytest.approx((w1 * 2.5 + w2 * 3.0) / s, abs=1e-6)
    assert g["rough"][c] == pytest.approx((w1 * float(np.float32(0.8)) + w2 * float(np.float32(0.2))) / s, abs=1e-7)


def test_gbuffer_miss_is_invalid():
    sc = scene([dict(mu=(5, 5, 0), scale=(0.1, 0.1), opacity=0.9)])
    g = oracle.gbuffer(sc, _cam((0.0, 0.0, 3.0)))
    assert g["valid"].sum() == 0 and np.all(g["alpha"] == 0)


def test_gbuffer_pixel_subset_rows():
    # traced pixels are independent: the subset's rows are the full image's rows of those pixels
    sc = wl.scene_objects(20000, seed=4)
    cam = wl.camera_orbit(4, 20, 16, 3.0)
    full = oracle.gbuffer(sc, cam)
    v = np.nonzero(full["valid"])[0]
    pix = np.array([319, 0, v[0], 160, v[-1], v[0], v[len(v) // 2]], np.int32)
    sub = oracle.gbuffer(sc, cam, pixels=pix)
    for k in ("pos", "normal", "albedo", "rough", "metal", "alpha", "depth", "valid", "flags"):
        assert np.array_equal(sub[k], full[k][pix]), k
    assert full["valid"][pix].sum() > 0
    with pytest.raises(ValueError):
        oracle.gbuffer(sc, cam, pixels=np.array([320], np.int32))
