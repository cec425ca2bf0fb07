"""Pins of the oracle's relighting query (Sec. III-E, Eq. 14-15): Trace_attr against
hand-built surfel stacks, the prefiltered map E against closed-form integrals, the
split-sum BRDF table against its mirror limit and an independent quadrature of the
specular lobe, and the relit estimate against the training estimate where they coincide."""
import math

import numpy as np
import pytest

import oracle
from tests._handmade import Q_NZ, gbuffer, random_gbuffer, scene
from paper_2607_22780_b300 import workloads as wl


def _dirs(H, W):
    th = np.pi * (np.arange(H) + 0.5) / H
    ph = 2 * np.pi * (np.arange(W) + 0.5) / W
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.sin(P), np.cos(T), np.sin(T) * np.cos(P)], -1)


def test_trace_attr_single_and_stacked_surfels():
    o = np.array([[0.0, 0.0, -1.0]], np.float32); d = np.array([[0.0, 0.0, 1.0]], np.float32)
    one = scene([dict(mu=(0, 0, 0), opacity=0.7, albedo=(0.2, 0.4, 0.6), rough=0.3, metal=1.0)])
    r = oracle.trace_attr(one, o, d)
    assert r["V"][0] == pytest.approx(1 - float(np.float32(0.7)), abs=1e-12)
    np.testing.assert_allclose(r["albedo"][0], np.float32([0.2, 0.4, 0.6]), atol=1e-7)
    assert r["rough"][0] == pytest.approx(0.3, abs=1e-7) and r["metal"][0] == 1.0
    np.testing.assert_allclose(r["normal"][0], (0, 0, -1), atol=1e-12)   # turned towards the origin
    two = scene([dict(mu=(0, 0, 0), opacity=0.5, albedo=(1, 0, 0), rough=0.2, quat=Q_NZ),
                 dict(mu=(0, 0, 0.5), opacity=0.6, albedo=(0, 0, 1), rough=0.8)])
    r = oracle.trace_attr(two, o, d)
    w1, w2 = 0.5, 0.5 * float(np.float32(0.6))
    assert r["V"][0] == pytest.approx(0.5 * (1 - float(np.float32(0.6))), abs=1e-12)
    np.testing.assert_allclose(r["albedo"][0], [w1 / (w1 + w2), 0, w2 / (w1 + w2)], atol=1e-12)
    assert r["rough"][0] == pytest.approx((w1 * float(np.float32(0.2)) + w2 * float(np.float32(0.8))) / (w1 + w2), abs=1e-12)
    miss = oracle.trace_attr(one, o, -d)
    assert miss["V"][0] == 1.0 and not miss["albedo"].any() and not miss["normal"].any()


def test_trace_attr_visibility_is_one_minus_opacity_of_trace():
    sc = wl.scene_random_soup(300, seed=5, extent=0.6, scale_lo=0.05, scale_hi=0.2)
    rng = np.random.default_rng(6)
    o = rng.uniform(-1.5, 1.5, (500, 3)).astype(np.float32)
    d = rng.normal(size=(500, 3)); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    a = oracle.trace_attr(sc, o, d)
    t = oracle.trace_rays(sc, o, d)
    np.testing.assert_allclose(a["V"], 1 - t["opacity"], atol=1e-12)
    hit = a["V"] < 1
    assert hit.sum() > 50
    np.testing.assert_allclose(np.linalg.norm(a["normal"][hit], axis=1), 1, atol=1e-12)
    assert np.all(np.einsum("ij,ij->i", a["normal"][hit], d[hit]) <= 1e-12)   # faces the ray origin


def test_prefilter_of_a_constant_map():
    pre = oracle.env_prefilter(wl.envmap_constant(2.0, 64, 32))
    np.testing.assert_allclose(pre["diff"], 2.0, rtol=2e-3)   # (1/pi) int cos = 1, texel quadrature
    np.testing.assert_allclose(pre["spec"], 2.0, rtol=1e-13)  # normalised lobe: exact


def test_diffuse_grid_of_a_cosine_sky_closed_form():
    # L(w) = max(0, w_y): (1/pi) int max(0, y.w) max(0, n.w) dw = (2/(3 pi)) ((pi - g) cos g + sin g)
    H, W = 128, 256
    d = _dirs(H, W)
    env = np.repeat(np.maximum(d[..., 1:2], 0.0), 3, axis=2).astype(np.float32)
    pre = oracle.env_prefilter(env)
    n = _dirs(oracle.DIFF_H, oracle.DIFF_W)
    g = np.arccos(np.clip(n[..., 1], -1, 1))
    ref = 2 / (3 * np.pi) * ((np.pi - g) * np.cos(g) + np.sin(g))
    np.testing.assert_allclose(pre["diff"][..., 0], ref, atol=2e-3)
    # a narrow specular lobe (r = 0.2) of a smooth map stays close to the map itself
    R = _dirs(oracle.SPEC_H, oracle.SPEC_W)
    assert np.abs(pre["spec"][0, ..., 1] - np.maximum(R[..., 1], 0)).max() < 0.03


def test_brdf_table_mirror_limit_and_energy():
    pre = oracle.env_prefilter(wl.envmap_constant(1.0, 16, 8))
    lut = pre["lut"]
    nv = (np.arange(oracle.LUT_N) + 0.5) / oracle.LUT_N
    # r = 1/64: a near mirror, G ~ 1, so A + B ~ 1 and B ~ (1 - nv)^5
    np.testing.assert_allclose(lut[:, 0, 1], (1 - nv) ** 5, atol=2e-3)
    np.testing.assert_allclose(lut[:, 0].sum(-1), 1.0, atol=1e-2)
    assert np.all(lut.sum(-1) <= 1 + 1e-12) and np.all(lut >= 0)


@pytest.mark.parametrize("i,j", [(8, 20), (20, 28), (28, 14), (4, 31)])
def test_brdf_table_against_lobe_quadrature(i, j):
    # A + B = directional albedo of the specular lobe with F = 1 (metal, white):
    # int f(v, l) (n.l) dl by a uniform (theta, phi) grid of l, with f from the oracle's BRDF
    pre = oracle.env_prefilter(wl.envmap_constant(1.0, 16, 8))
    nv = (i + 0.5) / oracle.LUT_N
    r = (j + 0.5) / oracle.LUT_N
    v = np.array([math.sqrt(1 - nv * nv), 0.0, nv])
    nt, nphi = 200, 400
    th = (np.arange(nt) + 0.5) / nt * (np.pi / 2)
    ph = (np.arange(nphi) + 0.5) / nphi * 2 * np.pi
    acc = 0.0
    for k, t in enumerate(th):
        ls = np.stack([np.sin(t) * np.cos(ph), np.sin(t) * np.sin(ph), np.full(nphi, np.cos(t))], -1)
        f = np.array([oracle.brdf(v, l, (0, 0, 1.0), (1, 1, 1), r, 1.0)[0] for l in ls])
        acc += (f * np.cos(t)).sum() * np.sin(t) * (np.pi / 2 / nt) * (2 * np.pi / nphi)
    assert pre["lut"][i, j].sum() == pytest.approx(acc, rel=1e-3, abs=2e-4)


def test_splitsum_under_a_constant_map():
    # E_spec = L exactly and E_diff = L (to quadrature) under a constant map L, so
    # white metal (F0 = 1, no diffuse) gives L (A + B), and the dielectric/metal difference
    # of a white surface is L (1 + 0.04 A + B) - L (A + B) = L (1 - 0.96 A)
    L = 1.5
    pre = oracle.env_prefilter(wl.envmap_constant(L, 64, 32))
    rng = np.random.default_rng(3)
    n = rng.normal(size=(20, 3)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    v = n + 0.5 * rng.normal(size=(20, 3)); v /= np.linalg.norm(v, axis=1, keepdims=True)
    back = np.einsum("ij,ij->i", n, v) < 0.05
    v[back] = n[back]
    r = rng.uniform(0.05, 1, 20)
    metal = oracle.splitsum(pre, np.ones((20, 3)), r, np.ones(20), n, v)[:, 0]
    diel = oracle.splitsum(pre, np.ones((20, 3)), r, np.zeros(20), n, v)[:, 0]
    black_diel = oracle.splitsum(pre, np.zeros((20, 3)), r, np.zeros(20), n, v)[:, 0]   # L (0.04 A + B)
    AB = metal / L
    A = (AB - black_diel / L) / 0.96
    assert np.all(AB > 0.2) and np.all(AB <= 1 + 1e-12) and np.all(A >= 0)
    np.testing.assert_allclose(diel - metal, L * (1 - 0.96 * A), atol=2e-3 * L)   # E_diff = L to 2e-3


def test_relight_without_occluders_equals_training_estimate():
    # no surfels: V_r = 1 for every sample, so Eq. 15 reduces to V L_new and the relit
    # estimate equals the training estimate under the same map and samples
    rng = np.random.default_rng(4)
    gb = random_gbuffer(rng, 48, eye=(0.0, 0.0, 3.0))
    env = wl.envmap_hdr(9, 64, 32)
    empty = scene([])
    pre = oracle.env_prefilter(env)
    a = oracle.shade_relight(empty, gb, env, pre, 8, 4, 4, seed=3)
    b = oracle.shade_pixels(empty, gb, env, 8, 4, 4, seed=3)
    np.testing.assert_array_equal(a["color"], b["color"])
    np.testing.assert_array_equal(a["vis"], b["vis"])
    assert not a["ind"].any()


def test_relight_behind_an_opaque_sheet():
    # a huge sheet of opacity 1 (alpha clamped at 0.99) above a Lambert point: V_r = 0.01
    # for every upward sample, so vis = 0.01 exactly and ind = 0.99 SplitSum of the sheet
    sheet = scene([dict(mu=(0, 0, 1.0), scale=(1e3, 1e3), opacity=1.0, albedo=(0.8, 0.8, 0.8), rough=1.0,
                        metal=0.0)])
    gb = gbuffer([[0, 0, 0]], [[0, 0, 1]], [[0.5, 0.5, 0.5]], [1.0], [0.0], eye=(0, 0, 5))
    env = wl.envmap_constant(1.0, 64, 32)
    pre = oracle.env_prefilter(env)
    r = oracle.shade_relight(sheet, gb, env, pre, 16, 0, 0, seed=1, brdf=0)
    assert r["vis"][0] == pytest.approx(0.01 * (1 - 0), abs=1e-6) or r["flags"][0]
    # each sample's indirect is 0.99 (0.8 E_diff(-z) + E_spec (0.04 A + B)) with E ~ 1
    assert 0.99 * 0.8 < r["ind"][0, 0] < 0.99 * 1.0


def test_lookups_are_continuous_at_the_poles():
    # phi is meaningless at the poles: directions 1e-7 rad off +y (and -y) at different phi
    # must read the same value (the lookups fade to the pole-row mean inside the polar caps)
    pre = oracle.env_prefilter(wl.envmap_hdr(3, 64, 32))
    for sgn in (1.0, -1.0):
        phis = np.linspace(0, 2 * np.pi, 17)[:-1]
        e = 1e-7
        n = np.stack([e * np.sin(phis), np.full(16, sgn), e * np.cos(phis)], -1)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        for r in (0.05, 0.3, 0.9):
            out = oracle.splitsum(pre, np.ones((16, 3)), np.full(16, r), np.zeros(16), n, n)
            assert np.ptp(out, axis=0).max() < 1e-5 * np.abs(out).max(), (sgn, r, np.ptp(out, axis=0))
