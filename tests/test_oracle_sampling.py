"""Pins of the oracle's random numbers, proposals, densities and BRDF (Sec. III-D, Eq. 4-5, Eq. 13)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2607_22780_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]
        n += 1
    assert n == 3


def test_sincos2pi_accuracy():
    t = np.concatenate([np.linspace(0, 1, 4097), np.random.default_rng(0).uniform(0, 1, 4000)])
    err = 0.0
    for x in t.astype(np.float32):
        s, c = oracle.sincos2pi(x)
        err = max(err, abs(s - math.sin(2 * math.pi * float(x))), abs(c - math.cos(2 * math.pi * float(x))))
    assert err < 3e-7


def test_atan2_accuracy():
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(5000, 2)).astype(np.float32)
    pts = np.concatenate([pts, [[0, 1], [1, 0], [0, -1], [-1, 0], [1, 1], [-1, -1], [1e-8, 1]]]).astype(np.float32)
    err = max(abs(oracle.atan2f(y, x) - math.atan2(float(y), float(x))) for y, x in pts)
    assert err < 4e-7


def test_texel_of_matches_angles_away_from_edges():
    rng = np.random.default_rng(2)
    W, H = 64, 32
    d = rng.normal(size=(3000, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    for v in d.astype(np.float32):
        th = math.acos(max(-1.0, min(1.0, float(v[1]))))
        ph = math.atan2(float(v[0]), float(v[2])) % (2 * math.pi)
        rf, cf = th / math.pi * H, ph / (2 * math.pi) * W
        if min(abs(rf - round(rf)), abs(cf - round(cf))) < 1e-4:
            continue
        assert oracle.texel_of(v, W, H) == (min(int(rf), H - 1), min(int(cf), W - 1))


def test_env_tables_are_cdfs():
    env = wl.envmap_hdr(3, 64, 32)
    marg, cond = oracle.env_tables_f32(env)
    assert marg[0] == 0 and marg[-1] == 1.0 and np.all(np.diff(marg) >= 0)
    assert np.all(cond[:, 0] == 0) and np.all(cond[:, -1] == 1.0) and np.all(np.diff(cond, axis=1) >= 0)
    lum = env @ np.array([0.2126, 0.7152, 0.0722])
    np.testing.assert_allclose(np.diff(marg), lum.sum(1) / lum.sum(), rtol=1e-4, atol=1e-7)


def _sphere_grid(nt=200, nph=400):
    ct = np.cos((np.arange(nt) + 0.5) * math.pi / nt)
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = np.stack([np.sin(T) * np.sin(P), np.cos(T), np.sin(T) * np.cos(P)], -1).reshape(-1, 3)
    dw = (np.sin(T) * (math.pi / nt) * (2 * math.pi / nph)).reshape(-1)
    return dirs, dw


@pytest.mark.parametrize("rough", [0.3, 0.6, 1.0])
def test_ggx_pdf_integrates_to_one(rough):
    # The reflected visible-normal density integrates to 1 over the whole sphere.
    n = np.array([0.0, 1.0, 0.0]); wo = np.array([0.3, 0.8, 0.1]); wo /= np.linalg.norm(wo)
    dirs, dw = _sphere_grid(400, 800)
    tot = sum(oracle.pdf_ggx(wo, n, rough, w) * a for w, a in zip(dirs, dw))
    assert tot == pytest.approx(1.0, abs=3e-3)


def test_env_pdf_integrates_to_one():
    env = wl.envmap_hdr(5, 32, 16)
    dirs, dw = _sphere_grid(160, 320)
    tot = sum(oracle.pdf_env(env, w) * a for w, a in zip(dirs, dw))
    assert tot == pytest.approx(1.0, abs=1e-3)


def _chi2(obs, exp):
    m = exp >= 5
    return float(np.sum((obs[m] - exp[m]) ** 2 / exp[m])), int(m.sum()) - 1


def _chi2_ok(stat, dof):
    # mean + 5 sigma of a chi-square with dof degrees of freedom
    return stat < dof + 5 * math.sqrt(2 * dof)


def test_cosine_samples_histogram():
    n = np.array([0.2, 0.9, -0.3]); n /= np.linalg.norm(n)
    env = wl.envmap_constant()
    w, ok = oracle.sample_many(0, env, n, n, 0.5, 11, 40000)
    assert ok.all()
    cos = w.astype(np.float64) @ n
    assert cos.min() >= 0
    # cos^2 theta is uniform under cosine-weighted sampling
    h, _ = np.histogram(cos ** 2, bins=20, range=(0, 1))
    s, dof = _chi2(h.astype(float), np.full(20, len(w) / 20))
    assert _chi2_ok(s, dof)


@pytest.mark.parametrize("rough", [0.25, 0.7])
def test_ggx_samples_histogram(rough):
    n = np.array([0.0, 0.0, 1.0]); wo = np.array([0.5, 0.2, 0.8]); wo /= np.linalg.norm(wo)
    env = wl.envmap_constant()
    N = 60000
    w, ok = oracle.sample_many(1, env, n, wo, rough, 7, N)
    assert ok.all()
    w = w.astype(np.float64); w /= np.linalg.norm(w, axis=1, keepdims=True)
    nt, nph = 12, 16
    th = np.arccos(np.clip(w[:, 2], -1, 1)); ph = np.arctan2(w[:, 1], w[:, 0]) % (2 * math.pi)
    obs, _, _ = np.histogram2d(th, ph, bins=[nt, nph], range=[[0, math.pi], [0, 2 * math.pi]])
    exp = np.zeros((nt, nph))
    sub = 6
    for i in range(nt):
        for j in range(nph):
            acc = 0.0
            for a in range(sub):
                for b in range(sub):
                    t = (i + (a + 0.5) / sub) * math.pi / nt
                    p = (j + (b + 0.5) / sub) * 2 * math.pi / nph
                    d = (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))
                    acc += oracle.pdf_ggx(wo, n, rough, d) * math.sin(t)
            exp[i, j] = acc * (math.pi / nt / sub) * (2 * math.pi / nph / sub) * N
    s, dof = _chi2(obs.ravel(), exp.ravel())
    assert _chi2_ok(s, dof), (s, dof)


def test_env_samples_histogram():
    env = wl.envmap_hdr(9, 16, 8, sun_gain=20.0, sun_width=0.05)
    N = 50000
    w, ok = oracle.sample_many(2, env, [0, 1, 0], [0, 1, 0], 0.5, 5, N)
    H, W = env.shape[:2]
    obs = np.zeros((H, W))
    for v in w:
        r, c = oracle.texel_of(v, W, H)
        obs[r, c] += 1
    lum = env.astype(np.float64) @ np.array([0.2126, 0.7152, 0.0722])
    s, dof = _chi2(obs.ravel(), (lum / lum.sum() * N).ravel())
    assert _chi2_ok(s, dof)


def test_fresnel_f0_at_normal_incidence():
    # w_i = w_o = n: h = n, D = 1/(pi a^2), G1 = 1, F = F0, so f_s = F0 / (4 pi a^2).
    n = np.array([0.0, 0.0, 1.0]); alb = np.array([0.9, 0.5, 0.1])
    r = 0.5; a = r * r
    for m in (0.0, 1.0):
        f = oracle.brdf(n, n, n, alb, r, m)
        fd = (1 - m) * alb / math.pi
        F0 = 0.04 * (1 - m) + m * alb
        np.testing.assert_allclose(f - fd, F0 / (4 * math.pi * a * a), rtol=1e-12)


def test_brdf_reciprocity_and_energy():
    rng = np.random.default_rng(4)
    n = np.array([0.0, 0.0, 1.0])
    for _ in range(50):
        a, b = rng.normal(size=3), rng.normal(size=3)
        a[2], b[2] = abs(a[2]), abs(b[2])
        a /= np.linalg.norm(a); b /= np.linalg.norm(b)
        alb = rng.uniform(0, 1, 3); r = rng.uniform(0.05, 1); m = rng.uniform()
        np.testing.assert_allclose(oracle.brdf(a, b, n, alb, r, m), oracle.brdf(b, a, n, alb, r, m), rtol=1e-12)
    # white furnace of a white metal: directional albedo <= 1
    dirs, dw = _sphere_grid(200, 200)
    up = dirs[:, 1] > 0
    nn = np.array([0.0, 1.0, 0.0]); wo = np.array([0.0, 1.0, 0.0])
    alb = sum(oracle.brdf(wo, w, nn, np.ones(3), 0.5, 1.0)[0] * w[1] * a for w, a in zip(dirs[up], dw[up]))
    assert 0.8 < alb <= 1.0


def test_ggx_D_normalised():
    # Int D(h) (h.n) dh = 1 over the hemisphere, for the GGX D used by the BRDF (via pdf_ggx at w_o = n:
    # p(w_i) = D(h) (h.n) / (4 (w_o.h)) with h.n = w_o.h, so Int p dw = Int D (h.n) dh).
    n = np.array([0.0, 1.0, 0.0])
    dirs, dw = _sphere_grid(400, 200)
    for r in (0.4, 0.8):
        tot = sum(oracle.pdf_ggx(n, n, r, w) * a for w, a in zip(dirs, dw))
        assert tot == pytest.approx(1.0, abs=3e-3)
