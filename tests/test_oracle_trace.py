"""Pins of the oracle's trace (Eq. 7 and Eq. 8) against closed forms and invariants."""
import math
import os

import numpy as np
import pytest

import oracle
from tests._handmade import Q_NX, Q_NY, Q_NZ, scene
from paper_2607_22780_b300 import workloads as wl

AMIN = 1.0 / 255.0


def _one(sc, o, d, **kw):
    r = oracle.trace_rays(sc, np.array([o], np.float32), np.array([d], np.float32), **kw)
    return {k: v[0] for k, v in r.items()}


def test_head_on_centre_alpha_equals_opacity():
    # Eq. 7: at the centre u = v = 0, so G = 1 and alpha = o.
    sc = scene([dict(mu=(0, 0, 0), quat=Q_NZ, scale=(0.1, 0.2), opacity=0.7, color=(0.2, 0.5, 0.9))])
    r = _one(sc, (0, 0, -2), (0, 0, 1))
    assert r["nhits"] == 1 and r["hits"][0] == 0
    assert r["opacity"] == pytest.approx(0.7, abs=1e-7)
    np.testing.assert_allclose(r["rgb"], 0.7 * np.array([0.2, 0.5, 0.9], np.float32), atol=1e-7)
    assert r["T"] == pytest.approx(1 - 0.7, abs=1e-7)


@pytest.mark.parametrize("x0,y0", [(0.05, 0.0), (0.0, 0.3), (0.12, -0.25), (-0.2, 0.1)])
def test_off_centre_gaussian(x0, y0):
    # Ray parallel to the normal at (x0, y0): u = x0/s_u, v = y0/s_v.
    su, sv, o = 0.1, 0.2, 0.6
    sc = scene([dict(mu=(0, 0, 0), quat=Q_NZ, scale=(su, sv), opacity=o, color=(1, 1, 1))])
    r = _one(sc, (x0, y0, -1), (0, 0, 1))
    u, v = np.float32(x0) / np.float32(su), np.float32(y0) / np.float32(sv)
    a = np.float32(o) * math.exp(-0.5 * (float(u) ** 2 + float(v) ** 2))
    if a >= AMIN:
        assert r["opacity"] == pytest.approx(a, rel=1e-6)
    else:
        assert r["nhits"] == 0 and r["opacity"] == 0


def test_oblique_ray_local_coordinates():
    # Surfel with normal +x; oblique ray from (-1, y, z) towards +x hits the plane x=0.
    su, sv, o = 0.3, 0.15, 0.8
    sc = scene([dict(mu=(0, 0, 0), quat=Q_NX, scale=(su, sv), opacity=o, color=(1, 0, 0))])
    d = np.array([1.0, 0.1, -0.05]); d /= np.linalg.norm(d)
    org = np.array([-1.0, 0.02, 0.03])
    r = _one(sc, org, d)
    d32 = d.astype(np.float32).astype(np.float64); o32 = org.astype(np.float32).astype(np.float64)
    tau = -o32[0] / d32[0]
    p = o32 + tau * d32
    # frame of Q_NX: t_u = R e_x = -z, t_v = R e_y = +y, n = +x
    u, v = -p[2] / su, p[1] / sv
    a = o * math.exp(-0.5 * (u * u + v * v))
    assert r["opacity"] == pytest.approx(a, rel=2e-6)


def test_two_stacked_front_to_back():
    # Eq. 8 by hand: c = a1 c1 + (1 - a1) a2 c2 with the nearer surfel first even if its id is larger.
    c_far, c_near = np.array([0.1, 0.9, 0.3]), np.array([0.8, 0.2, 0.4])
    sc = scene([dict(mu=(0, 0, 1), opacity=0.5, color=c_far),
                dict(mu=(0, 0, 0), opacity=0.6, color=c_near)])
    r = _one(sc, (0, 0, -2), (0, 0, 1))
    a1, a2 = np.float32(0.6), np.float32(0.5)
    exp = a1 * c_near.astype(np.float32) + (1 - a1) * a2 * c_far.astype(np.float32)
    np.testing.assert_allclose(r["rgb"], exp, atol=1e-7)
    assert list(r["hits"][:2]) == [1, 0]
    assert r["opacity"] == pytest.approx(a1 + (1 - a1) * a2, abs=1e-7)


def test_equal_depth_ordered_by_id():
    sc = scene([dict(mu=(0, 0, 0), opacity=0.5, color=(1, 0, 0)),
                dict(mu=(0, 0, 0), opacity=0.5, color=(0, 1, 0))])
    r = _one(sc, (0, 0, -2), (0, 0, 1))
    assert list(r["hits"][:2]) == [0, 1]
    np.testing.assert_allclose(r["rgb"], [0.5, 0.25, 0.0], atol=1e-12)


def test_early_termination_after_T_min():
    # alpha = 0.8 each: T = 0.2^k; 0.2^5 = 3.2e-4 > 1e-4 > 0.2^6 = 6.4e-5, so six hits.
    sc = scene([dict(mu=(0, 0, 0.1 * i), opacity=0.8, color=(1, 1, 1)) for i in range(10)])
    r = _one(sc, (0, 0, -1), (0, 0, 1))
    assert r["nhits"] == 6
    assert list(r["hits"][:6]) == list(range(6))
    assert r["T"] == pytest.approx((1 - float(np.float32(0.8))) ** 6, rel=1e-12)
    assert r["opacity"] + r["T"] == pytest.approx(1.0, abs=1e-14)


def test_alpha_max_clamp():
    sc = scene([dict(mu=(0, 0, 0), opacity=1.0, color=(1, 1, 1))])
    r = _one(sc, (0, 0, -2), (0, 0, 1))
    assert r["opacity"] == pytest.approx(0.99, abs=1e-7)


def test_alpha_min_rejects():
    # o G = 1.05 alpha_min is a hit, 0.95 alpha_min is not.
    o, s = 0.5, 0.1
    for f, hit in ((1.05, True), (0.95, False)):
        u = math.sqrt(2 * math.log(o / (f * AMIN)))
        sc = scene([dict(mu=(0, 0, 0), scale=(s, s), opacity=o)])
        r = _one(sc, (u * s, 0, -1), (0, 0, 1))
        assert (r["nhits"] == 1) == hit


def test_t_min_and_parallel_rays_rejected():
    sc = scene([dict(mu=(0, 0, 0), opacity=0.9)])
    assert _one(sc, (0, 0, -0.005), (0, 0, 1))["nhits"] == 0          # tau < t_min
    assert _one(sc, (0, 0, -0.02), (0, 0, 1))["nhits"] == 1           # tau > t_min
    assert _one(sc, (0, 0, -1), (0, 0, -1))["nhits"] == 0             # behind the origin
    assert _one(sc, (-1, 0, 0), (1, 0, 0))["nhits"] == 0              # in the plane, |n.d| = 0
    assert _one(sc, (0, 0, -1), (0, 0, 1), params=dict(t_max=0.5))["nhits"] == 0


def test_empty_scene():
    sc = scene([])
    r = _one(sc, (0, 0, 0), (0, 1, 0))
    assert r["nhits"] == 0 and r["opacity"] == 0 and np.all(r["rgb"] == 0) and r["T"] == 1


def test_two_sided_surfels():
    sc = scene([dict(mu=(0, 0, 0), opacity=0.7, color=(1, 1, 1))])
    a = _one(sc, (0, 0, -2), (0, 0, 1))
    b = _one(sc, (0, 0, 2), (0, 0, -1))
    assert a["opacity"] == b["opacity"] == pytest.approx(0.7, abs=1e-7)


def test_weights_plus_transmittance_is_one():
    # o_rt = sum T_k a_k = 1 - T_final (Eq. 8).
    sc = wl.scene_random_soup(300, seed=3, extent=0.5)
    rng = np.random.default_rng(0)
    o = rng.uniform(-1.5, 1.5, size=(400, 3))
    d = rng.normal(size=(400, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = oracle.trace_rays(sc, o, d)
    np.testing.assert_allclose(r["opacity"] + r["T"], 1.0, atol=1e-12)
    assert r["nhits"].max() > 3


def test_hits_match_independent_brute_force():
    # Depth order and membership against a vectorised FP64 plane/Gaussian test.
    sc = wl.scene_random_soup(200, seed=5, extent=0.5, scale_lo=0.05, scale_hi=0.2)
    rng = np.random.default_rng(1)
    o = rng.uniform(-1.5, 1.5, size=(200, 3)).astype(np.float32)
    d = rng.normal(size=(200, 3)); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r = oracle.trace_rays(sc, o, d, params=dict(T_min=0.0))
    q = sc.quat.astype(np.float64); q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    tu = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    tv = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    nn = np.cross(tu, tv)
    mu = sc.mu.astype(np.float64)
    bad = 0
    for i in range(200):
        oo, dd = o[i].astype(np.float64), d[i].astype(np.float64)
        nd = nn @ dd
        tau = np.einsum("ij,ij->i", nn, mu - oo) / nd
        p = oo + tau[:, None] * dd - mu
        u = np.einsum("ij,ij->i", p, tu) / sc.scale[:, 0]
        v = np.einsum("ij,ij->i", p, tv) / sc.scale[:, 1]
        a = sc.opacity * np.exp(-0.5 * (u * u + v * v))
        ok = (tau > 0.01) & (np.abs(nd) >= 1e-6) & (a >= AMIN)
        ids = np.nonzero(ok)[0]
        ids = ids[np.argsort(tau[ids], kind="stable")]
        got = r["hits"][i][:r["nhits"][i]]
        if r["flags"][i] == 0:
            k = min(len(ids), 64)
            if list(got[:k]) != list(ids[:k]):
                bad += 1
    assert bad == 0


def test_sh_degree0_colour():
    # color = max(0, C0 sh0 + 0.5) with C0 = 1/(2 sqrt(pi)), independent of direction.
    sh = np.zeros(48, np.float32); sh[0:3] = [0.3, -0.4, -3.0]
    sc = scene([dict(mu=(0, 0, 0), opacity=0.5, color=sh)], color_dim=48)
    for d in ((0, 0, 1), (0.3, 0.4, 0.866)):
        d = np.array(d) / np.linalg.norm(d)
        r = _one(sc, -d * 2, d)
        c0 = 0.5 / math.sqrt(math.pi)
        exp = np.maximum(0, c0 * sh[:3].astype(np.float64) + 0.5) * 0.5
        np.testing.assert_allclose(r["rgb"], exp, atol=1e-6)


def test_sh_basis_orthonormal():
    # Int Y_i Y_j dw = delta_ij by Gauss-Legendre x uniform-phi quadrature (exact for degree <= 6).
    xs, ws = np.polynomial.legendre.leggauss(16)
    nphi = 32
    G = np.zeros((16, 16))
    for ct, wt in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis((st * math.cos(ph), st * math.sin(ph), ct))
            G += wt * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_known_values():
    # At +z only m = 0 terms survive: Y_00, Y_10 = sqrt(3/4pi), Y_20 = 2 sqrt(5/16pi), Y_30 = 2 sqrt(7/16pi).
    Y = oracle.sh_basis((0, 0, 1))
    exp = np.zeros(16)
    exp[0] = math.sqrt(1 / (4 * math.pi)); exp[2] = math.sqrt(3 / (4 * math.pi))
    exp[6] = 2 * math.sqrt(5 / (16 * math.pi)); exp[12] = 2 * math.sqrt(7 / (16 * math.pi))
    np.testing.assert_allclose(Y, exp, atol=1e-15)


def test_normal_from_quat_axes():
    for q, n in ((Q_NZ, (0, 0, 1)), (Q_NY, (0, 1, 0)), (Q_NX, (1, 0, 0))):
        np.testing.assert_allclose(oracle.normal_from_quat(np.array(q, np.float32)), n, atol=1e-6)
    # unnormalised quaternion gives the same normal
    np.testing.assert_allclose(oracle.normal_from_quat(np.array(Q_NY, np.float32) * 3.0), (0, 1, 0), atol=1e-6)
