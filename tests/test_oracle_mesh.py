"""Pins of the oracle's mesh backend of Eq. 14 (Sec. III-E): hand-built triangles with
closed-form hits and barycentric attributes, an independent vectorised brute force of the
closest hit on a tessellated scene, and the relit estimate's reductions."""
import numpy as np
import pytest

import oracle
from tests._handmade import gbuffer, icosphere, random_gbuffer, scene
from paper_2607_22780_b300 import workloads as wl


def _mesh(pos, tri, normal=None, albedo=None, rough=None, metal=None):
    pos = np.asarray(pos, np.float32); tri = np.asarray(tri, np.int32)
    V = len(pos)
    return wl.Mesh(pos=pos, tri=tri,
                   normal=np.asarray(normal if normal is not None else np.tile([0, 0, 1.0], (V, 1)), np.float32),
                   albedo=np.asarray(albedo if albedo is not None else np.full((V, 3), 0.5), np.float32),
                   rough=np.asarray(rough if rough is not None else np.full(V, 0.5), np.float32),
                   metal=np.asarray(metal if metal is not None else np.zeros(V), np.float32))


def test_single_triangle_barycentric_attributes():
    m = _mesh([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]],
              albedo=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], rough=[0.2, 0.6, 1.0], metal=[0, 1, 0])
    o = np.array([[0.25, 0.5, -1.0]], np.float32); d = np.array([[0, 0, 1.0]], np.float32)
    r = oracle.mesh_trace_attr(m, o, d)
    # barycentrics (1 - u - v, u, v) = (0.25, 0.25, 0.5) at (x, y) = (u, v)
    assert r["V"][0] == 0 and r["flags"][0] == 0
    np.testing.assert_allclose(r["albedo"][0], [0.25, 0.25, 0.5], atol=1e-12)
    assert r["rough"][0] == pytest.approx(0.25 * 0.2 + 0.25 * 0.6 + 0.5 * 1.0, abs=1e-7)
    assert r["metal"][0] == pytest.approx(0.25, abs=1e-12)
    np.testing.assert_allclose(r["normal"][0], [0, 0, -1], atol=1e-12)   # turned towards the origin
    miss = oracle.mesh_trace_attr(m, np.array([[0.8, 0.8, -1.0]], np.float32), d)
    assert miss["V"][0] == 1 and not miss["albedo"].any()
    # on the hypotenuse: an edge hit, weights (0, 1/2, 1/2)
    edge = oracle.mesh_trace_attr(m, np.array([[0.5, 0.5, -1.0]], np.float32), d)
    assert edge["V"][0] == 0
    np.testing.assert_allclose(edge["albedo"][0], [0, 0.5, 0.5], atol=1e-12)


def test_nearest_of_stacked_triangles_and_t_range():
    tri = [[0, 1, 2], [3, 4, 5]]
    pos = [[-1, -1, 2], [3, -1, 2], [-1, 3, 2], [-1, -1, 1], [3, -1, 1], [-1, 3, 1]]
    m = _mesh(pos, tri, albedo=[[1, 0, 0]] * 3 + [[0, 1, 0]] * 3)
    o = np.array([[0, 0, 0.0]], np.float32); d = np.array([[0, 0, 1.0]], np.float32)
    assert oracle.mesh_trace_attr(m, o, d)["albedo"][0, 1] == 1.0        # z = 1 first
    far = oracle.mesh_trace_attr(m, np.array([[0, 0, 1.5]], np.float32), d)
    assert far["albedo"][0, 0] == 1.0                                     # behind: only z = 2
    p = dict(alpha_min=1 / 255, alpha_max=0.99, t_min=0.01, t_max=0.9, T_min=1e-4, eps_nd=1e-6, k=16)
    assert oracle.mesh_trace_attr(m, o, d, params=p)["V"][0] == 1          # both beyond t_max


def _brute_hits(m, o, d, tmin=0.01):
    """FP64 closest hit per ray by Cramer's rule over every triangle, and whether the ray is
    clear of FP32 ambiguity: no triangle within 1e-4 (barycentric) of its boundary in front
    of the origin, and the two nearest hits more than 1e-5 (relative) apart."""
    p = m.pos.astype(np.float64); t = m.tri
    v0, v1, v2 = p[t[:, 0]], p[t[:, 1]], p[t[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    best = np.full(len(o), np.inf); arg = np.full(len(o), -1); clear = np.ones(len(o), bool)
    for i in range(len(o)):
        di = d[i].astype(np.float64); oi = o[i].astype(np.float64)
        # solve oi + t di = v0 + u e1 + v e2 by Cramer's rule per triangle
        M = np.stack([-np.broadcast_to(di, e1.shape), e1, e2], -1)
        det = np.linalg.det(M)
        ok = np.abs(det) > 1e-14
        rhs = oi - v0
        sol = np.full((len(t), 3), np.nan)
        sol[ok] = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
        tt, u, v = sol[:, 0], sol[:, 1], sol[:, 2]
        margin = np.minimum(np.minimum(u, v), 1 - u - v)
        front = ok & (tt > tmin)
        hit = front & (margin >= 0)
        if (front & (np.abs(margin) < 1e-4)).any():
            clear[i] = False
        if hit.any():
            ts = np.sort(tt[hit])
            j = np.argmin(np.where(hit, tt, np.inf))
            best[i], arg[i] = tt[j], j
            if len(ts) > 1 and ts[1] - ts[0] <= 1e-5 * ts[0]:
                clear[i] = False
    return best, arg, clear


def test_closest_hit_against_independent_brute_force():
    m = wl.mesh_objects(7, res=12)
    rng = np.random.default_rng(1)
    o = rng.uniform(-2.5, 2.5, (150, 3)).astype(np.float32)
    tg = rng.uniform(-1.0, 0.5, (150, 3))
    d = tg - o; d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r = oracle.mesh_trace_attr(m, o, d)
    assert not r["flags"].any()
    best, arg, keep = _brute_hits(m, o, d)
    assert keep.mean() > 0.9 and (best[keep] < np.inf).sum() > 50
    np.testing.assert_array_equal(r["V"][keep] == 0, best[keep] < np.inf)
    hit = keep & (best < np.inf)
    w = np.zeros((hit.sum(), 3))
    # attributes of the brute-force triangle at its barycentrics
    tri = m.tri[arg[hit]]
    p = m.pos.astype(np.float64)
    x = o[hit] + best[hit, None] * d[hit]
    v0, v1, v2 = p[tri[:, 0]], p[tri[:, 1]], p[tri[:, 2]]
    tot = np.linalg.norm(np.cross(v1 - v0, v2 - v0), axis=1)
    w[:, 0] = np.linalg.norm(np.cross(v1 - x, v2 - x), axis=1) / tot
    w[:, 1] = np.linalg.norm(np.cross(v2 - x, v0 - x), axis=1) / tot
    w[:, 2] = np.linalg.norm(np.cross(v0 - x, v1 - x), axis=1) / tot
    alb = (w[..., None] * m.albedo[tri]).sum(1)
    np.testing.assert_allclose(r["albedo"][hit], alb, atol=1e-6)


def test_closed_mesh_blocks_every_ray_from_inside():
    # watertightness: seen from inside a closed mesh every ray hits, including rays aimed
    # exactly at shared vertices and edge midpoints, where a test that is not watertight
    # lets rays through the cracks between neighbours
    v, f = icosphere(3)
    m = _mesh(1.7 * v + [0.2, -0.1, 0.3], f, normal=v)
    rng = np.random.default_rng(9)
    c = np.array([0.2, -0.1, 0.3]) + rng.uniform(-0.3, 0.3, (4, 3))
    tgt = np.concatenate([m.pos, 0.5 * (m.pos[f[:, 0]] + m.pos[f[:, 1]]), rng.normal(size=(500, 3))])
    o = np.repeat(c, len(tgt), 0).astype(np.float32)
    dd = np.tile(tgt, (len(c), 1)) - np.repeat(c, len(tgt), 0)
    dd[len(tgt) - 500:len(tgt)] = tgt[-500:]
    d = (dd / np.linalg.norm(dd, axis=1, keepdims=True)).astype(np.float32)
    r = oracle.mesh_trace_attr(m, o, d)
    assert (r["V"] == 0).all()
    # hit normals are turned towards the (inside) origin
    assert (np.einsum("ij,ij->i", r["normal"], d) < 0).all()


def test_relight_reductions():
    rng = np.random.default_rng(4)
    gb = random_gbuffer(rng, 40, eye=(0.0, 0.0, 3.0))
    env = wl.envmap_hdr(9, 64, 32)
    pre = oracle.env_prefilter(env)
    none = _mesh(np.zeros((3, 3)), np.zeros((0, 3)))
    a = oracle.shade_relight_mesh(none, gb, env, pre, 8, 4, 4, seed=3)
    b = oracle.shade_pixels(scene([]), gb, env, 8, 4, 4, seed=3)   # no occluder: the training estimate
    np.testing.assert_array_equal(a["color"], b["color"])
    assert not a["ind"].any()
    # a huge opaque sheet above a Lambert point: every upward sample is blocked (V = 0)
    sheet = _mesh([[-1e3, -1e3, 1.0], [1e3, -1e3, 1.0], [0, 1e3, 1.0]], [[0, 1, 2]],
                  normal=np.tile([0, 0, -1.0], (3, 1)), albedo=np.full((3, 3), 0.8), rough=np.ones(3))
    g1 = gbuffer([[0, 0, 0]], [[0, 0, 1]], [[0.5, 0.5, 0.5]], [1.0], [0.0], eye=(0, 0, 5))
    envc = wl.envmap_constant(1.0, 64, 32)
    r = oracle.shade_relight_mesh(sheet, g1, envc, oracle.env_prefilter(envc), 16, 0, 0, seed=1, brdf=0)
    assert r["vis"][0] == 0.0 and 0.8 * 0.9 < r["ind"][0, 0] < 1.0
