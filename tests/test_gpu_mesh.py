"""GPU parity of the mesh backend of Eq. 14 (Sec. III-E) against the oracle: the LBVH of
triangles, the closest hit (decided in FP32 by the same watertight test on both sides, so
hit or miss agrees on every ray) and its barycentric attributes (1e-4; normals 5e-4), and
the relit MIS estimate within 1e-4 max(1, |ref|)."""
import numpy as np
import pytest
import torch

import oracle
from tests._gpu import hdr_tol, random_rays, t, unflagged, upsample_gbuffer
from tests._handmade import icosphere
from paper_2607_22780_b300 import _lib as L, api, workloads as wl

pytestmark = pytest.mark.gpu


def _mesh(pos, tri, **attrs):
    pos = np.asarray(pos, np.float32); tri = np.asarray(tri, np.int32).reshape(-1, 3)
    V = len(pos)
    dflt = dict(normal=np.tile([0, 0, 1.0], (V, 1)), albedo=np.full((V, 3), 0.5), rough=np.full(V, 0.5),
                metal=np.zeros(V))
    dflt.update(attrs)
    return wl.Mesh(pos=pos, tri=tri, **{k: np.asarray(v, np.float32) for k, v in dflt.items()})


def _attr(M, o, d, params=None):
    return [x.cpu().numpy() for x in api.mesh_trace_attr(M, t(o), t(d), params=params)]


def _check_attr(got, ref, min_hits):
    V, a, r, m, n = got
    keep = unflagged(ref["flags"])
    assert keep.all() and (ref["V"] == 0).sum() >= min_hits
    np.testing.assert_array_equal(V[keep], ref["V"][keep])
    for x, want, tol in ((a, ref["albedo"], 1e-4), (r, ref["rough"], 1e-4), (m, ref["metal"], 1e-4),
                         (n, ref["normal"], 5e-4)):
        err = np.abs(x - want).reshape(len(V), -1).max(1)
        assert err[keep].max() < tol, (tol, np.nonzero(keep & (err >= tol))[0][:8], err[keep].max())


def test_single_triangle_closed_form():
    m = _mesh([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]],
              albedo=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], rough=[0.2, 0.6, 1.0], metal=[0, 1, 0])
    M = api.MeshScene.from_workload(m)
    o = np.array([[0.25, 0.5, -1.0], [0.8, 0.8, -1.0], [0.25, 0.5, 1.0]], np.float32)
    d = np.array([[0, 0, 1.0], [0, 0, 1.0], [0, 0, -1.0]], np.float32)
    V, a, r, mm, n = _attr(M, o, d)
    np.testing.assert_array_equal(V, [0, 1, 0])
    np.testing.assert_allclose(a[0], [0.25, 0.25, 0.5], atol=1e-6)
    assert abs(r[0] - (0.25 * 0.2 + 0.25 * 0.6 + 0.5 * 1.0)) < 1e-6 and abs(mm[0] - 0.25) < 1e-6
    np.testing.assert_allclose(n[0], [0, 0, -1], atol=1e-6)   # turned towards the origin
    np.testing.assert_allclose(n[2], [0, 0, 1], atol=1e-6)
    assert not a[1].any() and not n[1].any()
    assert M.status() == 0


def test_empty_mesh_misses_everything():
    M = api.MeshScene.from_workload(_mesh(np.zeros((3, 3)), np.zeros((0, 3))))
    rng = np.random.default_rng(2)
    o, d = random_rays(rng, 100)
    V, a, _, _, _ = _attr(M, o, d)
    assert (V == 1).all() and not a.any()


def test_stacked_triangles_nearest_and_t_range():
    pos = [[-1, -1, 2], [3, -1, 2], [-1, 3, 2], [-1, -1, 1], [3, -1, 1], [-1, 3, 1]]
    m = _mesh(pos, [[0, 1, 2], [3, 4, 5]], albedo=[[1, 0, 0]] * 3 + [[0, 1, 0]] * 3)
    M = api.MeshScene.from_workload(m)
    d = np.array([[0, 0, 1.0]] * 2, np.float32)
    _, a, _, _, _ = _attr(M, np.array([[0, 0, 0], [0, 0, 1.5]], np.float32), d)
    assert a[0, 1] == 1.0 and a[1, 0] == 1.0
    p = api.trace_params(t_min=0.01, t_max=0.9)
    V, _, _, _, _ = _attr(M, np.array([[0, 0, 0]] * 2, np.float32), d, params=p)
    assert (V == 1).all()


@pytest.mark.parametrize("res", [6, 24])
def test_trace_attr_matches_oracle(res):
    m = wl.mesh_objects(13, res=res)
    rng = np.random.default_rng(14)
    o, d = random_rays(rng, 4000, -2.5, 2.5, 1.2)
    M = api.MeshScene.from_workload(m)
    assert M.info()["n_triangles"] == len(m.tri)
    _check_attr(_attr(M, o, d), oracle.mesh_trace_attr(m, o, d), 1000)
    assert M.status() == 0


def test_closed_mesh_blocks_every_ray_from_inside():
    # watertightness: rays from inside a closed icosphere, many aimed exactly at shared
    # vertices and edge midpoints, all hit
    v, f = icosphere(4)
    m = _mesh(1.7 * v + [0.2, -0.1, 0.3], f, normal=v)
    rng = np.random.default_rng(9)
    c = np.array([0.2, -0.1, 0.3]) + rng.uniform(-0.3, 0.3, (8, 3))
    tgt = np.concatenate([m.pos, 0.5 * (m.pos[f[:, 0]] + m.pos[f[:, 1]])])
    o = np.repeat(c, len(tgt), 0).astype(np.float32)
    dd = np.tile(tgt, (len(c), 1)) - o
    d = (dd / np.linalg.norm(dd, axis=1, keepdims=True)).astype(np.float32)
    M = api.MeshScene.from_workload(m)
    V, a, r, mm, n = _attr(M, o, d)
    assert (V == 0).all()
    sub = np.random.default_rng(1).choice(len(o), 2000, replace=False)
    _check_attr([x[sub] for x in (V, a, r, mm, n)], oracle.mesh_trace_attr(m, o[sub], d[sub]), 2000)
    assert M.status() == 0


def test_bad_vertex_index_is_reported():
    m = _mesh([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 7]])
    M = api.MeshScene.from_workload(m)
    _attr(M, np.array([[0.1, 0.1, -1.0]], np.float32), np.array([[0, 0, 1.0]], np.float32))
    assert M.status() & L.STATUS_BAD_INDEX


def test_relight_with_an_empty_mesh_equals_shading_without_occluders():
    # no triangle: every relighting ray misses (V = 1, no indirect), which is the training
    # estimate of a scene whose rays all escape
    from tests._handmade import random_gbuffer
    rng = np.random.default_rng(4)
    gb = random_gbuffer(rng, 300, eye=(0.0, 0.0, 3.0))
    M = api.MeshScene.from_workload(_mesh(np.zeros((3, 3)), np.zeros((0, 3))))
    sc = wl.scene_random_soup(10, seed=1, extent=0.1, scale_lo=0.01, scale_hi=0.02)
    sc.mu[:] += 50.0  # far away from every ray
    S = api.Scene.from_workload(sc)
    G = api.GBuffer.from_arrays(gb)
    E = api.Environment(t(wl.envmap_hdr(9, 64, 32)))
    a = api.shade_relight_mesh(M, G, E, 8, 4, 4, seed=3)
    b = api.shade_pixels(S, G, E, 8, 4, 4, seed=3)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def _check_relit(got, ref, pix=None):
    m = unflagged(ref["flags"])
    assert m.mean() > 0.95, m.mean()
    for a, r in zip(got, (ref["color"], ref["vis"], ref["ind"])):
        a = a.cpu().numpy()
        if pix is not None:
            a = a[pix]
        bad = (np.abs(a - r) > hdr_tol(r)).reshape(len(m), -1).any(1) & m
        assert bad.sum() == 0, (np.nonzero(bad)[0][:5], a[bad][:3], r[bad][:3])


def test_relight_mesh_matches_oracle():
    # the analytic objects as triangles; the G-buffer of the surfel scene of the same layout
    m = wl.mesh_objects(17, res=12)
    sc = wl.scene_objects(150000, seed=17)
    gb32 = oracle.gbuffer_f32(oracle.gbuffer(sc, wl.camera_orbit(17, 40, 32, 3.0)))
    env = wl.envmap_hdr(117, 128, 64)
    ref = oracle.shade_relight_mesh(m, gb32, env, oracle.env_prefilter(env), 16, 8, 8, seed=77)
    M = api.MeshScene.from_workload(m)
    got = api.shade_relight_mesh(M, api.GBuffer.from_arrays(gb32), api.Environment(t(env)), 16, 8, 8, seed=77)
    assert gb32["valid"].sum() > 400
    _check_relit(got, ref)
    assert float(got[2].abs().sum()) > 0 and (got[1].cpu().numpy() < 1).any() and M.status() == 0


def test_relight_mesh_full_size_sampled_pixels():
    m = wl.mesh_objects(2607, res=64)
    sc = wl.scene_objects(300_000, seed=2607)
    gb32 = upsample_gbuffer(oracle.gbuffer_f32(oracle.gbuffer(sc, wl.camera_orbit(2607, 100, 100, 3.0))), 8)
    env = wl.envmap_hdr(4242, 512, 256)
    M = api.MeshScene.from_workload(m)
    got = api.shade_relight_mesh(M, api.GBuffer.from_arrays(gb32), api.Environment(t(env)), 16, 8, 8, seed=5)
    pix = np.random.default_rng(3).choice(np.nonzero(gb32["valid"])[0], 48, replace=False).astype(np.int32)
    ref = oracle.shade_relight_mesh(m, gb32, env, oracle.env_prefilter(env), 16, 8, 8, seed=5, pixels=pix)
    _check_relit(got, ref, pix)
    assert np.isfinite(got[0].cpu().numpy()).all() and M.status() == 0
