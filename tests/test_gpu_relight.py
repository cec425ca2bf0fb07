"""GPU parity of relighting (Sec. III-E, Eq. 14-15) against the FP64 oracle: the prefiltered
map E (1e-4 relative), Trace_attr per ray (1e-4; normals 5e-4), and the relit MIS estimate
on unflagged pixels within 1e-4 max(1, |ref|), as for shading (observed: 3e-6)."""
import numpy as np
import pytest
import torch

import oracle
from tests._gpu import hdr_tol, random_rays, scene_gpu, t, unflagged, upsample_gbuffer
from tests._handmade import random_gbuffer
from paper_2607_22780_b300 import api, workloads as wl

pytestmark = pytest.mark.gpu


def _tables(E):
    f = E.prefiltered.cpu().numpy()
    d = 3 * oracle.DIFF_W * oracle.DIFF_H
    s = 3 * (oracle.SPEC_LEVELS - 1) * oracle.SPEC_W * oracle.SPEC_H
    lut = 2 * oracle.LUT_N ** 2
    return (f[:d].reshape(oracle.DIFF_H, oracle.DIFF_W, 3),
            f[d:d + s].reshape(oracle.SPEC_LEVELS - 1, oracle.SPEC_H, oracle.SPEC_W, 3),
            f[d + s:d + s + lut].reshape(oracle.LUT_N, oracle.LUT_N, 2),
            f[d + s + lut:d + s + lut + 6 * (oracle.SPEC_LEVELS + 1)].reshape(oracle.SPEC_LEVELS + 1, 2, 3))


@pytest.mark.parametrize("size", [(64, 32), (512, 256)])
def test_prefilter_matches_oracle(size):
    env = wl.envmap_hdr(5, *size)
    E = api.Environment(t(env))
    E.prefilter()
    diff, spec, lut, poles = _tables(E)
    ref = oracle.env_prefilter(env)
    # pole-row means of the diffuse grid, the specular levels and the map
    grids = [ref["diff"]] + list(ref["spec"]) + [env.astype(np.float64)]
    ref_poles = np.stack([np.stack([g[0].mean(0), g[-1].mean(0)]) for g in grids])
    for a, r in ((diff, ref["diff"]), (spec, ref["spec"]), (lut, ref["lut"]), (poles, ref_poles)):
        err = np.abs(a - r) - 1e-4 * np.maximum(np.abs(r), 1e-2)
        assert err.max() <= 0, (np.unravel_index(err.argmax(), err.shape), a.ravel()[err.argmax()], r.ravel()[err.argmax()])


def test_trace_attr_matches_oracle():
    sc = wl.scene_objects(20000, seed=13)
    rng = np.random.default_rng(14)
    o, d = random_rays(rng, 3000, -2.0, 2.0, 1.5)
    S = scene_gpu(sc)
    V, a, r, m, n = (x.cpu().numpy() for x in api.trace_attr(S, t(o), t(d)))
    ref = oracle.trace_attr(sc, o, d)
    keep = unflagged(ref["flags"])
    assert keep.mean() > 0.99 and (ref["V"][keep] < 1).sum() > 500
    assert np.abs(V - ref["V"])[keep].max() < 1e-4
    for got, want, tol in ((a, ref["albedo"], 1e-4), (r, ref["rough"], 1e-4), (m, ref["metal"], 1e-4),
                           (n, ref["normal"], 5e-4)):
        err = np.abs(got - want).reshape(len(V), -1).max(1)
        assert err[keep].max() < tol, (tol, err[keep].max())
    assert S.status() == 0


def test_relight_without_occluders_equals_shading_bitwise():
    rng = np.random.default_rng(4)
    gb = random_gbuffer(rng, 300, eye=(0.0, 0.0, 3.0))
    sc = wl.scene_random_soup(10, seed=1, extent=0.1, scale_lo=0.01, scale_hi=0.02)
    sc.mu[:] += 50.0  # far away from every ray
    S = scene_gpu(sc)
    G = api.GBuffer.from_arrays(gb)
    E = api.Environment(t(wl.envmap_hdr(9, 64, 32)))
    a = api.shade_relight(S, G, E, 8, 4, 4, seed=3)
    b = api.shade_pixels(S, G, E, 8, 4, 4, seed=3)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def _objects_case(n=30000, W=48, H=40, seed=17):
    sc = wl.scene_objects(n, seed=seed)
    cam = wl.camera_orbit(seed, W, H, 3.0)
    gb32 = oracle.gbuffer_f32(oracle.gbuffer(sc, cam))
    env = wl.envmap_hdr(seed + 100, 128, 64)
    return sc, gb32, env


def _check_relit(got, ref, pix=None):
    m = unflagged(ref["flags"])
    assert m.mean() > 0.95
    for a, r, rel in ((got[0], ref["color"], 1e-4), (got[1], ref["vis"], 1e-4), (got[2], ref["ind"], 1e-4)):
        a = a.cpu().numpy()
        if pix is not None:
            a = a[pix]
        bad = (np.abs(a - r) > hdr_tol(r, rel)).reshape(len(m), -1).any(1) & m
        assert bad.sum() == 0, (np.nonzero(bad)[0][:5], a[bad][:3], r[bad][:3])


def test_relight_matches_oracle():
    sc, gb32, env = _objects_case()
    ref = oracle.shade_relight(sc, gb32, env, oracle.env_prefilter(env), 16, 8, 8, seed=77)
    S = scene_gpu(sc)
    got = api.shade_relight(S, api.GBuffer.from_arrays(gb32), api.Environment(t(env)), 16, 8, 8, seed=77)
    _check_relit(got, ref)
    assert float(got[2].abs().sum()) > 0 and S.status() == 0


def test_relight_full_size_sampled_pixels():
    sc = wl.scene_objects(300_000, seed=2607)
    gb32 = upsample_gbuffer(oracle.gbuffer_f32(oracle.gbuffer(sc, wl.camera_orbit(2607, 100, 100, 3.0))), 8)
    env = wl.envmap_hdr(4242, 512, 256)
    S = scene_gpu(sc)
    got = api.shade_relight(S, api.GBuffer.from_arrays(gb32), api.Environment(t(env)), 16, 8, 8, seed=5)
    pix = np.random.default_rng(3).choice(np.nonzero(gb32["valid"])[0], 48, replace=False).astype(np.int32)
    ref = oracle.shade_relight(sc, gb32, env, oracle.env_prefilter(env), 16, 8, 8, seed=5, pixels=pix)
    _check_relit(got, ref, pix)
    assert np.isfinite(got[0].cpu().numpy()).all() and S.status() == 0
