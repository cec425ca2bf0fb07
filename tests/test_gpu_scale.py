"""Parity at the workloads' own scales.

* Differentiable 2DGRT on the 300k-surfel object scene: the FP64 oracle gradient of a
  32x32 view (L2 loss against the seeded target), and central finite differences of the
  GPU forward on 64 random parameters of the 400x400, 16 rays/pixel frame.
* The 2M-surfel unbounded scene at 1920x1080 with 16 rays/pixel (8/4/4): G-buffer,
  shading and gradients of sampled pixels against the oracle, the whole frame for
  finiteness and device status."""
import numpy as np
import pytest
import torch

import oracle
from tests._gpu import (GRAD_FIELDS, check_gbuffer_rows, check_grads, gbuffer_to_arrays, hdr_tol, scene_gpu, t,
                        unflagged, upsample_gbuffer)
from paper_2607_22780_b300 import api, workloads as wl

pytestmark = pytest.mark.gpu

SEED = 2607
ALLOC = (8, 4, 4)


@pytest.fixture(scope="module")
def objects_300k():
    return wl.scene_objects(300_000, seed=SEED)


def test_c3_crop_gradient_matches_oracle(objects_300k):
    sc = objects_300k
    cam = wl.camera_orbit(SEED, 32, 32, 3.0)
    gb32 = oracle.gbuffer_f32(oracle.gbuffer(sc, cam))
    env = wl.envmap_hdr(SEED, 512, 256)
    tgt = wl.target_image(SEED, 32, 32).reshape(-1, 3)
    fwd = oracle.shade_pixels(sc, gb32, env, *ALLOC, seed=SEED)
    keep = np.nonzero((fwd["flags"] == 0) & (gb32["valid"] == 1))[0].astype(np.int32)
    assert len(keep) > 300
    # L = 1/2 sum over kept pixels |c - target|^2, upstream gradient from the oracle's forward
    dc = (fwd["color"][keep] - tgt[keep]).astype(np.float32)
    ref = oracle.backward_pixels(sc, gb32, env, *ALLOC, seed=SEED, dL_dcolor=dc, pixels=keep)
    assert np.all(ref["flags"] == 0)
    S = scene_gpu(sc)
    g = api.shade_backward(S, api.GBuffer.from_arrays(gb32), api.Environment(t(env)), *ALLOC, SEED, t(dc),
                           pixels=t(keep, torch.int32))
    check_grads(g, ref)
    assert S.status() == 0


def _fd_params(g, rng, per_field=(13, 13, 13, 13, 12), frac=0.05):
    """Random (field, flat index) pairs among entries with |g| >= frac * max |g| of the field."""
    out = []
    for f, n in zip(GRAD_FIELDS, per_field):
        a = getattr(g, f).reshape(-1).cpu().numpy()
        cand = np.nonzero(np.abs(a) >= frac * np.abs(a).max())[0]
        out += [(f, int(i)) for i in rng.choice(cand, size=min(n, len(cand)), replace=False)]
    return out


def test_c3_gradient_vs_central_differences(objects_300k):
    # 400x400 frame, 16 rays/pixel, L2 loss against the seeded target, 64 random parameters.
    # The rendered loss is piecewise smooth: a step that moves a hit across the alpha_min
    # cut-off, or across an exact depth tie (coplanar surfels), jumps.  Each parameter walks
    # a ladder of steps h0 / 4^k; a step is clean when the composited-hit total at +-h is
    # unchanged and the loss change |g| 2h (>= 5e-4) stands above the FP32 rounding of the
    # image (~2e-5); the first two consecutive clean steps whose quotients agree within 1% give
    # the finite difference, which must match the analytic gradient within 2%.
    sc = objects_300k
    S = scene_gpu(sc)
    cam = wl.camera_orbit(SEED, 400, 400, 3.0)
    G = api.gbuffer_primary(S, cam)
    E = api.Environment(t(wl.envmap_hdr(SEED, 512, 256)))
    tgt = t(wl.target_image(SEED, 400, 400).reshape(-1, 3)).double()
    valid = G.valid.double().unsqueeze(1)

    def loss():
        col, _, _ = api.shade_pixels(S, G, E, *ALLOC, seed=SEED)
        return 0.5 * float((((col.double() - tgt) * valid) ** 2).sum())

    def composited():
        return int(api.shade_count(S, G, E, *ALLOC, seed=SEED)[2])

    L0, c0 = loss(), composited()
    col, _, _ = api.shade_pixels(S, G, E, *ALLOC, seed=SEED)
    dl = ((col.double() - tgt) * valid).float().contiguous()
    g = api.shade_backward(S, G, E, *ALLOC, SEED, dl)
    h0 = dict(mu=1e-4, quat=1e-3, scale=None, opacity=1e-3, color=4e-2)

    def step(f, i, h):
        """(quotient, clean) for the central difference of step h."""
        p = getattr(S, f).view(-1)
        x = float(p[i])
        xp, xm = np.float32(x + h), np.float32(x - h)
        p[i] = float(xp)
        S.refit()
        lp, cp = loss(), composited()
        p[i] = float(xm)
        S.refit()
        lm, cm = loss(), composited()
        p[i] = x
        return (lp - lm) / (float(xp) - float(xm)), cp == c0 and cm == c0

    rng = np.random.default_rng(64)
    rows = []
    for f, i in _fd_params(g, rng):
        a = float(getattr(g, f).view(-1)[i])
        h = h0[f] if h0[f] is not None else 1e-2 * abs(float(getattr(S, f).view(-1)[i]))
        prev, fd = None, None
        for k in range(6):
            hk = h / 4 ** k
            if abs(a) * 2 * hk < 5e-4:
                break
            q, clean = step(f, i, hk)
            if not clean:
                prev = None
                continue
            if prev is not None and abs(q - prev) <= 0.01 * max(abs(q), abs(prev)):
                fd = prev
                break
            prev = q
        rows.append((f, i, a, fd))
    S.refit()
    assert loss() == L0  # parameters restored exactly, forward deterministic
    print("\n".join("%-8s %8d  g=% .6e  fd=%s" % (f, i, a, "-" if d is None else "% .6e" % d) for f, i, a, d in rows))
    checked = [r for r in rows if r[3] is not None]
    bad = [r for r in checked if abs(r[3] - r[2]) > 0.02 * max(abs(r[3]), abs(r[2]))]
    per_field = {f: sum(r[0] == f for r in checked) for f in GRAD_FIELDS}
    assert len(rows) == 64
    assert len(checked) >= 32 and min(per_field.values()) >= 3, per_field
    assert not bad, bad


@pytest.fixture(scope="module")
def large_2m():
    sc = wl.scene_large(2_000_000, seed=SEED)
    return sc, scene_gpu(sc)


def test_c4_gbuffer_sampled_pixels(large_2m):
    sc, S = large_2m
    cam = wl.camera_orbit(SEED, 1920, 1080, 12.0)
    g = api.gbuffer_primary(S, cam)
    got = gbuffer_to_arrays(g, cam.eye, 1920, 1080)
    assert got["valid"].mean() > 0.3
    rng = np.random.default_rng(5)
    pix = np.concatenate([rng.choice(np.nonzero(got["valid"])[0], 48, replace=False),
                          rng.choice(1920 * 1080, 16, replace=False)]).astype(np.int32)
    check_gbuffer_rows(got, oracle.gbuffer(sc, cam, pixels=pix), pix, min_valid=44)
    assert S.status() == 0


def test_c4_shading_and_gradients_sampled_pixels(large_2m):
    # 1920x1080 frame: the oracle's 48x27 view enlarged 40x (an oracle-made G-buffer at
    # full size), k = 16; whole-frame forward and backward, sampled pixels vs the oracle
    sc, S = large_2m
    gb32 = upsample_gbuffer(oracle.gbuffer_f32(oracle.gbuffer(sc, wl.camera_orbit(SEED, 48, 27, 12.0))), 40)
    assert gb32["W"] == 1920 and gb32["H"] == 1080
    env = wl.envmap_hdr(SEED + 1, 512, 256)
    G = api.GBuffer.from_arrays(gb32)
    E = api.Environment(t(env))
    col, vis, ind = api.shade_pixels(S, G, E, *ALLOC, seed=SEED)
    rng = np.random.default_rng(6)
    pix = rng.choice(np.nonzero(gb32["valid"])[0], size=48, replace=False).astype(np.int32)
    ref = oracle.shade_pixels(sc, gb32, env, *ALLOC, seed=SEED, pixels=pix)
    m = unflagged(ref["flags"])
    assert m.sum() >= 40
    for a, r in ((col, ref["color"]), (vis, ref["vis"]), (ind, ref["ind"])):
        a = a.cpu().numpy()[pix]
        bad = (np.abs(a - r) > hdr_tol(r)).reshape(len(pix), -1).any(1) & m
        assert bad.sum() == 0, (a[bad], r[bad])
    # gradients of the sampled, unflagged pixels against the oracle
    keep = pix[m]
    w = rng.normal(size=(len(keep), 3)).astype(np.float32)
    refg = oracle.backward_pixels(sc, gb32, env, *ALLOC, seed=SEED, dL_dcolor=w, pixels=keep)
    assert np.all(refg["flags"] == 0)
    gs = api.shade_backward(S, G, E, *ALLOC, SEED, t(w), pixels=t(keep, torch.int32))
    check_grads(gs, refg)
    # the whole frame (33M ray slots, recomputed in several chunks) with the same upstream
    # gradient on those pixels and zero elsewhere gives the same gradients
    dc = torch.zeros_like(col)
    dc[torch.from_numpy(keep).long().cuda()] = t(w)
    gf = api.shade_backward(S, G, E, *ALLOC, SEED, dc)
    for f in GRAD_FIELDS:
        x, y = getattr(gf, f), getattr(gs, f)
        assert torch.isfinite(x).all(), f
        assert torch.allclose(x, y, rtol=1e-4, atol=1e-6 * float(y.abs().max())), f
    assert S.status() == 0
