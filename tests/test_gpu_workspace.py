"""Caller-supplied workspace of the shading calls (the boundary's workspace convention):
with a workspace of the reported size, shade_pixels, shade_batch and the adjoint give the
same results as with pool scratch, and reuse of one workspace across calls is safe."""
import numpy as np
import pytest
import torch

from paper_2607_22780_b300 import api, workloads as wl

pytestmark = pytest.mark.gpu

ALLOC = (8, 4, 4)


def _setup(n=20_000, img=48, seed=3):
    sc = wl.scene_objects(n, seed=seed)
    S = api.Scene.from_workload(sc)
    cam = wl.camera_orbit(seed, img, img, 3.0)
    G = api.gbuffer_primary(S, cam)
    E = api.Environment(torch.from_numpy(wl.envmap_hdr(seed, 64, 32)).cuda())
    return S, G, E


def _ws(nbytes):
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda")


def test_shade_pixels_with_workspace_is_bit_identical():
    S, G, E = _setup()
    P = G.W * G.H
    ref = api.shade_pixels(S, G, E, *ALLOC, seed=5)
    ws = _ws(api.shade_workspace_size(P * sum(ALLOC)))
    for seed in (5, 5):                      # the same workspace twice in a row
        got = api.shade_pixels(S, G, E, *ALLOC, seed=seed, workspace=ws)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    # a workspace one byte short is refused
    with pytest.raises(api.L.GrtError):
        api.shade_pixels(S, G, E, *ALLOC, seed=5, workspace=ws[:api.shade_workspace_size(P * sum(ALLOC)) - 1])
    assert S.status() == 0


def test_shade_batch_with_workspace_is_bit_identical():
    S, G, E = _setup()
    P = G.W * G.H
    half = P // 2
    reqs = [api.ShadeRequest(S, G, E, *ALLOC, seed=9, pixel_offset=0, count=half),
            api.ShadeRequest(S, G, E, 4, 2, 2, seed=11, pixel_offset=half, count=P - half)]
    rays = half * sum(ALLOC) + (P - half) * 8
    ws = _ws(api.shade_workspace_size(rays))
    api.shade_batch(reqs, workspace=ws)
    a = api.shade_pixels(S, G, E, *ALLOC, seed=9, pixels=torch.arange(half, dtype=torch.int32, device="cuda"))
    b = api.shade_pixels(S, G, E, 4, 2, 2, seed=11, pixels=torch.arange(half, P, dtype=torch.int32, device="cuda"))
    assert torch.equal(reqs[0].color, a[0]) and torch.equal(reqs[1].color, b[0])


@pytest.mark.parametrize("saved", [False, True])
def test_shade_backward_with_workspace_matches_pool(saved):
    S, G, E = _setup()
    P = G.W * G.H
    rng = np.random.default_rng(4)
    dc = torch.from_numpy(rng.normal(size=(P, 3)).astype(np.float32)).cuda()
    rec = None
    if saved:
        *_, rec = api.shade_pixels_save(S, G, E, *ALLOC, seed=7, max_hits=64)
    ref = api.shade_backward(S, G, E, *ALLOC, 7, dc, saved=rec)
    ws = _ws(api.shade_backward_workspace_size(P, *ALLOC, saved=saved))
    for _ in range(2):
        got = api.shade_backward(S, G, E, *ALLOC, 7, dc, saved=rec, workspace=ws)
        for f in ("mu", "quat", "scale", "opacity", "color"):
            a, b = getattr(got, f), getattr(ref, f)
            # the same additions in another order of float atomics
            tol = 1e-4 * float(b.abs().max()) + 1e-12
            assert float((a - b).abs().max()) <= tol, f
    assert S.status() == 0
