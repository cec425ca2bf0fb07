"""GPU parity of the cross-bilateral denoiser (Sec. III-D) against the FP64 oracle, every
pixel: |gpu - ref| <= 1e-4 max(1, |ref|) (FP32 exp/pow of up to 289 weights per pixel)."""
import numpy as np
import pytest
import torch

import oracle
from tests._gpu import t, upsample_gbuffer
from paper_2607_22780_b300 import _lib, api, workloads as wl

pytestmark = pytest.mark.gpu


def _guides(W, H, seed, n=20000):
    sc = wl.scene_objects(n, seed=seed)
    g = oracle.gbuffer(sc, wl.camera_orbit(seed, W, H, 3.0))
    return (np.asarray(g["depth"], np.float32), np.asarray(g["normal"], np.float32),
            np.asarray(g["valid"], np.int32))


def _noisy(rng, P):
    return rng.lognormal(-1.0, 1.0, size=(P, 3)).astype(np.float32)


def _check(color, depth, normal, valid, W, H, **prm):
    got = api.denoise(t(color), t(depth), t(normal), t(valid, torch.int32), W, H, **prm).cpu().numpy()
    q = dict(api.DENOISE_DEFAULTS)
    q.update(prm)
    ref = oracle.denoise(color, depth, normal, valid, W, H, **q)
    err = np.abs(got - ref) - 1e-4 * np.maximum(1.0, np.abs(ref))
    assert err.max() <= 0, (np.unravel_index(err.argmax(), err.shape), got.ravel()[err.argmax()], ref.ravel()[err.argmax()])
    return got, ref


@pytest.mark.parametrize("radius,sigma_n", [(0, 64.0), (1, 64.0), (3, 64.0), (5, 8.0), (8, 128.0)])
def test_denoise_matches_oracle(radius, sigma_n):
    W, H = 70, 37  # ragged against the 32x8 tiles
    depth, normal, valid = _guides(W, H, seed=61)
    rng = np.random.default_rng(radius)
    color = _noisy(rng, W * H)
    color[valid == 0] = 0
    _check(color, depth, normal, valid, W, H, radius=radius, sigma_n=sigma_n, sigma_s=1.5 + radius)


def test_denoise_tiny_and_degenerate_images():
    rng = np.random.default_rng(3)
    for W, H in ((1, 1), (2, 3), (5, 1), (1, 9)):
        P = W * H
        normal = rng.normal(size=(P, 3)).astype(np.float32) * 0.2 + np.float32([0, 0, 1])
        depth = rng.uniform(1, 2, P).astype(np.float32)
        valid = (rng.uniform(size=P) < 0.8).astype(np.int32)
        normal[0] = 0  # a valid pixel without a normal keeps its colour
        _check(_noisy(rng, P), depth, normal, valid, W, H, radius=4, sigma_n=4.0)


def test_denoise_full_frame_800():
    # the oracle's 100x100 G-buffer enlarged to 800x800 as guides, seeded HDR noise
    sc = wl.scene_objects(300_000, seed=2607)
    g = oracle.gbuffer(sc, wl.camera_orbit(2607, 100, 100, 3.0))
    small = dict(pos=g["pos"], normal=np.asarray(g["normal"], np.float32), albedo=g["albedo"], rough=g["rough"],
                 metal=g["metal"], valid=np.asarray(g["valid"], np.int32), eye=g["eye"], W=100, H=100)
    small["pos"] = np.asarray(g["depth"], np.float32)[:, None].repeat(3, 1)  # carry depth through the enlargement
    big = upsample_gbuffer(small, 8)
    depth = np.ascontiguousarray(big["pos"][:, 0])
    rng = np.random.default_rng(8)
    color = _noisy(rng, 800 * 800)
    got, ref = _check(color, depth, big["normal"], big["valid"], 800, 800)
    assert np.abs(got - color).max() > 0.1  # it did filter


def test_denoise_argument_errors():
    z = torch.zeros((4, 3), device="cuda")
    d = torch.ones(4, device="cuda")
    v = torch.ones(4, dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.GrtError):
        api.denoise(z, d, z, v, 2, 2, radius=_lib.GRT_DENOISE_MAX_RADIUS + 1)
    with pytest.raises(_lib.GrtError):
        api.denoise(z, d, z, v, 2, 2, out=z)
    with pytest.raises(_lib.GrtError):
        api.denoise(z, d, z, v, 2, 2, sigma_s=0.0)
