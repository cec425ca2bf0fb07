"""Pins of the oracle's cross-bilateral denoiser (Sec. III-D): closed forms of the three
weight factors on tiny images, and invariants of a normalised weighted average."""
import math

import numpy as np
import pytest

import oracle


def _line(colors, depth=None, normals=None, valid=None):
    n = len(colors)
    col = np.repeat(np.asarray(colors, float)[:, None], 3, axis=1)
    dep = np.ones(n) if depth is None else np.asarray(depth, float)
    nrm = np.tile([0.0, 0.0, 1.0], (n, 1)) if normals is None else np.asarray(normals, float)
    val = np.ones(n, np.int32) if valid is None else np.asarray(valid, np.int32)
    return col, dep, nrm, val


def test_constant_image_is_unchanged():
    rng = np.random.default_rng(0)
    W, H = 17, 11
    col = np.tile([0.3, 0.6, 0.9], (W * H, 1))
    dep = rng.uniform(1, 3, W * H)
    nrm = rng.normal(size=(W * H, 3))
    out = oracle.denoise(col, dep, nrm, np.ones(W * H), W, H, radius=3, sigma_n=2.0)
    np.testing.assert_allclose(out, col, rtol=0, atol=1e-15)


def test_spatial_weight_three_pixels():
    # flat depth, equal normals: only exp(-|p-p'|^2 / (2 s^2)) acts
    s = 0.8
    w = math.exp(-1 / (2 * s * s))
    out = oracle.denoise(*_line([0, 1, 0]), 3, 1, radius=1, sigma_s=s)
    assert out[1, 0] == pytest.approx(1 / (1 + 2 * w), abs=1e-14)
    assert out[0, 0] == pytest.approx(w / (1 + w), abs=1e-14)
    assert out[2, 1] == pytest.approx(w / (1 + w), abs=1e-14)


def test_depth_weight_on_a_ramp():
    # D = x: gradient 1 (central inside, one-sided at the ends); |D(p)-D(p')| = 1 and
    # s_d |grad D . (p-p')| + e_d = s_d + e_d for both neighbours of the centre
    s, sd, ed = 1.0, 0.5, 1e-3
    ws = math.exp(-1 / (2 * s * s))
    wd = math.exp(-1 / (sd * 1 + ed))
    out = oracle.denoise(*_line([0, 1, 0], depth=[0, 1, 2]), 3, 1, radius=1, sigma_s=s, sigma_d=sd, eps_d=ed)
    assert out[1, 0] == pytest.approx(1 / (1 + 2 * ws * wd), abs=1e-14)


def test_depth_step_needs_the_gradient():
    # a jump of 5 with zero gradient at the centre: the neighbour weight is exp(-5 / e_d) ~ 0
    out = oracle.denoise(*_line([1, 0, 0], depth=[6, 1, 1]), 3, 1, radius=1, sigma_s=10.0, eps_d=1e-2)
    # the centre's gradient is (1 - 6) / 2 = -2.5 (central), so the left neighbour gets
    # exp(-5 / (1 * 2.5 + 0.01)); the right one exp(0) = 1
    wl = math.exp(-5 / (2.5 + 0.01)) * math.exp(-1 / 200)
    wr = math.exp(-1 / 200)
    assert out[1, 0] == pytest.approx(wl / (1 + wl + wr), abs=1e-14)


def test_normal_weight_and_normalisation():
    n0 = [0.0, 0.0, 3.0]                              # not unit: normalised inside
    n1 = [math.sqrt(3) / 2, 0.0, 0.5]                # cos = 0.5 to n0
    out = oracle.denoise(*_line([0, 1], normals=[n0, n1]), 2, 1, radius=1, sigma_s=1e9, sigma_n=2.0)
    assert out[0, 0] == pytest.approx(0.25 / 1.25, abs=1e-14)
    ortho = oracle.denoise(*_line([0, 1], normals=[[0, 0, 1], [1, 0, 0]]), 2, 1, radius=1, sigma_s=1e9)
    assert ortho[0, 0] == 0 and ortho[1, 0] == 1


def test_invalid_pixels_and_radius_zero():
    col, dep, nrm, val = _line([0.2, 5.0, 0.4], valid=[1, 0, 1])
    out = oracle.denoise(col, dep, nrm, val, 3, 1, radius=2, sigma_s=1e9)
    assert out[1, 0] == 5.0                                   # invalid keeps its input
    assert out[0, 0] == pytest.approx(0.3, abs=1e-15)         # mixes only with valid pixel 2
    rng = np.random.default_rng(1)
    c = rng.uniform(size=(30, 3))
    same = oracle.denoise(c, rng.uniform(1, 2, 30), rng.normal(size=(30, 3)), np.ones(30), 6, 5, radius=0)
    np.testing.assert_array_equal(same, c)


def test_output_is_a_convex_combination_of_the_window():
    rng = np.random.default_rng(2)
    W, H, r = 23, 19, 2
    col = rng.uniform(size=(W * H, 3))
    dep = rng.uniform(1, 1.1, W * H)
    nrm = rng.normal(size=(W * H, 3)) * 0.1 + [0, 0, 1]
    out = oracle.denoise(col, dep, nrm, np.ones(W * H), W, H, radius=r, sigma_n=8.0)
    img = col.reshape(H, W, 3)
    for p in rng.choice(W * H, 40, replace=False):
        x, y = p % W, p // W
        win = img[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].reshape(-1, 3)
        assert np.all(out[p] >= win.min(0) - 1e-15) and np.all(out[p] <= win.max(0) + 1e-15)


def test_zero_normal_keeps_input():
    col, dep, nrm, val = _line([0.2, 0.7, 0.4], normals=[[0, 0, 1], [0, 0, 0], [0, 0, 1]])
    out = oracle.denoise(col, dep, nrm, val, 3, 1, radius=2, sigma_s=1e9)
    assert out[1, 0] == 0.7                         # no normal to compare with
    assert out[0, 0] == pytest.approx(0.3, abs=1e-15)  # the zero-normal neighbour gets weight 0
