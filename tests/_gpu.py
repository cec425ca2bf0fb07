"""Helpers shared by the GPU parity tests (inputs from workloads, expectations from oracle)."""
import numpy as np
import torch

from paper_2607_22780_b300 import api, workloads as wl

DEV = "cuda"


def t(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV).contiguous()


def scene_gpu(sc, **params):
    return api.Scene.from_workload(sc, params=api.trace_params(**params) if params else None)


def random_rays(rng, R, lo=-1.5, hi=1.5, target=0.8):
    o = rng.uniform(lo, hi, size=(R, 3))
    tg = rng.uniform(-target, target, size=(R, 3))
    d = tg - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def unflagged(flags):
    return np.asarray(flags) == 0


def hits_equal(gpu_hits, gpu_n, ora_hits, ora_n, mask):
    """Rows (under mask) whose composited id lists agree exactly."""
    gh, gn = gpu_hits.cpu().numpy(), gpu_n.cpu().numpy()
    ok = np.ones(len(gn), bool)
    for i in np.nonzero(mask)[0]:
        k = min(gn[i], gh.shape[1])
        ok[i] = gn[i] == ora_n[i] and np.array_equal(gh[i, :k], ora_hits[i, :k])
    return ok


def hdr_tol(ref, rel=1e-4):
    return rel * np.maximum(1.0, np.abs(ref))


def upsample_gbuffer(gb, f):
    """Nearest-neighbour enlargement of a G-buffer by an integer factor: each pixel of the
    source becomes an f x f block (a full-resolution input made from a small oracle view)."""
    W, H = int(gb["W"]), int(gb["H"])
    out = dict(eye=gb["eye"], W=W * f, H=H * f)
    for k in ("pos", "normal", "albedo", "rough", "metal", "valid"):
        a = np.asarray(gb[k])
        img = a.reshape(H, W, -1)
        img = np.repeat(np.repeat(img, f, axis=0), f, axis=1)
        out[k] = np.ascontiguousarray(img.reshape((H * f * W * f,) + a.shape[1:]))
    return out


def gbuffer_to_arrays(g, eye, W, H):
    """A device G-buffer copied to host arrays (for checks that read it, never as oracle input)."""
    return dict(pos=g.pos.cpu().numpy(), normal=g.normal.cpu().numpy(), albedo=g.albedo.cpu().numpy(),
                rough=g.rough.cpu().numpy(), metal=g.metal.cpu().numpy(), valid=g.valid.cpu().numpy(),
                alpha=g.alpha.cpu().numpy() if g.alpha is not None else None,
                depth=g.depth.cpu().numpy() if g.depth is not None else None,
                eye=np.asarray(eye, np.float32), W=W, H=H)


# G-buffer tolerances (FP32 kernel against the FP64 oracle).  The error comes from the FP32
# hit point p = o + tau d, rounded at the scale of |p|, against surfel scales down to 1e-3:
# it perturbs each alpha, hence the normalised weights of Eq. 9, so depth and position errors
# grow with the depth D (observed at most 3.4e-5 D on 2M-surfel 1080p views at D ~ 20,
# 7e-6 D on the 300k-surfel and C1 views), the unit normal's error with the spread of the
# blended normals (observed 1.6e-4), weighted attributes in [0, 1] by at most 8.1e-5.
GB_TOL_DEPTH_REL = 1e-4   # depth and position: 1e-4 max(1, D)
GB_TOL_NORMAL = 3e-4
GB_TOL_ATTR = 1e-4        # albedo, roughness, metallic, opacity


def gbuffer_tolerance(k, depth):
    """Per-pixel tolerance of G-buffer field k (depth: the oracle's depth of the pixels)."""
    if k in ("pos", "depth"):
        return GB_TOL_DEPTH_REL * np.maximum(1.0, np.abs(depth))
    return GB_TOL_NORMAL if k == "normal" else GB_TOL_ATTR


def check_gbuffer_rows(got, ref, pix, min_valid):
    """GPU G-buffer rows at pixels `pix` against the oracle's rows for the same pixels."""
    m = unflagged(ref["flags"])
    assert np.array_equal(got["valid"][pix][m], ref["valid"][m])
    v = m & (ref["valid"] == 1)
    assert v.sum() >= min_valid, v.sum()
    for k in ("pos", "normal", "albedo", "rough", "metal"):
        err = np.abs(got[k][pix][v] - ref[k][v]).reshape(int(v.sum()), -1).max(1)
        tol = gbuffer_tolerance(k, ref["depth"][v])
        assert np.all(err < tol), (k, float(err.max()), float((err / tol).max()))


GRAD_FIELDS = ("mu", "quat", "scale", "opacity", "color")


def check_grads(g, ref, rel=2e-3, absf=1e-5):
    """|g - ref| <= rel |ref| + absf max|ref| per parameter block (FP32 atomics vs FP64)."""
    for f in GRAD_FIELDS:
        a = getattr(g, f).cpu().numpy().astype(np.float64)
        r = ref[f]
        scale = np.abs(r).max()
        assert scale > 0, f
        err = np.abs(a - r) - (rel * np.abs(r) + absf * scale)
        assert err.max() <= 0, (f, np.unravel_index(err.argmax(), err.shape), a.ravel()[err.argmax()],
                                r.ravel()[err.argmax()])
