"""Python API over libgrt: torch tensors in, torch tensors out, every step in CUDA.

PyTorch provides device memory and streams only; each function below marshals its
arguments and makes exactly one libgrt call (include/grt.h) on the current stream.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _lib as L

DEFAULT_PARAMS = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=0.01, t_max=3.0e38, T_min=1e-4,
                      eps_nd=1e-6, k=16, build_passes=1, gbuffer_k=0)


def trace_params(**kw) -> L.TraceParams:
    p = dict(DEFAULT_PARAMS)
    p.update({k: v for k, v in kw.items() if v is not None})
    return L.TraceParams(*[float(p[k]) for k in ("alpha_min", "alpha_max", "t_min", "t_max", "T_min", "eps_nd")],
                         int(p["k"]), int(p["build_passes"]), int(p["gbuffer_k"]))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _dev(t, dtype=torch.float32, name="tensor", shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Scene:
    """Surfels resident on the device plus their LBVH (grt_build_bvh).

    Tensors: mu[N,3], quat[N,4] (w,x,y,z), scale[N,2], opacity[N], color[N,3|48],
    albedo[N,3], rough[N], metal[N]; float32, contiguous, on one CUDA device.
    """

    def __init__(self, mu, quat, scale, opacity, color, albedo=None, rough=None, metal=None, params=None,
                 stream=None):
        n = int(mu.shape[0])
        self.n = n
        self.mu = _dev(mu, name="mu", shape=(n, 3))
        self.quat = _dev(quat, name="quat", shape=(n, 4))
        self.scale = _dev(scale, name="scale", shape=(n, 2))
        self.opacity = _dev(opacity, name="opacity", shape=(n,))
        self.color = _dev(color, name="color")
        if self.color.shape[0] != n or self.color.shape[1] not in (3, 48):
            raise ValueError("color must be [N,3] or [N,48]")
        self.albedo = _dev(albedo, name="albedo", shape=(n, 3))
        self.rough = _dev(rough, name="rough", shape=(n,))
        self.metal = _dev(metal, name="metal", shape=(n,))
        self.params = params if params is not None else trace_params()
        self._bvh = C.c_void_p(None)
        self._lib = L.load()
        L.check(self._lib.grt_build_bvh(C.byref(self.surfels()), C.byref(self.params), C.byref(self._bvh),
                                        _stream(stream)))

    FIELDS = ("mu", "quat", "scale", "opacity", "color", "albedo", "rough", "metal")

    def save(self, path):
        """Write the surfel parameters to a .npz file.  The tree is not stored: Scene.load
        builds it again from the parameters."""
        arrays = {f: getattr(self, f).detach().cpu().numpy() for f in self.FIELDS if getattr(self, f) is not None}
        np.savez(path, **arrays)

    @staticmethod
    def load(path, device="cuda", params=None) -> "Scene":
        """A resident scene from a .npz file written by Scene.save (its tree built anew)."""
        with np.load(path) as z:
            missing = [f for f in Scene.FIELDS[:5] if f not in z.files]
            if missing:
                raise ValueError(f"{path}: no {', '.join(missing)}")
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
            return Scene(*[t(z[f]) if f in z.files else None for f in Scene.FIELDS], params=params)

    @staticmethod
    def from_workload(sc, device="cuda", params=None) -> "Scene":
        t = lambda a: torch.from_numpy(a).to(device).contiguous()
        return Scene(t(sc.mu), t(sc.quat), t(sc.scale), t(sc.opacity), t(sc.color), t(sc.albedo), t(sc.rough),
                     t(sc.metal), params=params)

    @property
    def color_dim(self) -> int:
        return int(self.color.shape[1])

    @property
    def handle(self):
        return self._bvh

    def surfels(self) -> L.Surfels:
        return L.Surfels(self.n, self.color_dim, _ptr(self.mu), _ptr(self.quat), _ptr(self.scale),
                         _ptr(self.opacity), _ptr(self.color), _ptr(self.albedo), _ptr(self.rough),
                         _ptr(self.metal))

    def refit(self, stream=None):
        L.check(self._lib.grt_refit_bvh(self._bvh, C.byref(self.surfels()), C.byref(self.params),
                                        _stream(stream)))

    def rebuild(self, stream=None):
        """Full LBVH rebuild in place (same surfel count)."""
        L.check(self._lib.grt_rebuild_bvh(self._bvh, C.byref(self.surfels()), C.byref(self.params),
                                          _stream(stream)))

    def rebuild_noalloc(self, stream=None):
        """Full LBVH rebuild in place that allocates no device memory (fixed library
        scratch, at most GRT_NOALLOC_MAX_SURFELS surfels; calls must not overlap)."""
        L.check(self._lib.grt_rebuild_bvh_noalloc(self._bvh, C.byref(self.surfels()), C.byref(self.params),
                                                  _stream(stream)))

    def info(self) -> dict:
        i = L.BvhInfo()
        L.check(self._lib.grt_bvh_info(self._bvh, C.byref(i)))
        return dict(n_surfels=i.n_surfels, n_nodes=i.n_nodes, device_bytes=i.device_bytes, bounds=list(i.bounds))

    def status(self, stream=None) -> int:
        s = C.c_int32(0)
        L.check(self._lib.grt_bvh_status(self._bvh, C.byref(s), _stream(stream)))
        return s.value

    def close(self):
        if self._bvh:
            self._lib.grt_bvh_destroy(self._bvh)
            self._bvh = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_forward(scene: Scene, ray_o, ray_d, params=None, max_hits: int = 0, stream=None):
    """c_rt[R,3], o_rt[R] (Eq. 8); with max_hits > 0 also hits[R,max_hits], nhits[R]."""
    R = int(ray_o.shape[0])
    _dev(ray_o, name="ray_o", shape=(R, 3))
    _dev(ray_d, name="ray_d", shape=(R, 3))
    dev = ray_o.device
    rgb = torch.empty((R, 3), device=dev)
    op = torch.empty((R,), device=dev)
    hits = torch.empty((R, max_hits), device=dev, dtype=torch.int32) if max_hits > 0 else None
    nh = torch.empty((R,), device=dev, dtype=torch.int32) if max_hits > 0 else None
    p = params if params is not None else scene.params
    L.check(L.load().grt_trace_forward(scene.handle, C.byref(scene.surfels()), C.byref(p), _ptr(ray_o),
                                       _ptr(ray_d), R, _ptr(rgb), _ptr(op), _ptr(hits), max_hits, _ptr(nh),
                                       _stream(stream)))
    return (rgb, op, hits, nh) if max_hits > 0 else (rgb, op)


@dataclasses.dataclass
class SurfelGrads:
    mu: torch.Tensor
    quat: torch.Tensor
    scale: torch.Tensor
    opacity: torch.Tensor
    color: torch.Tensor

    @staticmethod
    def zeros(scene: Scene) -> "SurfelGrads":
        z = lambda t: torch.zeros_like(t)
        return SurfelGrads(z(scene.mu), z(scene.quat), z(scene.scale), z(scene.opacity), z(scene.color))

    def struct(self) -> L.Grads:
        return L.Grads(_ptr(self.mu), _ptr(self.quat), _ptr(self.scale), _ptr(self.opacity), _ptr(self.color))


def trace_backward(scene: Scene, ray_o, ray_d, dL_drgb, dL_dopacity=None, grads: Optional[SurfelGrads] = None,
                   params=None, stream=None) -> SurfelGrads:
    R = int(ray_o.shape[0])
    _dev(ray_o, name="ray_o", shape=(R, 3))
    _dev(ray_d, name="ray_d", shape=(R, 3))
    _dev(dL_drgb, name="dL_drgb", shape=(R, 3))
    _dev(dL_dopacity, name="dL_dopacity", shape=(R,))
    g = grads if grads is not None else SurfelGrads.zeros(scene)
    p = params if params is not None else scene.params
    L.check(L.load().grt_trace_backward(scene.handle, C.byref(scene.surfels()), C.byref(p), _ptr(ray_o),
                                        _ptr(ray_d), R, _ptr(dL_drgb), _ptr(dL_dopacity), C.byref(g.struct()),
                                        _stream(stream)))
    return g


def trace_count(scene: Scene, ray_o, ray_d, params=None, stream=None):
    """(internal nodes visited, surfel records tested, hits composited) summed over rays."""
    R = int(ray_o.shape[0])
    c = torch.zeros(3, dtype=torch.int64, device=ray_o.device)
    p = params if params is not None else scene.params
    L.check(L.load().grt_trace_count(scene.handle, C.byref(scene.surfels()), C.byref(p), _ptr(ray_o), _ptr(ray_d),
                                     R, _ptr(c), _stream(stream)))
    return c


# ----------------------------------------------------------------------------- G-buffer

class GBuffer:
    """Per-pixel shading state (Eq. 9): pos, normal, albedo, rough, metal, valid (+alpha, depth)."""

    def __init__(self, W, H, eye, pos, normal, albedo, rough, metal, valid, alpha=None, depth=None):
        self.W, self.H = int(W), int(H)
        self.eye = tuple(float(x) for x in eye)
        self.pos, self.normal, self.albedo = pos, normal, albedo
        self.rough, self.metal, self.valid = rough, metal, valid
        self.alpha, self.depth = alpha, depth

    @staticmethod
    def empty(W, H, eye, device="cuda") -> "GBuffer":
        P = W * H
        f = lambda *s: torch.empty(s, device=device)
        return GBuffer(W, H, eye, f(P, 3), f(P, 3), f(P, 3), f(P), f(P),
                       torch.empty(P, dtype=torch.int32, device=device), f(P), f(P))

    @staticmethod
    def from_arrays(d: dict, device="cuda") -> "GBuffer":
        t = lambda a, dt=torch.float32: torch.as_tensor(a, dtype=dt).to(device).contiguous()
        return GBuffer(d["W"], d["H"], d["eye"], t(d["pos"]), t(d["normal"]), t(d["albedo"]), t(d["rough"]),
                       t(d["metal"]), t(d["valid"], torch.int32))

    def struct(self) -> L.GBuffer:
        P = self.W * self.H
        for name, t, shp in (("pos", self.pos, (P, 3)), ("normal", self.normal, (P, 3)),
                             ("albedo", self.albedo, (P, 3)), ("rough", self.rough, (P,)),
                             ("metal", self.metal, (P,))):
            _dev(t, name=name, shape=shp)
        _dev(self.valid, dtype=torch.int32, name="valid", shape=(P,))
        return L.GBuffer(_ptr(self.pos), _ptr(self.normal), _ptr(self.albedo), _ptr(self.rough),
                         _ptr(self.metal), _ptr(self.valid), (C.c_float * 3)(*self.eye), self.W, self.H)


def gbuffer_primary(scene: Scene, camera, params=None, out: Optional[GBuffer] = None, stream=None) -> GBuffer:
    """Traced primary G-buffer for a workloads.Camera (eye, target, up, tan_half_fovy, width, height)."""
    W, H = camera.width, camera.height
    g = out if out is not None else GBuffer.empty(W, H, camera.eye, device=scene.mu.device)
    cam = (C.c_float * 10)(*[float(x) for x in camera.as_array()])
    p = params if params is not None else scene.params
    L.check(L.load().grt_gbuffer_primary(scene.handle, C.byref(scene.surfels()), C.byref(p), cam, W, H,
                                         _ptr(g.pos), _ptr(g.normal), _ptr(g.albedo), _ptr(g.rough),
                                         _ptr(g.metal), _ptr(g.alpha), _ptr(g.depth), _ptr(g.valid),
                                         _stream(stream)))
    return g


# ----------------------------------------------------------------------------- environment

class Environment:
    """Equirectangular HDR map rgb[H,W,3] with its proposal tables (grt_env_prepare)."""

    def __init__(self, rgb: torch.Tensor, stream=None):
        H, W = int(rgb.shape[0]), int(rgb.shape[1])
        _dev(rgb, name="rgb", shape=(H, W, 3))
        self.rgb, self.W, self.H = rgb, W, H
        self.prefiltered = None
        lib = L.load()
        nbytes = lib.grt_env_tables_bytes(W, H)
        self.tables = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device=rgb.device)
        L.check(lib.grt_env_prepare(_ptr(rgb), W, H, _ptr(self.tables), _stream(stream)))

    def update(self, rgb: torch.Tensor, stream=None):
        if tuple(rgb.shape) != (self.H, self.W, 3):
            raise ValueError("update needs the same map size")
        self.rgb = _dev(rgb, name="rgb")
        self.prefiltered = None
        L.check(L.load().grt_env_prepare(_ptr(rgb), self.W, self.H, _ptr(self.tables), _stream(stream)))

    def struct(self) -> L.EnvMap:
        return L.EnvMap(self.W, self.H, _ptr(self.tables))

    def prefilter(self, stream=None) -> torch.Tensor:
        """Prefiltered form E of this map for relighting (grt_env_prefilter), cached until
        the next update()."""
        lib = L.load()
        nb = lib.grt_env_prefilter_bytes()
        buf = torch.empty(nb // 4, dtype=torch.float32, device=self.rgb.device)
        L.check(lib.grt_env_prefilter(_ptr(self.rgb), self.W, self.H, _ptr(buf), nb, _stream(stream)))
        self.prefiltered = buf
        return buf


def sampling(n_cos, n_ggx, n_env, seed, brdf=1) -> L.Sampling:
    return L.Sampling(int(n_cos), int(n_ggx), int(n_env), int(brdf), int(seed) & 0xFFFFFFFFFFFFFFFF)


def _workspace(ws):
    """(pointer, bytes) of an optional caller workspace (a CUDA uint8 tensor, 256-byte aligned)."""
    if ws is None:
        return None, 0
    _dev(ws, dtype=torch.uint8, name="workspace")
    return ws.data_ptr(), int(ws.numel())


def shade_workspace_size(n_rays: int) -> int:
    """Workspace bytes of shade_pixels / shade_batch over n_rays ray slots (pixels x N_r)."""
    nb = L.load().grt_shade_workspace_size(int(n_rays))
    if nb == 0:
        raise L.GrtError(L.GRT_ERR_ARG, L.load().grt_last_error().decode())
    return int(nb)


def shade_backward_workspace_size(n_pixels: int, n_cos, n_ggx, n_env, saved: bool = False) -> int:
    """Workspace bytes of shade_backward (recomputing, or with a saved forward record)."""
    s = sampling(n_cos, n_ggx, n_env, 0, 1)
    nb = L.load().grt_shade_backward_workspace_size(int(n_pixels), C.byref(s), int(bool(saved)))
    if nb == 0:
        raise L.GrtError(L.GRT_ERR_ARG, L.load().grt_last_error().decode())
    return int(nb)


def shade_pixels(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None,
                 params=None, outputs=None, light: bool = False, workspace=None, stream=None):
    """MIS shading (Eq. 13): colour[P,3], visibility[P], indirect[P,3] for the pixel list,
    and with light=True also the mean incident radiance light[P,3] of Eq. 16.  `workspace`:
    optional caller buffer (uint8 CUDA tensor of at least shade_workspace_size(P x N_r)
    bytes) used instead of the stream-ordered pool."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    if pixels is not None:
        _dev(pixels, dtype=torch.int32, name="pixels", shape=(n,))
    dev = gb.pos.device
    if outputs is None:
        outputs = (torch.empty((n, 3), device=dev), torch.empty((n,), device=dev), torch.empty((n, 3), device=dev))
    col, vis, ind = outputs[:3]
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    if light:
        lt = outputs[3] if len(outputs) > 3 else torch.empty((n, 3), device=dev)
        L.check(L.load().grt_shade_pixels_light(scene.handle, C.byref(scene.surfels()), C.byref(p),
                                                C.byref(gb.struct()), C.byref(env.struct()), C.byref(s),
                                                _ptr(pixels), n, _ptr(col), _ptr(vis), _ptr(ind), _ptr(lt),
                                                _stream(stream)))
        return col, vis, ind, lt
    wp, wn = _workspace(workspace)
    L.check(L.load().grt_shade_pixels(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                      C.byref(env.struct()), C.byref(s), _ptr(pixels), n, _ptr(col), _ptr(vis),
                                      _ptr(ind), wp, wn, _stream(stream)))
    return col, vis, ind


@dataclasses.dataclass
class MaterialGrads:
    """Gradients into the environment map [H,W,3] and the per-pixel materials."""
    env: torch.Tensor
    albedo: torch.Tensor
    rough: torch.Tensor
    metal: torch.Tensor


def shade_backward_material(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, dL_dcolor,
                            dL_dlight=None, brdf=1, pixels=None, grads: Optional[MaterialGrads] = None, params=None,
                            stream=None) -> MaterialGrads:
    """Adjoint of shade_pixels (colour and the Eq. 16 mean incident radiance) into the map
    and the per-pixel albedo, roughness and metallic; directions and proposal held fixed.
    Gradients accumulate into `grads` (zeros when omitted)."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    _dev(dL_dcolor, name="dL_dcolor", shape=(n, 3))
    _dev(dL_dlight, name="dL_dlight", shape=(n, 3))
    dev = gb.pos.device
    if grads is None:
        grads = MaterialGrads(torch.zeros((env.H, env.W, 3), device=dev), torch.zeros((n, 3), device=dev),
                              torch.zeros(n, device=dev), torch.zeros(n, device=dev))
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    L.check(L.load().grt_shade_backward_material(scene.handle, C.byref(scene.surfels()), C.byref(p),
                                                 C.byref(gb.struct()), C.byref(env.struct()), C.byref(s),
                                                 _ptr(pixels), n, _ptr(dL_dcolor), _ptr(dL_dlight), _ptr(grads.env),
                                                 _ptr(grads.albedo), _ptr(grads.rough), _ptr(grads.metal),
                                                 _stream(stream)))
    return grads


class SavedShade:
    """Forward record of one shading pass kept for its backward (grt_shade_pixels_save):
    per secondary ray its direction, (c_rt, T) and first `max_hits` composited hits.
    Valid for the scene, G-buffer, map, sampling and pixel list it was made with, while the
    surfels stay unchanged."""

    def __init__(self, buf: torch.Tensor, n_pixels: int, sampling_args: tuple, max_hits: int, pixels):
        self.buf = buf
        self.n_pixels = n_pixels
        self.sampling_args = sampling_args
        self.max_hits = max_hits
        self.pixels = pixels

    @property
    def nbytes(self) -> int:
        return int(self.buf.numel())


def shade_saved_bytes(n_pixels: int, n_cos, n_ggx, n_env, max_hits: int = 64) -> int:
    s = sampling(n_cos, n_ggx, n_env, 0, 1)
    nb = L.load().grt_shade_saved_bytes(int(n_pixels), C.byref(s), int(max_hits))
    if nb == 0:
        raise L.GrtError(L.GRT_ERR_ARG, L.load().grt_last_error().decode())
    return int(nb)


def shade_pixels_save(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None,
                      max_hits: int = 64, params=None, outputs=None, workspace=None, stream=None):
    """shade_pixels that also keeps the forward record for shade_backward(saved=...):
    36 + 12 max_hits bytes per ray slot (pixels x N_r) plus an overflow area for rays with
    more hits (192 more hits each for one ray in 256).  Returns (colour, visibility,
    indirect, SavedShade)."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    if pixels is not None:
        _dev(pixels, dtype=torch.int32, name="pixels", shape=(n,))
    dev = gb.pos.device
    if outputs is None:
        outputs = (torch.empty((n, 3), device=dev), torch.empty((n,), device=dev), torch.empty((n, 3), device=dev))
    col, vis, ind = outputs
    nb = shade_saved_bytes(n, n_cos, n_ggx, n_env, max_hits)
    buf = torch.empty(nb, dtype=torch.uint8, device=dev)
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    L.check(L.load().grt_shade_pixels_save(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                           C.byref(env.struct()), C.byref(s), _ptr(pixels), n, _ptr(col), _ptr(vis),
                                           _ptr(ind), int(max_hits), _ptr(buf), nb, *_workspace(workspace),
                                           _stream(stream)))
    return col, vis, ind, SavedShade(buf, n, (n_cos, n_ggx, n_env, seed, brdf), int(max_hits), pixels)


def shade_count(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None,
                params=None, stream=None):
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    c = torch.zeros(3, dtype=torch.int64, device=gb.pos.device)
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    L.check(L.load().grt_shade_count(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                     C.byref(env.struct()), C.byref(s), _ptr(pixels), n, _ptr(c), _stream(stream)))
    return c


def shade_backward(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, dL_dcolor, dL_dvis=None,
                   dL_dind=None, brdf=1, pixels=None, grads: Optional[SurfelGrads] = None, params=None,
                   saved: Optional[SavedShade] = None, workspace=None, stream=None) -> SurfelGrads:
    """Adjoint of shade_pixels w.r.t. the surfels (gradients accumulate into `grads`).
    With `saved` (from shade_pixels_save with the same arguments) the forward record is
    replayed; otherwise samples and hit lists are recomputed.  `workspace`: optional caller
    buffer of at least shade_backward_workspace_size(...) bytes instead of the pool."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    _dev(dL_dcolor, name="dL_dcolor", shape=(n, 3))
    _dev(dL_dvis, name="dL_dvis", shape=(n,))
    _dev(dL_dind, name="dL_dind", shape=(n, 3))
    g = grads if grads is not None else SurfelGrads.zeros(scene)
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    lib = L.load()
    if saved is None:
        L.check(lib.grt_shade_backward(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                       C.byref(env.struct()), C.byref(s), _ptr(pixels), n, _ptr(dL_dcolor),
                                       _ptr(dL_dvis), _ptr(dL_dind), C.byref(g.struct()), *_workspace(workspace),
                                       _stream(stream)))
        return g
    if saved.n_pixels != n or saved.sampling_args != (n_cos, n_ggx, n_env, seed, brdf) or saved.pixels is not pixels:
        raise ValueError("saved record was made with other pixels or sampling")
    L.check(lib.grt_shade_backward_saved(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                         C.byref(env.struct()), C.byref(s), _ptr(pixels), n, _ptr(dL_dcolor),
                                         _ptr(dL_dvis), _ptr(dL_dind), saved.max_hits, _ptr(saved.buf), saved.nbytes,
                                         C.byref(g.struct()), *_workspace(workspace), _stream(stream)))
    return g


@dataclasses.dataclass
class ShadeRequest:
    """One request of a batched shading launch (grt_shade_batch)."""
    scene: Scene
    gbuffer: GBuffer
    env: Environment
    n_cos: int
    n_ggx: int
    n_env: int
    seed: int
    brdf: int = 1
    pixels: Optional[torch.Tensor] = None
    color: Optional[torch.Tensor] = None
    vis: Optional[torch.Tensor] = None
    ind: Optional[torch.Tensor] = None
    pixel_offset: int = 0          # with pixels None: shade pixels [offset, offset + count)
    count: Optional[int] = None

    @property
    def n_pixels(self) -> int:
        if self.pixels is not None:
            return int(self.pixels.shape[0])
        return self.count if self.count is not None else self.gbuffer.W * self.gbuffer.H - self.pixel_offset


def shade_batch(requests, params=None, workspace=None, stream=None):
    """Shade several requests in one persistent launch; fills each request's outputs.
    `workspace`: optional caller buffer of at least shade_workspace_size(total ray slots)."""
    if not requests:
        return
    if len(requests) > L.GRT_MAX_BATCH:
        raise ValueError(f"at most {L.GRT_MAX_BATCH} requests per launch")
    keep = []
    arr = (L.ShadeRequest * len(requests))()
    for i, r in enumerate(requests):
        n = r.n_pixels
        dev = r.gbuffer.pos.device
        if r.color is None:
            r.color = torch.empty((n, 3), device=dev)
        sf = r.scene.surfels()
        keep.append(sf)
        arr[i] = L.ShadeRequest(r.scene.handle, C.pointer(sf), r.gbuffer.struct(), r.env.struct(),
                                sampling(r.n_cos, r.n_ggx, r.n_env, r.seed, r.brdf), _ptr(r.pixels), n,
                                0 if r.pixels is not None else int(r.pixel_offset),
                                _ptr(r.color), _ptr(r.vis), _ptr(r.ind))
    p = params if params is not None else requests[0].scene.params
    L.check(L.load().grt_shade_batch(arr, len(requests), C.byref(p), *_workspace(workspace), _stream(stream)))


def trace_attr(scene: Scene, ray_o, ray_d, params=None, stream=None):
    """Trace_attr (Eq. 14): (V[R], albedo[R,3], rough[R], metal[R], normal[R,3])."""
    R = int(ray_o.shape[0])
    _dev(ray_o, name="ray_o", shape=(R, 3))
    _dev(ray_d, name="ray_d", shape=(R, 3))
    dev = ray_o.device
    V, a, r, m, n = (torch.empty(R, device=dev), torch.empty((R, 3), device=dev), torch.empty(R, device=dev),
                     torch.empty(R, device=dev), torch.empty((R, 3), device=dev))
    p = params if params is not None else scene.params
    L.check(L.load().grt_trace_attr(scene.handle, C.byref(scene.surfels()), C.byref(p), _ptr(ray_o), _ptr(ray_d), R,
                                    _ptr(V), _ptr(a), _ptr(r), _ptr(m), _ptr(n), _stream(stream)))
    return V, a, r, m, n


def shade_relight(scene: Scene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None,
                  params=None, outputs=None, stream=None):
    """MIS relighting under `env` (Eq. 15 in Eq. 13): colour[P,3], visibility[P], indirect[P,3]."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    if pixels is not None:
        _dev(pixels, dtype=torch.int32, name="pixels", shape=(n,))
    dev = gb.pos.device
    if outputs is None:
        outputs = (torch.empty((n, 3), device=dev), torch.empty((n,), device=dev), torch.empty((n, 3), device=dev))
    col, vis, ind = outputs
    pre = env.prefiltered if env.prefiltered is not None else env.prefilter(stream)
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else scene.params
    L.check(L.load().grt_shade_relight(scene.handle, C.byref(scene.surfels()), C.byref(p), C.byref(gb.struct()),
                                       C.byref(env.struct()), _ptr(pre), C.byref(s), _ptr(pixels), n, _ptr(col),
                                       _ptr(vis), _ptr(ind), _stream(stream)))
    return col, vis, ind


class MeshScene:
    """Triangle mesh resident on the device plus its LBVH (grt_build_mesh_bvh): the mesh
    backend of the relighting query.  Tensors: pos[V,3], tri[T,3] (int32), normal[V,3],
    albedo[V,3], rough[V], metal[V]; float32 unless stated, contiguous, on one CUDA device."""

    def __init__(self, pos, tri, normal, albedo, rough, metal, params=None, stream=None):
        nv, nt = int(pos.shape[0]), int(tri.shape[0])
        self.n_vertices, self.n_triangles = nv, nt
        self.pos = _dev(pos, name="pos", shape=(nv, 3))
        self.tri = _dev(tri, dtype=torch.int32, name="tri", shape=(nt, 3))
        self.normal = _dev(normal, name="normal", shape=(nv, 3))
        self.albedo = _dev(albedo, name="albedo", shape=(nv, 3))
        self.rough = _dev(rough, name="rough", shape=(nv,))
        self.metal = _dev(metal, name="metal", shape=(nv,))
        self.params = params if params is not None else trace_params()
        self._bvh = C.c_void_p(None)
        self._lib = L.load()
        L.check(self._lib.grt_build_mesh_bvh(C.byref(self.mesh()), C.byref(self._bvh), _stream(stream)))

    @staticmethod
    def from_workload(m, device="cuda", params=None) -> "MeshScene":
        t = lambda a: torch.from_numpy(a).to(device).contiguous()
        return MeshScene(t(m.pos), t(m.tri.astype("int32")), t(m.normal), t(m.albedo), t(m.rough), t(m.metal),
                         params=params)

    @property
    def handle(self):
        return self._bvh

    def mesh(self) -> L.Mesh:
        return L.Mesh(self.n_vertices, self.n_triangles, _ptr(self.pos), _ptr(self.tri), _ptr(self.normal),
                      _ptr(self.albedo), _ptr(self.rough), _ptr(self.metal))

    def info(self) -> dict:
        i = L.BvhInfo()
        L.check(self._lib.grt_bvh_info(self._bvh, C.byref(i)))
        return dict(n_triangles=i.n_surfels, n_nodes=i.n_nodes, device_bytes=i.device_bytes, bounds=list(i.bounds))

    def status(self, stream=None) -> int:
        s = C.c_int32(0)
        L.check(self._lib.grt_bvh_status(self._bvh, C.byref(s), _stream(stream)))
        return s.value

    def close(self):
        if self._bvh:
            self._lib.grt_bvh_destroy(self._bvh)
            self._bvh = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_trace_attr(mesh: MeshScene, ray_o, ray_d, params=None, stream=None):
    """Trace_attr (Eq. 14), mesh backend: (V[R], albedo[R,3], rough[R], metal[R], normal[R,3])."""
    R = int(ray_o.shape[0])
    _dev(ray_o, name="ray_o", shape=(R, 3))
    _dev(ray_d, name="ray_d", shape=(R, 3))
    dev = ray_o.device
    V, a, r, m, n = (torch.empty(R, device=dev), torch.empty((R, 3), device=dev), torch.empty(R, device=dev),
                     torch.empty(R, device=dev), torch.empty((R, 3), device=dev))
    p = params if params is not None else mesh.params
    L.check(L.load().grt_mesh_trace_attr(mesh.handle, C.byref(mesh.mesh()), C.byref(p), _ptr(ray_o), _ptr(ray_d),
                                         R, _ptr(V), _ptr(a), _ptr(r), _ptr(m), _ptr(n), _stream(stream)))
    return V, a, r, m, n


def shade_relight_mesh(mesh: MeshScene, gb: GBuffer, env: Environment, n_cos, n_ggx, n_env, seed, brdf=1,
                       pixels=None, params=None, outputs=None, stream=None):
    """MIS relighting under `env` (Eq. 15) with the mesh backend answering Eq. 14:
    colour[P,3], visibility[P], indirect[P,3]."""
    n = int(pixels.shape[0]) if pixels is not None else gb.W * gb.H
    if pixels is not None:
        _dev(pixels, dtype=torch.int32, name="pixels", shape=(n,))
    dev = gb.pos.device
    if outputs is None:
        outputs = (torch.empty((n, 3), device=dev), torch.empty((n,), device=dev), torch.empty((n, 3), device=dev))
    col, vis, ind = outputs
    pre = env.prefiltered if env.prefiltered is not None else env.prefilter(stream)
    s = sampling(n_cos, n_ggx, n_env, seed, brdf)
    p = params if params is not None else mesh.params
    L.check(L.load().grt_shade_relight_mesh(mesh.handle, C.byref(mesh.mesh()), C.byref(p), C.byref(gb.struct()),
                                            C.byref(env.struct()), _ptr(pre), C.byref(s), _ptr(pixels), n,
                                            _ptr(col), _ptr(vis), _ptr(ind), _stream(stream)))
    return col, vis, ind


DENOISE_DEFAULTS = dict(radius=3, sigma_s=2.0, sigma_d=1.0, sigma_n=64.0, eps_d=1e-3)


def denoise(color, depth, normal, valid, W: int, H: int, out=None, stream=None, **params):
    """Cross-bilateral denoiser (Sec. III-D) of a W x H image: colour[P,3] guided by
    depth[P], normal[P,3] and valid[P] (int32).  Parameters: radius, sigma_s, sigma_d,
    sigma_n, eps_d (defaults in DENOISE_DEFAULTS)."""
    P_ = int(W) * int(H)
    _dev(color, name="color", shape=(P_, 3))
    _dev(depth, name="depth", shape=(P_,))
    _dev(normal, name="normal", shape=(P_, 3))
    _dev(valid, dtype=torch.int32, name="valid", shape=(P_,))
    q = dict(DENOISE_DEFAULTS)
    q.update(params)
    prm = L.DenoiseParams(int(q["radius"]), float(q["sigma_s"]), float(q["sigma_d"]), float(q["sigma_n"]),
                          float(q["eps_d"]))
    out = torch.empty_like(color) if out is None else _dev(out, name="out", shape=(P_, 3))
    L.check(L.load().grt_denoise(_ptr(color), _ptr(depth), _ptr(normal), _ptr(valid), int(W), int(H),
                                 C.byref(prm), _ptr(out), _stream(stream)))
    return out


def phase_timing(enable: Optional[bool] = None, read: bool = False):
    """Turn per-kernel timing of shading calls on/off; with read=True return the last
    call's (sample_ms, trace_ms, accumulate_ms)."""
    ms = (C.c_float * 3)() if read else None
    L.check(L.load().grt_phase_timing(-1 if enable is None else int(bool(enable)), ms))
    return tuple(ms) if read else None


def adjoint_timing(enable: Optional[bool] = None, read: bool = False):
    """Turn per-kernel timing of adjoint passes on/off; with read=True return the last
    pass's (weights_ms, replay_ms, walk_ms)."""
    ms = (C.c_float * 3)() if read else None
    L.check(L.load().grt_adjoint_timing(-1 if enable is None else int(bool(enable)), ms))
    return tuple(ms) if read else None


def version() -> str:
    return L.load().grt_version().decode()
