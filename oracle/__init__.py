"""FP64 brute-force oracle for 2D Gaussian ray tracing of secondary rays.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product path never
calls it and shares no code with it.

The arithmetic lives in ``grt_oracle.c`` (plain C, FP64, OpenMP over rays); this
module compiles it with gcc on first use and marshals numpy arrays.  Every
function takes a :class:`paper_2607_22780_b300.workloads.Scene`-like object
(attributes mu, quat, scale, opacity, color, albedo, rough, metal).

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FLAG_ALPHA_MIN = 1
FLAG_ALPHA_MAX = 2
FLAG_T_MIN = 4
FLAG_VALID = 8
# audit flags (audit_rays / audit_pixels): near-boundary causes of an FP32/FP64 decision split
AUDIT_TIE = 16
AUDIT_PLANE_TIE = 32
AUDIT_RANGE = 64
AUDIT_GRAZE = 128
AUDIT_HORIZON = 256
AUDIT_DIR = 512


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int), ("color_dim", C.c_int)] + \
        [(k, C.POINTER(C.c_double)) for k in ("mu", "quat", "scale", "opacity", "color",
                                              "albedo", "rough", "metal")]


class _Params(C.Structure):
    _fields_ = [(k, C.c_float) for k in ("alpha_min", "alpha_max", "t_min", "t_max", "T_min", "eps_nd")]


class _GBuf(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_float)) for k in ("pos", "normal", "albedo", "rough", "metal")] + \
        [("valid", C.POINTER(C.c_int32)), ("eye", C.POINTER(C.c_float)), ("W", C.c_int), ("H", C.c_int)]


class _Env(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("rgb", C.POINTER(C.c_float))]


class _Sampling(C.Structure):
    _fields_ = [("n_cos", C.c_int), ("n_ggx", C.c_int), ("n_env", C.c_int),
                ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("brdf", C.c_int)]


class _Grads(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in ("g_mu", "g_quat", "g_scale", "g_opacity", "g_color")]


def _declare(L):
    P = C.c_void_p
    L.or_trace_rays.argtypes = [P, P, C.c_int, P, P, P, P, P, C.c_int, P, P, P, C.c_int]
    L.or_gbuffer.argtypes = [P, P, P, C.c_int, C.c_int, P, C.c_int] + [P] * 9 + [C.c_int]
    L.or_shade_pixels.argtypes = [P, P, P, P, P, P, C.c_int, P, P, P, P, P, C.c_int]
    L.or_backward_material.argtypes = [P, P, P, P, P, P, C.c_int, P, P, P, P, P, P, P, C.c_int]
    L.or_backward_rays.argtypes = [P, P, C.c_int, P, P, P, P, P, P, C.c_int]
    L.or_backward_pixels.argtypes = [P, P, P, P, P, P, C.c_int, P, P, P, P, P, C.c_int]
    L.or_audit_rays.argtypes = [P, P, C.c_int, P, P, P, C.c_int, P, P, P, P, P, C.c_int]
    L.or_audit_pixels.argtypes = [P, P, P, P, P, P, C.c_int, C.c_int, P, P, P, P, P, C.c_int]
    L.or_sample_direction_d64.argtypes = [P, P, P, P, P, C.c_float, C.c_int, C.c_int, P, P]
    L.or_philox4x32_10.argtypes = [P, P, P]
    L.or_sincos2pi.argtypes = [C.c_float, P, P]
    L.or_atan2f.argtypes = [C.c_float, C.c_float]
    L.or_atan2f.restype = C.c_float
    L.or_texel_of.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int, C.c_int, P, P]
    L.or_env_tables_f32.argtypes = [C.c_int, C.c_int, P, P, P]
    L.or_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, P]
    L.or_pdf_ggx.argtypes = [P, P, C.c_double, P]
    L.or_pdf_ggx.restype = C.c_double
    L.or_brdf.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_int, P]
    L.or_sample_direction.argtypes = [P, P, P, P, P, C.c_float, C.c_int, C.c_int, P]
    L.or_sample_many.argtypes = [C.c_int, P, P, P, C.c_float, C.c_uint32, C.c_int, P, P]
    L.or_pdf_env_dir.argtypes = [P, P]
    L.or_pdf_env_dir.restype = C.c_double
    L.or_camera_ray.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
    L.or_normal_from_quat.argtypes = [P, P]
    L.or_env_prefilter.argtypes = [C.c_int, C.c_int, P, P, P, P]
    L.or_splitsum_many.argtypes = [C.c_int, P, P, P, P, P, C.c_int, C.c_int, P, P, P, P, P]
    L.or_trace_attr.argtypes = [P, P, C.c_int, P, P, P, P, P, P, P, P, C.c_int]
    L.or_shade_relight.argtypes = [P, P, P, P, P, P, P, P, P, C.c_int, P, P, P, P, C.c_int]
    L.or_mesh_trace_attr.argtypes = [P, P, C.c_int, P, P, P, P, P, P, P, P, C.c_int]
    L.or_shade_relight_mesh.argtypes = [P, P, P, P, P, P, P, P, P, C.c_int, P, P, P, P, C.c_int]
    L.or_denoise.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                             C.c_double, P, C.c_int]


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Keep:
    """Holds numpy arrays alive while ctypes structs point into them."""

    def __init__(self):
        self.refs = []

    def f(self, a):
        a = _f32(a)
        self.refs.append(a)
        return _fp(a)

    def d(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))


def _scene(sc, keep):
    s = _Scene()
    s.n = int(sc.mu.shape[0])
    s.color_dim = int(sc.color.shape[1])
    for k in ("mu", "quat", "scale", "opacity", "color", "albedo", "rough", "metal"):
        setattr(s, k, keep.d(getattr(sc, k)))
    return s


DEFAULT_PARAMS = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=0.01, t_max=3.0e38,
                      T_min=1e-4, eps_nd=1e-6)


def _params(p):
    q = dict(DEFAULT_PARAMS)
    if p:
        q.update(p)
    return _Params(*[float(q[k]) for k, _ in _Params._fields_])


def _gbuf(gb, keep):
    g = _GBuf()
    for k in ("pos", "normal", "albedo", "rough", "metal"):
        setattr(g, k, keep.f(gb[k]))
    v = np.ascontiguousarray(gb["valid"], np.int32)
    keep.refs.append(v)
    g.valid = v.ctypes.data_as(C.POINTER(C.c_int32))
    g.eye = keep.f(np.asarray(gb["eye"], np.float32))
    g.W = int(gb["W"]); g.H = int(gb["H"])
    return g


def _env(env, keep):
    e = _Env()
    e.H, e.W = int(env.shape[0]), int(env.shape[1])
    e.rgb = keep.f(env)
    return e


def _sampling(n_cos, n_ggx, n_env, seed, brdf):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return _Sampling(int(n_cos), int(n_ggx), int(n_env), seed & 0xFFFFFFFF, seed >> 32, int(brdf))


def _ref(x):
    return C.byref(x)


# ----------------------------------------------------------------------------- API

def trace_rays(scene, ray_o, ray_d, params=None, max_hits=64, nthreads=0):
    """Trace rays (Eq. 8).  Returns dict rgb[R,3], opacity[R], T[R], hits[R,max_hits],
    nhits[R], flags[R] (FP64 values, int32 ids)."""
    keep = _Keep()
    ro, rd = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R = ro.shape[0]
    rgb = np.zeros((R, 3)); op = np.zeros(R); T = np.zeros(R)
    hits = np.full((R, max(max_hits, 1)), -1, np.int32); nh = np.zeros(R, np.int32)
    fl = np.zeros(R, np.uint32)
    s = _scene(scene, keep); P = _params(params)
    lib().or_trace_rays(_ref(s), _ref(P), R, _ptr(ro), _ptr(rd), _ptr(rgb), _ptr(op), _ptr(T),
                        max_hits, _ptr(hits), _ptr(nh), _ptr(fl), nthreads)
    return dict(rgb=rgb, opacity=op, T=T, hits=hits, nhits=nh, flags=fl)


def audit_rays(scene, ray_o, ray_d, ray_d64=None, params=None, max_hits=64, nthreads=0):
    """The rays traced twice: list A with the FP32 decisions of every other function here
    (plane test and depth order of Eq. 7-8), list B with those decisions in FP64 (along
    ray_d64 when given).  Returns dict hits_a, n_a, hits_b, n_b (composited ids and counts)
    and flags (FLAG_* / AUDIT_* near-boundary causes, each from an a-priori bound)."""
    keep = _Keep()
    ro, rd = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R = ro.shape[0]
    d64 = None if ray_d64 is None else np.ascontiguousarray(ray_d64, np.float64).reshape(R, 3)
    out = dict(hits_a=np.full((R, max_hits), -1, np.int32), n_a=np.zeros(R, np.int32),
               hits_b=np.full((R, max_hits), -1, np.int32), n_b=np.zeros(R, np.int32), flags=np.zeros(R, np.uint32))
    s = _scene(scene, keep); P = _params(params)
    lib().or_audit_rays(_ref(s), _ref(P), R, _ptr(ro), _ptr(rd), _ptr(d64), max_hits, _ptr(out["hits_a"]),
                        _ptr(out["n_a"]), _ptr(out["hits_b"]), _ptr(out["n_b"]), _ptr(out["flags"]), nthreads)
    return out


def audit_pixels(scene, gb, env, n_cos, n_ggx, n_env, seed, pixels, brdf=1, params=None, max_hits=64, nthreads=0):
    """audit_rays for the MIS shading rays of `pixels` (slot i * N_r + j = sample j of
    pixels[i]): list A from the FP32 sampler and decisions, list B from an FP64 sampler
    (same uniforms and texel choice, libm trigonometry) and FP64 decisions.  n_a = n_b = -1
    marks a slot with no sample on either side."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params); g = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    pl = np.ascontiguousarray(pixels, np.int32)
    R = pl.shape[0] * (n_cos + n_ggx + n_env)
    out = dict(hits_a=np.full((R, max_hits), -1, np.int32), n_a=np.zeros(R, np.int32),
               hits_b=np.full((R, max_hits), -1, np.int32), n_b=np.zeros(R, np.int32), flags=np.zeros(R, np.uint32))
    lib().or_audit_pixels(_ref(s), _ref(P), _ref(g), _ref(e), _ref(S), _ptr(pl), pl.shape[0], max_hits,
                          _ptr(out["hits_a"]), _ptr(out["n_a"]), _ptr(out["hits_b"]), _ptr(out["n_b"]),
                          _ptr(out["flags"]), nthreads)
    return out


def gbuffer(scene, camera, params=None, pixels=None, nthreads=0):
    """Primary G-buffer of a pinhole camera (Eq. 9 along the camera ray).

    With `pixels` (raster indices y*W + x) only those pixels are traced; row i of every
    output then belongs to pixels[i]."""
    keep = _Keep()
    W, H = camera.width, camera.height
    if pixels is None:
        pl = None
        P_ = W * H
    else:
        pl = np.ascontiguousarray(pixels, np.int32)
        if pl.size and (pl.min() < 0 or pl.max() >= W * H):
            raise ValueError("pixel index outside the image")
        P_ = pl.shape[0]
    out = dict(pos=np.zeros((P_, 3)), normal=np.zeros((P_, 3)), albedo=np.zeros((P_, 3)),
               rough=np.zeros(P_), metal=np.zeros(P_), alpha=np.zeros(P_), depth=np.zeros(P_),
               valid=np.zeros(P_, np.int32), flags=np.zeros(P_, np.uint32))
    s = _scene(scene, keep); P = _params(params)
    cam = _f32(camera.as_array())
    lib().or_gbuffer(_ref(s), _ref(P), _ptr(cam), W, H, _ptr(pl), P_, _ptr(out["pos"]), _ptr(out["normal"]),
                     _ptr(out["albedo"]), _ptr(out["rough"]), _ptr(out["metal"]), _ptr(out["alpha"]),
                     _ptr(out["depth"]), _ptr(out["valid"]), _ptr(out["flags"]), nthreads)
    out["eye"] = np.asarray(camera.eye, np.float32)
    out["W"], out["H"] = W, H
    return out


def gbuffer_f32(gb):
    """The G-buffer as the FP32 arrays both sides shade from."""
    return dict(pos=_f32(gb["pos"]), normal=_f32(gb["normal"]), albedo=_f32(gb["albedo"]),
                rough=_f32(gb["rough"]), metal=_f32(gb["metal"]),
                valid=np.ascontiguousarray(gb["valid"], np.int32),
                eye=np.asarray(gb["eye"], np.float32), W=int(gb["W"]), H=int(gb["H"]))


def shade_pixels(scene, gb, env, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None, params=None,
                 nthreads=0):
    """MIS shading (Eq. 13).  Returns dict color[P,3], vis[P], ind[P,3], light[P,3] (the
    mean incident radiance of Eq. 16), flags[P]."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params); g = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    if pixels is None:
        pl = None; n = int(gb["W"]) * int(gb["H"])
    else:
        pl = np.ascontiguousarray(pixels, np.int32); n = pl.shape[0]
    col = np.zeros((n, 3)); vis = np.zeros(n); ind = np.zeros((n, 3)); fl = np.zeros(n, np.uint32)
    light = np.zeros((n, 3))
    lib().or_shade_pixels(_ref(s), _ref(P), _ref(g), _ref(e), _ref(S), _ptr(pl), n, _ptr(col),
                          _ptr(vis), _ptr(ind), _ptr(light), _ptr(fl), nthreads)
    return dict(color=col, vis=vis, ind=ind, light=light, flags=fl)


def backward_material(scene, gb, env, n_cos, n_ggx, n_env, seed, dL_dcolor, dL_dlight=None, brdf=1, pixels=None,
                      params=None, nthreads=0):
    """Adjoint of the MIS estimate (Eq. 13) and of the mean incident radiance (Eq. 16) with
    respect to the map and the per-pixel materials, directions and proposal held fixed.
    Returns dict env[H,W,3], albedo[n,3], rough[n], metal[n], flags[n]."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params); g = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    if pixels is None:
        pl = None; n = int(gb["W"]) * int(gb["H"])
    else:
        pl = np.ascontiguousarray(pixels, np.int32); n = pl.shape[0]
    H, W = np.asarray(env).shape[:2]
    dc = np.ascontiguousarray(dL_dcolor, np.float64).reshape(n, 3)
    dl = None if dL_dlight is None else np.ascontiguousarray(dL_dlight, np.float64).reshape(n, 3)
    out = dict(env=np.zeros((H, W, 3)), albedo=np.zeros((n, 3)), rough=np.zeros(n), metal=np.zeros(n),
               flags=np.zeros(n, np.uint32))
    lib().or_backward_material(_ref(s), _ref(P), _ref(g), _ref(e), _ref(S), _ptr(pl), n, _ptr(dc), _ptr(dl),
                               _ptr(out["env"]), _ptr(out["albedo"]), _ptr(out["rough"]), _ptr(out["metal"]),
                               _ptr(out["flags"]), nthreads)
    return out


def _grads(scene):
    N = scene.mu.shape[0]
    return dict(mu=np.zeros((N, 3)), quat=np.zeros((N, 4)), scale=np.zeros((N, 2)),
                opacity=np.zeros(N), color=np.zeros((N, scene.color.shape[1])))


def _grads_struct(g):
    return _Grads(*[g[k].ctypes.data_as(C.POINTER(C.c_double))
                    for k in ("mu", "quat", "scale", "opacity", "color")])


def backward_rays(scene, ray_o, ray_d, dL_drgb, dL_dopacity, params=None, nthreads=0):
    """Analytic FP64 gradient of sum(dL_drgb*c_rt + dL_dopacity*o_rt) w.r.t. surfels."""
    keep = _Keep()
    ro, rd = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R = ro.shape[0]
    a = np.ascontiguousarray(dL_drgb, np.float64).reshape(R, 3)
    b = np.ascontiguousarray(dL_dopacity, np.float64).reshape(R)
    g = _grads(scene); gs = _grads_struct(g)
    fl = np.zeros(R, np.uint32)
    s = _scene(scene, keep); P = _params(params)
    lib().or_backward_rays(_ref(s), _ref(P), R, _ptr(ro), _ptr(rd), _ptr(a), _ptr(b), _ref(gs),
                           _ptr(fl), nthreads)
    g["flags"] = fl
    return g


def backward_pixels(scene, gb, env, n_cos, n_ggx, n_env, seed, dL_dcolor, dL_dvis=None,
                    dL_dind=None, brdf=1, pixels=None, params=None, nthreads=0):
    """Analytic FP64 gradient of the shaded outputs w.r.t. surfels (pixel mode)."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params); gbs = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    if pixels is None:
        pl = None; n = int(gb["W"]) * int(gb["H"])
    else:
        pl = np.ascontiguousarray(pixels, np.int32); n = pl.shape[0]
    dc = np.ascontiguousarray(dL_dcolor, np.float64).reshape(n, 3)
    dv = None if dL_dvis is None else np.ascontiguousarray(dL_dvis, np.float64).reshape(n)
    di = None if dL_dind is None else np.ascontiguousarray(dL_dind, np.float64).reshape(n, 3)
    g = _grads(scene); gs = _grads_struct(g)
    fl = np.zeros(n, np.uint32)
    lib().or_backward_pixels(_ref(s), _ref(P), _ref(gbs), _ref(e), _ref(S), _ptr(pl), n, _ptr(dc),
                             _ptr(dv), _ptr(di), _ref(gs), _ptr(fl), nthreads)
    g["flags"] = fl
    return g


# ----------------------------------------------------------------------------- helpers

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32); k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sincos2pi(t):
    s = C.c_float(); c = C.c_float()
    lib().or_sincos2pi(float(t), C.byref(s), C.byref(c))
    return s.value, c.value


def atan2f(y, x):
    return lib().or_atan2f(float(y), float(x))


def texel_of(d, W, H):
    r = C.c_int(); c = C.c_int()
    lib().or_texel_of(float(d[0]), float(d[1]), float(d[2]), W, H, C.byref(r), C.byref(c))
    return r.value, c.value


def env_tables_f32(env):
    H, W = env.shape[:2]
    marg = np.zeros(H + 1, np.float32); cond = np.zeros((H, W + 1), np.float32)
    e = _f32(env)
    lib().or_env_tables_f32(W, H, _ptr(e), _ptr(marg), _ptr(cond))
    return marg, cond


def sh_basis(d):
    Y = np.zeros(16)
    lib().or_sh_basis(float(d[0]), float(d[1]), float(d[2]), _ptr(Y))
    return Y


def pdf_ggx(wo, n, rough, wi):
    a = [np.ascontiguousarray(v, np.float64) for v in (wo, n, wi)]
    return lib().or_pdf_ggx(_ptr(a[0]), _ptr(a[1]), float(rough), _ptr(a[2]))


def brdf(wo, wi, n, albedo, rough, metal, mode=1):
    a = [np.ascontiguousarray(v, np.float64) for v in (wo, wi, n, albedo)]
    f = np.zeros(3)
    lib().or_brdf(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), float(rough), float(metal),
                  int(mode), _ptr(f))
    return f


def sample_many(proposal, env, nrm, wo, rough, seed, count):
    """Directions of one proposal (0 cosine, 1 GGX, 2 environment) without horizon cut."""
    keep = _Keep()
    e = _env(env, keep)
    n = _f32(nrm); w = _f32(wo)
    out = np.zeros((count, 3), np.float32); ok = np.zeros(count, np.int32)
    lib().or_sample_many(int(proposal), _ref(e), _ptr(n), _ptr(w), float(rough), int(seed), count,
                         _ptr(out), _ptr(ok))
    return out, ok


def pdf_env(env, w):
    keep = _Keep()
    e = _env(env, keep)
    ww = _f32(w)
    return lib().or_pdf_env_dir(_ref(e), _ptr(ww))


def camera_ray(camera, px, py):
    cam = _f32(camera.as_array())
    o = np.zeros(3, np.float32); d = np.zeros(3, np.float32)
    lib().or_camera_ray(_ptr(cam), camera.width, camera.height, px, py, _ptr(o), _ptr(d))
    return o, d


def camera_rays(camera):
    W, H = camera.width, camera.height
    o = np.zeros((H * W, 3), np.float32); d = np.zeros((H * W, 3), np.float32)
    for p in range(W * H):
        o[p], d[p] = camera_ray(camera, p % W, p // W)
    return o, d


def normal_from_quat(q):
    qq = _f32(q); n = np.zeros(3, np.float32)
    lib().or_normal_from_quat(_ptr(qq), _ptr(n))
    return n


def denoise(color, depth, normal, valid, W, H, radius=3, sigma_s=2.0, sigma_d=1.0, sigma_n=64.0, eps_d=1e-3,
            nthreads=0):
    """Cross-bilateral denoiser (Sec. III-D) in FP64: colour[P,3], depth[P], normal[P,3],
    valid[P] of a W x H image -> denoised colour[P,3]."""
    P_ = int(W) * int(H)
    col = np.ascontiguousarray(color, np.float64).reshape(P_, 3)
    dep = np.ascontiguousarray(depth, np.float64).reshape(P_)
    nrm = np.ascontiguousarray(normal, np.float64).reshape(P_, 3)
    val = np.ascontiguousarray(valid, np.int32).reshape(P_)
    out = np.zeros((P_, 3))
    lib().or_denoise(_ptr(col), _ptr(dep), _ptr(nrm), _ptr(val), int(W), int(H), int(radius), float(sigma_s),
                     float(sigma_d), float(sigma_n), float(eps_d), _ptr(out), nthreads)
    return out


# ----------------------------------------------------------------------------- relighting

DIFF_W, DIFF_H, SPEC_W, SPEC_H, SPEC_LEVELS, LUT_N = 32, 16, 64, 32, 6, 32


def env_prefilter(env):
    """Prefiltered form E of a novel map (Sec. III-E, Eq. 15): diffuse grid [16,32,3],
    specular levels r = 0.2..1 [5,32,64,3], split-sum BRDF table [32 (nv), 32 (r), 2]."""
    e = _f32(env)
    H, W = e.shape[:2]
    diff = np.zeros((DIFF_H, DIFF_W, 3))
    spec = np.zeros((SPEC_LEVELS - 1, SPEC_H, SPEC_W, 3))
    lut = np.zeros((LUT_N, LUT_N, 2))
    lib().or_env_prefilter(W, H, _ptr(e), _ptr(diff), _ptr(spec), _ptr(lut))
    return dict(diff=diff, spec=spec, lut=lut, env=e)


def splitsum(pre, albedo, rough, metal, normal, view):
    """SplitSum(a, r, m, n, E) seen from direction `view`, for arrays of N surface states."""
    a = np.ascontiguousarray(albedo, np.float64).reshape(-1, 3)
    n_ = a.shape[0]
    r = np.ascontiguousarray(rough, np.float64).reshape(n_)
    m = np.ascontiguousarray(metal, np.float64).reshape(n_)
    nr = np.ascontiguousarray(normal, np.float64).reshape(n_, 3)
    v = np.ascontiguousarray(view, np.float64).reshape(n_, 3)
    e = pre["env"]
    out = np.zeros((n_, 3))
    lib().or_splitsum_many(n_, _ptr(a), _ptr(r), _ptr(m), _ptr(nr), _ptr(v), e.shape[1], e.shape[0], _ptr(e),
                           _ptr(pre["diff"]), _ptr(pre["spec"]), _ptr(pre["lut"]), _ptr(out))
    return out


def trace_attr(scene, ray_o, ray_d, params=None, nthreads=0):
    """Trace_attr (Eq. 14), Gaussian backend: V[R], albedo[R,3], rough[R], metal[R], normal[R,3]."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params)
    ro = _f32(ray_o).reshape(-1, 3); rd = _f32(ray_d).reshape(-1, 3)
    R = ro.shape[0]
    out = dict(V=np.zeros(R), albedo=np.zeros((R, 3)), rough=np.zeros(R), metal=np.zeros(R),
               normal=np.zeros((R, 3)), flags=np.zeros(R, np.uint32))
    lib().or_trace_attr(_ref(s), _ref(P), R, _ptr(ro), _ptr(rd), _ptr(out["V"]), _ptr(out["albedo"]),
                        _ptr(out["rough"]), _ptr(out["metal"]), _ptr(out["normal"]), _ptr(out["flags"]), nthreads)
    return out


def shade_relight(scene, gb, env, pre, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None, params=None, nthreads=0):
    """MIS relighting (Eq. 15 in Eq. 13) under the novel map `env` with its prefiltered
    form `pre` (env_prefilter).  Returns dict color[P,3], vis[P], ind[P,3], flags[P]."""
    keep = _Keep()
    s = _scene(scene, keep); P = _params(params); g = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    if pixels is None:
        pl = None; n = int(gb["W"]) * int(gb["H"])
    else:
        pl = np.ascontiguousarray(pixels, np.int32); n = pl.shape[0]
    col = np.zeros((n, 3)); vis = np.zeros(n); ind = np.zeros((n, 3)); fl = np.zeros(n, np.uint32)
    lib().or_shade_relight(_ref(s), _ref(P), _ref(g), _ref(e), _ptr(pre["diff"]), _ptr(pre["spec"]),
                           _ptr(pre["lut"]), _ref(S), _ptr(pl), n, _ptr(col), _ptr(vis), _ptr(ind), _ptr(fl),
                           nthreads)
    return dict(color=col, vis=vis, ind=ind, flags=fl)



# ----------------------------------------------------------------------------- mesh backend

class _Mesh(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("pos", C.c_void_p), ("tri", C.c_void_p), ("normal", C.c_void_p),
                ("albedo", C.c_void_p), ("rough", C.c_void_p), ("metal", C.c_void_p)]


def _mesh(m, keep):
    arrs = [_f32(m.pos), np.ascontiguousarray(m.tri, np.int32), _f32(m.normal), _f32(m.albedo), _f32(m.rough),
            _f32(m.metal)]
    keep.refs.extend(arrs)
    return _Mesh(arrs[0].shape[0], arrs[1].shape[0], *[_ptr(a) for a in arrs])


def mesh_trace_attr(mesh, ray_o, ray_d, params=None, nthreads=0):
    """Trace_attr (Eq. 14), mesh backend: V[R] (0 hit, 1 miss), albedo[R,3], rough[R],
    metal[R], normal[R,3], flags[R] (always 0: the hit is decided in FP32, as in the kernel,
    by the watertight ray/triangle test)."""
    keep = _Keep()
    m = _mesh(mesh, keep); P = _params(params)
    ro = _f32(ray_o).reshape(-1, 3); rd = _f32(ray_d).reshape(-1, 3)
    R = ro.shape[0]
    out = dict(V=np.zeros(R), albedo=np.zeros((R, 3)), rough=np.zeros(R), metal=np.zeros(R),
               normal=np.zeros((R, 3)), flags=np.zeros(R, np.uint32))
    lib().or_mesh_trace_attr(_ref(m), _ref(P), R, _ptr(ro), _ptr(rd), _ptr(out["V"]), _ptr(out["albedo"]),
                             _ptr(out["rough"]), _ptr(out["metal"]), _ptr(out["normal"]), _ptr(out["flags"]),
                             nthreads)
    return out


def shade_relight_mesh(mesh, gb, env, pre, n_cos, n_ggx, n_env, seed, brdf=1, pixels=None, params=None, nthreads=0):
    """MIS relighting (Eq. 15) with the mesh backend of Eq. 14."""
    keep = _Keep()
    m = _mesh(mesh, keep); P = _params(params); g = _gbuf(gb, keep); e = _env(env, keep)
    S = _sampling(n_cos, n_ggx, n_env, seed, brdf)
    if pixels is None:
        pl = None; n = int(gb["W"]) * int(gb["H"])
    else:
        pl = np.ascontiguousarray(pixels, np.int32); n = pl.shape[0]
    col = np.zeros((n, 3)); vis = np.zeros(n); ind = np.zeros((n, 3)); fl = np.zeros(n, np.uint32)
    lib().or_shade_relight_mesh(_ref(m), _ref(P), _ref(g), _ref(e), _ptr(pre["diff"]), _ptr(pre["spec"]),
                                _ptr(pre["lut"]), _ref(S), _ptr(pl), n, _ptr(col), _ptr(vis), _ptr(ind), _ptr(fl),
                                nthreads)
    return dict(color=col, vis=vis, ind=ind, flags=fl)
