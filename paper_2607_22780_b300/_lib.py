"""ctypes view of libgrt (include/grt.h).  Argument marshalling only.

The library is built in-tree by ``paper_2607_22780_b300.build``; loading fails loudly
when it is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrt.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "grt.h")

GRT_OK, GRT_ERR_ARG, GRT_ERR_OOM, GRT_ERR_CUDA, GRT_ERR_OVERFLOW, GRT_ERR_TIMEOUT, GRT_ERR_UNSUPPORTED = range(7)
GRT_MAX_BATCH = 48
GRT_NOALLOC_MAX_SURFELS = 524288
GRT_MAX_SAVED_HITS = 64
GRT_MAX_BUILD_PASSES = 4
GRT_GBUFFER_SMALL_FRAME = 3 << 18
GRT_DENOISE_MAX_RADIUS = 8
STATUS_STACK_OVERFLOW = 1
STATUS_NONFINITE = 2
STATUS_BAD_TREE = 4
STATUS_BAD_INDEX = 8

P = C.c_void_p


class Surfels(C.Structure):
    _fields_ = [("n", C.c_int32), ("color_dim", C.c_int32)] + \
        [(k, P) for k in ("mu", "quat", "scale", "opacity", "color", "albedo", "rough", "metal")]


class TraceParams(C.Structure):
    _fields_ = [(k, C.c_float) for k in ("alpha_min", "alpha_max", "t_min", "t_max", "T_min", "eps_nd")] + \
        [("k", C.c_int32), ("build_passes", C.c_int32), ("gbuffer_k", C.c_int32)]


class BvhInfo(C.Structure):
    _fields_ = [("n_surfels", C.c_int32), ("n_nodes", C.c_int32), ("device_bytes", C.c_size_t),
                ("bounds", C.c_float * 6)]


class Grads(C.Structure):
    _fields_ = [(k, P) for k in ("mu", "quat", "scale", "opacity", "color")]


class Mesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_triangles", C.c_int32)] + \
        [(k, P) for k in ("pos", "tri", "normal", "albedo", "rough", "metal")]


class EnvMap(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("tables", P)]


class GBuffer(C.Structure):
    _fields_ = [(k, P) for k in ("pos", "normal", "albedo", "rough", "metal", "valid")] + \
        [("eye", C.c_float * 3), ("W", C.c_int32), ("H", C.c_int32)]


class Sampling(C.Structure):
    _fields_ = [("n_cos", C.c_int32), ("n_ggx", C.c_int32), ("n_env", C.c_int32), ("brdf", C.c_int32),
                ("seed", C.c_uint64)]


class DenoiseParams(C.Structure):
    _fields_ = [("radius", C.c_int32), ("sigma_s", C.c_float), ("sigma_d", C.c_float), ("sigma_n", C.c_float),
                ("eps_d", C.c_float)]


class ShadeRequest(C.Structure):
    _fields_ = [("bvh", P), ("surfels", C.POINTER(Surfels)), ("gbuffer", GBuffer), ("env", EnvMap),
                ("sampling", Sampling), ("pixel_list", P), ("n_pixels", C.c_int32),
                ("pixel_offset", C.c_int32), ("out_color", P), ("out_vis", P), ("out_ind", P)]


# name -> (restype, argtypes)
SIGNATURES = {
    "grt_build_bvh": (C.c_int, [C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(P), P]),
    "grt_refit_bvh": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P]),
    "grt_rebuild_bvh": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P]),
    "grt_rebuild_bvh_noalloc": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P]),
    "grt_bvh_destroy": (None, [P]),
    "grt_bvh_info": (C.c_int, [P, C.POINTER(BvhInfo)]),
    "grt_bvh_status": (C.c_int, [P, C.POINTER(C.c_int32), P]),
    "grt_trace_forward": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P, P, C.c_int32, P, P, P,
                                    C.c_int32, P, P]),
    "grt_trace_backward": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P, P, C.c_int32, P, P,
                                     C.POINTER(Grads), P]),
    "grt_gbuffer_primary": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(C.c_float),
                                      C.c_int32, C.c_int32, P, P, P, P, P, P, P, P, P]),
    "grt_env_tables_bytes": (C.c_size_t, [C.c_int32, C.c_int32]),
    "grt_env_prepare": (C.c_int, [P, C.c_int32, C.c_int32, P, P]),
    "grt_shade_workspace_size": (C.c_size_t, [C.c_int64]),
    "grt_shade_backward_workspace_size": (C.c_size_t, [C.c_int32, C.POINTER(Sampling), C.c_int32]),
    "grt_shade_pixels": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                   C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P, P, C.c_size_t,
                                   P]),
    "grt_shade_backward": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                     C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P,
                                     C.POINTER(Grads), P, C.c_size_t, P]),
    "grt_shade_saved_bytes": (C.c_size_t, [C.c_int32, C.POINTER(Sampling), C.c_int32]),
    "grt_shade_pixels_save": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                        C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P,
                                        C.c_int32, P, C.c_size_t, P, C.c_size_t, P]),
    "grt_shade_backward_saved": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                           C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P,
                                           C.c_int32, P, C.c_size_t, C.POINTER(Grads), P, C.c_size_t, P]),
    "grt_shade_pixels_light": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                         C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P, P, P]),
    "grt_shade_backward_material": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                              C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P, P, P,
                                              P, P, P]),
    "grt_shade_batch": (C.c_int, [C.POINTER(ShadeRequest), C.c_int32, C.POINTER(TraceParams), P, C.c_size_t, P]),
    "grt_trace_count": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P, P, C.c_int32, P, P]),
    "grt_shade_count": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                  C.POINTER(EnvMap), C.POINTER(Sampling), P, C.c_int32, P, P]),
    "grt_phase_timing": (C.c_int, [C.c_int32, C.POINTER(C.c_float)]),
    "grt_adjoint_timing": (C.c_int, [C.c_int32, C.POINTER(C.c_float)]),
    "grt_denoise": (C.c_int, [P, P, P, P, C.c_int32, C.c_int32, C.POINTER(DenoiseParams), P, P]),
    "grt_trace_attr": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), P, P, C.c_int32, P, P, P, P, P, P]),
    "grt_env_prefilter_bytes": (C.c_size_t, []),
    "grt_env_prefilter": (C.c_int, [P, C.c_int32, C.c_int32, P, C.c_size_t, P]),
    "grt_shade_relight": (C.c_int, [P, C.POINTER(Surfels), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                    C.POINTER(EnvMap), P, C.POINTER(Sampling), P, C.c_int32, P, P, P, P]),
    "grt_build_mesh_bvh": (C.c_int, [C.POINTER(Mesh), C.POINTER(P), P]),
    "grt_mesh_trace_attr": (C.c_int, [P, C.POINTER(Mesh), C.POINTER(TraceParams), P, P, C.c_int32, P, P, P, P, P,
                                      P]),
    "grt_shade_relight_mesh": (C.c_int, [P, C.POINTER(Mesh), C.POINTER(TraceParams), C.POINTER(GBuffer),
                                         C.POINTER(EnvMap), P, C.POINTER(Sampling), P, C.c_int32, P, P, P, P]),
    "grt_last_error": (C.c_char_p, []),
    "grt_version": (C.c_char_p, []),
}


def header_symbols(path: str = HEADER):
    """Function names declared in include/grt.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(grt_[a-z_]+)\s*\(", txt)))


_lib = None


class GrtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"grt error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libgrt.so (raises OSError when the built library is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"{path} is missing: build it with `python -m paper_2607_22780_b300.build`")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != GRT_OK:
        raise GrtError(rc, load().grt_last_error().decode())
