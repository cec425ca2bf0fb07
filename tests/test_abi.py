"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares
(no compute calls: this runs without a GPU)."""
import ctypes

import pytest

from paper_2607_22780_b300 import _lib, build


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _lib.header_symbols()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert set(declared) == set(_lib.SIGNATURES), set(declared) ^ set(_lib.SIGNATURES)


def test_version_and_error_calls_without_gpu():
    lib = _lib.load()
    assert b"sm_103a" in lib.grt_version()
    # argument validation fails before touching the device
    out = ctypes.c_void_p()
    rc = lib.grt_build_bvh(None, None, ctypes.byref(out), None)
    assert rc == _lib.GRT_ERR_ARG
    assert b"surfels" in lib.grt_last_error()


def test_bad_params_rejected_without_gpu():
    lib = _lib.load()
    s = _lib.Surfels(0, 3)
    p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 7)   # k = 7 not built
    rc = lib.grt_trace_forward(None, ctypes.byref(s), ctypes.byref(p), None, None, 0, None, None, None, 0, None,
                               None)
    assert rc == _lib.GRT_ERR_ARG  # bvh is NULL comes first
    assert lib.grt_env_tables_bytes(512, 256) >= 512 * 256 * 16
    assert lib.grt_env_tables_bytes(0, 256) == 0


def test_build_passes_checked_without_gpu():
    lib = _lib.load()
    s = _lib.Surfels(0, 3)
    out = ctypes.c_void_p()
    for bad in (-1, _lib.GRT_MAX_BUILD_PASSES + 1):
        p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16, bad)
        assert lib.grt_build_bvh(ctypes.byref(s), ctypes.byref(p), ctypes.byref(out), None) == _lib.GRT_ERR_ARG
        assert b"build_passes" in lib.grt_last_error()
        assert not out.value


def test_gbuffer_k_checked_without_gpu():
    # 0 (chosen by frame size) and the built k-buffer sizes pass; anything else is refused
    # before a request is read
    lib = _lib.load()
    req = (_lib.ShadeRequest * 1)()
    for bad in (-1, 2, 12, 64):
        p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16, 1, bad)
        assert lib.grt_shade_batch(req, 1, ctypes.byref(p), None, 0, None) == _lib.GRT_ERR_UNSUPPORTED
        assert b"gbuffer_k" in lib.grt_last_error()
    p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16, 1, 32)
    rc = lib.grt_shade_batch(req, 1, ctypes.byref(p), ctypes.c_void_p((1 << 20) + 4), 1 << 20, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()  # params accepted


def test_saved_record_size_and_checks_without_gpu():
    lib = _lib.load()
    smp = _lib.Sampling(8, 4, 4, 1, 7)
    R = 1000 * 16
    nb = lib.grt_shade_saved_bytes(1000, ctypes.byref(smp), 16)
    # directions and (c_rt, T) 32 B, hit count 4 B, (id, tau, alpha) 12 B per slot, per ray;
    # an overflow area of max(64, R / 256) slots of 4 + 12 x 192 B
    ov = max(64, R // 256) * (4 + 12 * 192)
    assert R * (36 + 12 * 16) + ov <= nb <= R * (36 + 12 * 16) + ov + 12 * 256
    assert lib.grt_shade_saved_bytes(1000, ctypes.byref(smp), 0) < nb
    assert lib.grt_shade_saved_bytes(1000, ctypes.byref(smp), _lib.GRT_MAX_SAVED_HITS + 1) == 0
    assert b"max_hits" in lib.grt_last_error()
    assert lib.grt_shade_saved_bytes(-1, ctypes.byref(smp), 4) == 0
    # a buffer that is too small (or misaligned) is rejected before any device work
    s = _lib.Surfels(0, 3)
    p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16)
    g, e = _lib.GBuffer(), _lib.EnvMap()
    rc = lib.grt_shade_pixels_save(None, ctypes.byref(s), ctypes.byref(p), ctypes.byref(g), ctypes.byref(e),
                                   ctypes.byref(smp), None, 1000, ctypes.c_void_p(1 << 20), None, None, 16,
                                   ctypes.c_void_p(1 << 20), nb - 1, None, 0, None)
    assert rc == _lib.GRT_ERR_ARG and b"bytes" in lib.grt_last_error()
    rc = lib.grt_shade_backward_saved(None, ctypes.byref(s), ctypes.byref(p), ctypes.byref(g), ctypes.byref(e),
                                      ctypes.byref(smp), None, 1000, ctypes.c_void_p(1 << 20), None, None, 16,
                                      ctypes.c_void_p((1 << 20) + 16), nb, None, None, 0, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()


def test_workspace_sizes_and_checks_without_gpu():
    """Workspace convention of the shading calls: the size queries, and a misaligned or
    undersized caller workspace refused before any device work."""
    lib = _lib.load()
    smp = _lib.Sampling(16, 8, 8, 1, 7)
    R = 640_000 * 32
    nb = lib.grt_shade_workspace_size(R)
    # direction + (c_rt, T) 32 B and the ray order 12 B per slot, plus counters
    assert R * 44 <= nb <= R * 44 + 4_500_000  # plus 2^20 bucket counters and the scan's tile sums
    assert lib.grt_shade_workspace_size(0) > 0
    assert lib.grt_shade_workspace_size(-1) == 0 and b"n_rays" in lib.grt_last_error()
    saved = lib.grt_shade_backward_workspace_size(640_000, ctypes.byref(smp), 1)
    assert saved >= R * 24
    recomp = lib.grt_shade_backward_workspace_size(640_000, ctypes.byref(smp), 0)
    # two chunk buffers of at most 8M rays, each with a 64-hit transient record and its
    # overflow area (one slot of 4 + 12 x 192 bytes per 256 rays)
    chunk = (8 << 20) * (36 + 12 * 64 + 40) + ((8 << 20) // 256) * (4 + 12 * 192)
    assert (8 << 20) * (36 + 12 * 64) < recomp < 2 * chunk + 2 * 4_500_000
    assert lib.grt_shade_backward_workspace_size(-1, ctypes.byref(smp), 0) == 0
    s = _lib.Surfels(0, 3)
    p = _lib.TraceParams(1 / 255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16)
    g, e = _lib.GBuffer(), _lib.EnvMap()
    smp2 = _lib.Sampling(8, 4, 4, 1, 7)
    rc = lib.grt_shade_pixels(None, ctypes.byref(s), ctypes.byref(p), ctypes.byref(g), ctypes.byref(e),
                              ctypes.byref(smp2), None, 10, ctypes.c_void_p(1 << 20), None, None,
                              ctypes.c_void_p((1 << 20) + 64), 1 << 20, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()
    rc = lib.grt_shade_backward(None, ctypes.byref(s), ctypes.byref(p), ctypes.byref(g), ctypes.byref(e),
                                ctypes.byref(smp2), None, 10, ctypes.c_void_p(1 << 20), None, None, None,
                                ctypes.c_void_p((1 << 20) + 8), 1 << 20, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()
    req = (_lib.ShadeRequest * 1)()
    rc = lib.grt_shade_batch(req, 1, ctypes.byref(p), ctypes.c_void_p((1 << 20) + 4), 1 << 20, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()


def test_python_constants_match_the_header():
    # every integer #define of include/grt.h that the binding mirrors has the header's value
    import re
    from pathlib import Path
    hdr = (Path(__file__).resolve().parents[1] / "include" / "grt.h").read_text()
    defines = {}
    for name, expr in re.findall(r"^#define (GRT_\w+)\s+([^/\n]+)", hdr, flags=re.M):
        expr = expr.strip()
        if re.fullmatch(r"[0-9()<>\s]+", expr):
            defines[name] = eval(expr)  # digits, shifts and parentheses only
    assert {"GRT_OK", "GRT_MAX_BATCH", "GRT_GBUFFER_SMALL_FRAME", "GRT_STATUS_BAD_TREE"} <= set(defines)
    mirrored = 0
    for name, value in defines.items():
        for py in (name, name.replace("GRT_", "", 1)):
            if hasattr(_lib, py):
                assert getattr(_lib, py) == value, (name, getattr(_lib, py), value)
                mirrored += 1
                break
    assert mirrored >= 12
