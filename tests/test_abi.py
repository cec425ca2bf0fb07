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


def test_saved_record_size_and_checks_without_gpu():
    lib = _lib.load()
    smp = _lib.Sampling(8, 4, 4, 1, 7)
    R = 1000 * 16
    nb = lib.grt_shade_saved_bytes(1000, ctypes.byref(smp), 16)
    # directions and (c_rt, T) 32 B, hit count 4 B, (id, tau, alpha) 12 B per slot, per ray
    assert R * (36 + 12 * 16) <= nb <= R * (36 + 12 * 16) + 7 * 256
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
                                   ctypes.c_void_p(1 << 20), nb - 1, None)
    assert rc == _lib.GRT_ERR_ARG and b"bytes" in lib.grt_last_error()
    rc = lib.grt_shade_backward_saved(None, ctypes.byref(s), ctypes.byref(p), ctypes.byref(g), ctypes.byref(e),
                                      ctypes.byref(smp), None, 1000, ctypes.c_void_p(1 << 20), None, None, 16,
                                      ctypes.c_void_p((1 << 20) + 16), nb, None, None)
    assert rc == _lib.GRT_ERR_ARG and b"aligned" in lib.grt_last_error()
