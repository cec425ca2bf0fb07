"""The allocation-free BVH rebuild (grt_rebuild_bvh_noalloc) against the ordinary one.

Callers that cannot let a library allocate device memory -- an application that owns and
pre-reserves the whole device budget -- rebuild their BVH through this entry point, whose
sort scratch is a fixed array inside libgrt.  This file is collected last on purpose.
It checks, through the C ABI, that two rebuilds in a row (the second one reusing the
array the first one left behind, on a different scene size) trace exactly like
grt_rebuild_bvh, that a scene above the fixed limit is refused before any GPU work, and
that a call draws nothing from the device's memory pool or from cudaMalloc.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2607_22780_b300 import _lib as L
from paper_2607_22780_b300 import api, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-4  # radiance tolerance used by the trace parity tests


def _rays(seed, R=4096):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-2.0, 2.0, size=(R, 3))
    d = rng.uniform(-1.0, 1.0, size=(R, 3)) - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (torch.as_tensor(o, dtype=torch.float32, device="cuda").contiguous(),
            torch.as_tensor(d, dtype=torch.float32, device="cuda").contiguous())


def _trace(S, o, d):
    rgb, op, hits, nh = api.trace_forward(S, o, d, max_hits=32)
    torch.cuda.synchronize()
    return rgb, op, hits, nh


def _noalloc(S):
    lib = L.load()
    rc = lib.grt_rebuild_bvh_noalloc(S.handle, ctypes.byref(S.surfels()), ctypes.byref(S.params),
                                     torch.cuda.current_stream().cuda_stream)
    L.check(rc)


@pytest.mark.parametrize("order", [(200_000, 37_000), (37_000, 200_000)])
def test_noalloc_rebuild_matches_allocating_rebuild_twice(order):
    for n in order:
        sc = wl.scene_objects(n, seed=n)
        S = api.Scene.from_workload(sc)
        o, d = _rays(n)
        S.rebuild()
        ref = _trace(S, o, d)
        for _ in range(2):            # two calls in a row share the scratch array
            _noalloc(S)
            got = _trace(S, o, d)
            assert torch.equal(got[2], ref[2]) and torch.equal(got[3], ref[3])
            assert float((got[0] - ref[0]).abs().max()) <= TOL
            assert float((got[1] - ref[1]).abs().max()) <= TOL
        assert S.status() == 0
        S.close()


def test_noalloc_rejects_scenes_above_the_limit():
    n = L.GRT_NOALLOC_MAX_SURFELS + 1
    sc = wl.scene_random_soup(n, seed=1, extent=1.0, scale_lo=0.001, scale_hi=0.002)
    S = api.Scene.from_workload(sc)
    rc = L.load().grt_rebuild_bvh_noalloc(S.handle, ctypes.byref(S.surfels()), ctypes.byref(S.params), None)
    assert rc == L.GRT_ERR_ARG
    assert b"exceeds" in L.load().grt_last_error()
    S.close()


def test_noalloc_rebuild_allocates_no_device_memory():
    """The defining property: after the first call (which looks up the scratch address),
    a rebuild leaves the device's default pool and its free memory untouched."""
    from cuda.bindings import driver as dr, runtime as rt

    sc = wl.scene_objects(100_000, seed=3)
    S = api.Scene.from_workload(sc)
    _noalloc(S)                                   # first call on the device: address lookup
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    A = rt.cudaMemPoolAttr

    def attr(a):
        e, v = rt.cudaMemPoolGetAttribute(pool, a)
        assert e == rt.cudaError_t.cudaSuccess
        return int(v)

    used0 = attr(A.cudaMemPoolAttrUsedMemCurrent)
    reserved0 = attr(A.cudaMemPoolAttrReservedMemCurrent)
    (e,) = rt.cudaMemPoolSetAttribute(pool, A.cudaMemPoolAttrUsedMemHigh, dr.cuuint64_t(0))
    assert e == rt.cudaError_t.cudaSuccess
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        _noalloc(S)
    torch.cuda.synchronize()
    assert attr(A.cudaMemPoolAttrUsedMemHigh) <= used0
    assert attr(A.cudaMemPoolAttrReservedMemCurrent) == reserved0
    assert torch.cuda.mem_get_info()[0] == free0
    # the allocating rebuild, for contrast, does draw its sort scratch from the pool
    S.rebuild()
    torch.cuda.synchronize()
    assert attr(A.cudaMemPoolAttrUsedMemHigh) > used0
    assert S.status() == 0
    S.close()
