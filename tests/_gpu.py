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
