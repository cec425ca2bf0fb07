"""Hand-built surfel scenes with closed-form answers (no method arithmetic)."""
import math

import numpy as np

from paper_2607_22780_b300.workloads import Scene

# (w,x,y,z) quaternions of frames whose normal n is an axis
Q_NZ = (1.0, 0.0, 0.0, 0.0)                                   # t_u=x, t_v=y, n=+z
Q_NY = (math.cos(-math.pi / 4), math.sin(-math.pi / 4), 0.0, 0.0)   # n=+y
Q_NX = (math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0)     # n=+x


def scene(surfels, color_dim=3):
    """surfels: list of dicts with mu, quat, scale, opacity, color (+ optional albedo...)."""
    n = len(surfels)
    if n == 0:
        return Scene(mu=np.zeros((0, 3), np.float32), quat=np.zeros((0, 4), np.float32),
                     scale=np.zeros((0, 2), np.float32), opacity=np.zeros(0, np.float32),
                     color=np.zeros((0, color_dim), np.float32), albedo=np.zeros((0, 3), np.float32),
                     rough=np.zeros(0, np.float32), metal=np.zeros(0, np.float32))
    g = lambda k, d: np.array([s.get(k, d) for s in surfels], np.float32)
    return Scene(mu=g("mu", None).reshape(n, 3), quat=g("quat", Q_NZ).reshape(n, 4),
                 scale=g("scale", (0.1, 0.1)).reshape(n, 2), opacity=g("opacity", 0.5).reshape(n),
                 color=g("color", (0.5,) * color_dim).reshape(n, color_dim),
                 albedo=g("albedo", (0.5, 0.5, 0.5)).reshape(n, 3),
                 rough=g("rough", 0.5).reshape(n), metal=g("metal", 0.0).reshape(n))


def gbuffer(pos, normal, albedo, rough, metal, eye, valid=None):
    P = len(pos)
    return dict(pos=np.asarray(pos, np.float32).reshape(P, 3),
                normal=np.asarray(normal, np.float32).reshape(P, 3),
                albedo=np.asarray(albedo, np.float32).reshape(P, 3),
                rough=np.asarray(rough, np.float32).reshape(P),
                metal=np.asarray(metal, np.float32).reshape(P),
                valid=np.ones(P, np.int32) if valid is None else np.asarray(valid, np.int32),
                eye=np.asarray(eye, np.float32), W=P, H=1)


def random_gbuffer(rng, P, eye=(0.0, 0.0, 5.0)):
    n = rng.normal(size=(P, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    pos = rng.uniform(-0.5, 0.5, size=(P, 3))
    # make the normal face the eye so the view direction is above the hemisphere
    v = np.asarray(eye) - pos
    flip = np.sum(n * v, axis=1) < 0
    n[flip] *= -1
    return gbuffer(pos, n, rng.uniform(0.05, 1.0, size=(P, 3)), rng.uniform(0.1, 1.0, P),
                   (rng.uniform(size=P) < 0.5).astype(np.float32), eye)


def icosphere(levels):
    """Closed unit icosphere with shared vertices (each edge split at its midpoint, pushed
    to the sphere), every face wound outwards."""
    g = (1 + 5 ** 0.5) / 2
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    v = [np.array(x, float) / np.linalg.norm(x) for x in v]
    for _ in range(levels):
        mid = {}

        def m_(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                x = v[a] + v[b]
                v.append(x / np.linalg.norm(x))
                mid[k] = len(v) - 1
            return mid[k]
        f = [t for a, b, c in f for t in ((a, m_(a, b), m_(c, a)), (b, m_(b, c), m_(a, b)),
                                          (c, m_(c, a), m_(b, c)), (m_(a, b), m_(b, c), m_(c, a)))]
    return np.array(v), np.array(f)
