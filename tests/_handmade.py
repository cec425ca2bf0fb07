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
