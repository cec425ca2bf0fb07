"""Seeded synthetic inputs for 2D Gaussian ray tracing of secondary rays.

This module only draws inputs: surfel scenes, environment maps, cameras, pixel
subsets and loss targets.  It holds none of the method's arithmetic (no ray
generation, no intersection, no compositing, no sampling of directions, no
shading), so that both the CUDA path and the FP64 oracle can consume the very
same FP32 arrays.

Scene recipes follow the paper's structural parameters (Sec. IV-A: object
centric scenes, 2D Gaussian surfels with tangent frames, opacity, SH colour and
albedo/roughness/metallic) with the sizes of the synthetic workloads:

* ``scene_sphere_plane``  -- 8k surfels on a unit sphere plus a 4x4 ground plane.
* ``scene_objects``       -- 300k surfels on 3 spheres, 2 tori, a box and a plane.
* ``scene_large``         -- 1M/2M surfels: 40x40 plane, 50 primitives, r=50 shell.
* ``mesh_objects``        -- the objects scene's layout as a triangle mesh with per-vertex
                             normals and materials (for the mesh relighting backend).

Every surfel stores: centre mu[3], rotation quaternion (w,x,y,z) whose matrix
columns are (t_u, t_v, n) with n the surface normal, scales (s_u, s_v),
opacity o, colour (RGB or degree-3 SH, 48 = 16 x 3 coefficients), albedo[3],
roughness, metallic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Scene", "Camera", "scene_sphere_plane", "scene_objects", "scene_large",
    "scene_random_soup", "envmap_constant", "envmap_hdr", "camera_orbit",
    "camera_c1", "quat_from_frames", "Mesh", "mesh_objects",
]


@dataclasses.dataclass
class Scene:
    mu: np.ndarray        # [N,3] f32
    quat: np.ndarray      # [N,4] f32 (w,x,y,z), unit up to f32 rounding
    scale: np.ndarray     # [N,2] f32
    opacity: np.ndarray   # [N]   f32
    color: np.ndarray     # [N,C] f32, C = 3 (RGB) or 48 (SH degree 3, [16][3])
    albedo: np.ndarray    # [N,3] f32
    rough: np.ndarray     # [N]   f32
    metal: np.ndarray     # [N]   f32

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @property
    def color_dim(self) -> int:
        return int(self.color.shape[1])

    def arrays(self):
        return dict(mu=self.mu, quat=self.quat, scale=self.scale, opacity=self.opacity,
                    color=self.color, albedo=self.albedo, rough=self.rough, metal=self.metal)

    def subset(self, idx) -> "Scene":
        return Scene(**{k: np.ascontiguousarray(v[idx]) for k, v in self.arrays().items()})

    def save(self, path):
        np.savez(path, **self.arrays())

    @staticmethod
    def load(path) -> "Scene":
        z = np.load(path)
        return Scene(**{k: z[k] for k in ("mu", "quat", "scale", "opacity", "color",
                                          "albedo", "rough", "metal")})


@dataclasses.dataclass
class Camera:
    """Pinhole camera: eye, look-at target, up vector, tan(vertical fov / 2)."""
    eye: tuple
    target: tuple
    up: tuple
    tan_half_fovy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        return np.array([*self.eye, *self.target, *self.up, self.tan_half_fovy], np.float32)


# ----------------------------------------------------------------------------- frames

def quat_from_frames(tu: np.ndarray, tv: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Quaternions (w,x,y,z) of rotation matrices with columns (tu, tv, n).

    Uses the trace-branch conversion of a rotation matrix (Shepperd's method) in
    float64; the result is normalised and stored as float32.
    """
    R = np.stack([tu, tv, n], axis=-1).astype(np.float64)   # [N,3,3], columns
    m00, m11, m22 = R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]
    tr = m00 + m11 + m22
    q = np.empty((R.shape[0], 4), np.float64)
    c0 = tr > 0
    c1 = (~c0) & (m00 >= m11) & (m00 >= m22)
    c2 = (~c0) & (~c1) & (m11 >= m22)
    c3 = (~c0) & (~c1) & (~c2)
    s = np.sqrt(np.maximum(tr[c0] + 1.0, 1e-300)) * 2
    q[c0] = np.stack([0.25 * s, (R[c0, 2, 1] - R[c0, 1, 2]) / s,
                      (R[c0, 0, 2] - R[c0, 2, 0]) / s, (R[c0, 1, 0] - R[c0, 0, 1]) / s], -1)
    s = np.sqrt(np.maximum(1.0 + m00[c1] - m11[c1] - m22[c1], 1e-300)) * 2
    q[c1] = np.stack([(R[c1, 2, 1] - R[c1, 1, 2]) / s, 0.25 * s,
                      (R[c1, 0, 1] + R[c1, 1, 0]) / s, (R[c1, 0, 2] + R[c1, 2, 0]) / s], -1)
    s = np.sqrt(np.maximum(1.0 + m11[c2] - m00[c2] - m22[c2], 1e-300)) * 2
    q[c2] = np.stack([(R[c2, 0, 2] - R[c2, 2, 0]) / s, (R[c2, 0, 1] + R[c2, 1, 0]) / s,
                      0.25 * s, (R[c2, 1, 2] + R[c2, 2, 1]) / s], -1)
    s = np.sqrt(np.maximum(1.0 + m22[c3] - m00[c3] - m11[c3], 1e-300)) * 2
    q[c3] = np.stack([(R[c3, 1, 0] - R[c3, 0, 1]) / s, (R[c3, 0, 2] + R[c3, 2, 0]) / s,
                      (R[c3, 1, 2] + R[c3, 2, 1]) / s, 0.25 * s], -1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _random_tangent_frames(rng: np.random.Generator, n: np.ndarray):
    """Tangent frames (tu, tv) about unit normals n, rotated by a uniform angle."""
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    helper = np.where(np.abs(n[:, 1:2]) < 0.9, np.array([[0.0, 1.0, 0.0]]),
                      np.array([[1.0, 0.0, 0.0]]))
    a = np.cross(helper, n)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(n, a)
    ang = rng.uniform(0.0, 2 * np.pi, size=(n.shape[0], 1))
    tu = np.cos(ang) * a + np.sin(ang) * b
    tv = np.cross(n, tu)
    return tu, tv, n


def _finish(rng, pos, nrm, scale_lo, scale_hi, color_dim, *, rgb_albedo=False,
            rough=None, metal=None) -> Scene:
    N = pos.shape[0]
    tu, tv, n = _random_tangent_frames(rng, nrm.astype(np.float64))
    quat = quat_from_frames(tu, tv, n)
    scale = np.exp(rng.uniform(np.log(scale_lo), np.log(scale_hi), size=(N, 2))).astype(np.float32)
    opacity = rng.beta(5.0, 2.0, size=N).astype(np.float32)
    if color_dim == 3:
        color = rng.uniform(0.0, 1.0, size=(N, 3)).astype(np.float32)
    else:
        color = rng.normal(0.0, 0.3, size=(N, 48)).astype(np.float32)
    albedo = color.copy() if (rgb_albedo and color_dim == 3) else \
        rng.uniform(0.0, 1.0, size=(N, 3)).astype(np.float32)
    if rough is None:
        rough = rng.uniform(0.05, 1.0, size=N).astype(np.float32)
    if metal is None:
        metal = (rng.uniform(size=N) < 0.3).astype(np.float32)
    return Scene(mu=np.ascontiguousarray(pos, np.float32), quat=quat, scale=scale,
                 opacity=opacity, color=np.ascontiguousarray(color), albedo=albedo,
                 rough=np.asarray(rough, np.float32), metal=np.asarray(metal, np.float32))


# ----------------------------------------------------------------------------- shapes

def _sphere(rng, k, centre, radius, inward=False):
    v = rng.normal(size=(k, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pos = np.asarray(centre) + radius * v
    return pos, (-v if inward else v)


def _plane_y(rng, k, y, half_x, half_z, cx=0.0, cz=0.0):
    pos = np.stack([rng.uniform(cx - half_x, cx + half_x, k), np.full(k, float(y)),
                    rng.uniform(cz - half_z, cz + half_z, k)], 1)
    nrm = np.tile(np.array([[0.0, 1.0, 0.0]]), (k, 1))
    return pos, nrm


def _torus(rng, k, centre, R, r, axis):
    """Uniform-by-area samples on a torus (rejection on the area element)."""
    us, vs = [], []
    while sum(len(u) for u in us) < k:
        m = 2 * k
        u = rng.uniform(0, 2 * np.pi, m)
        v = rng.uniform(0, 2 * np.pi, m)
        keep = rng.uniform(0, R + r, m) < (R + r * np.cos(v))
        us.append(u[keep]); vs.append(v[keep])
    u = np.concatenate(us)[:k]; v = np.concatenate(vs)[:k]
    loc = np.stack([(R + r * np.cos(v)) * np.cos(u), r * np.sin(v), (R + r * np.cos(v)) * np.sin(u)], 1)
    nl = np.stack([np.cos(v) * np.cos(u), np.sin(v), np.cos(v) * np.sin(u)], 1)
    # rotate local +y onto `axis`
    ax = np.asarray(axis, np.float64); ax /= np.linalg.norm(ax)
    y = np.array([0.0, 1.0, 0.0])
    c = float(np.dot(y, ax)); w = np.cross(y, ax); s = np.linalg.norm(w)
    if s < 1e-12:
        Rm = np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    else:
        w /= s
        K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        Rm = np.eye(3) + s * K + (1 - c) * K @ K
    return loc @ Rm.T + np.asarray(centre), nl @ Rm.T


def _box(rng, k, centre, half):
    """Uniform samples on the surface of an axis-aligned cube."""
    face = rng.integers(0, 6, k)
    a = rng.uniform(-half, half, k); b = rng.uniform(-half, half, k)
    pos = np.zeros((k, 3)); nrm = np.zeros((k, 3))
    ax = face // 2; sgn = np.where(face % 2 == 0, 1.0, -1.0)
    for d in range(3):
        sel = ax == d
        o1, o2 = [e for e in range(3) if e != d]
        pos[sel, d] = sgn[sel] * half
        pos[sel, o1] = a[sel]; pos[sel, o2] = b[sel]
        nrm[sel, d] = sgn[sel]
    return pos + np.asarray(centre), nrm


def _alloc(total, areas):
    areas = np.asarray(areas, np.float64)
    cnt = np.floor(total * areas / areas.sum()).astype(np.int64)
    cnt[np.argmax(areas)] += total - cnt.sum()
    return cnt


# ----------------------------------------------------------------------------- scenes

def scene_sphere_plane(n: int = 8000, seed: int = 2607) -> Scene:
    """8k RGB surfels: unit sphere at the origin plus a 4x4 plane at y=-1.

    Split by area (4*pi vs 16).  Scales log-uniform [0.01, 0.05], opacity
    Beta(5,2), RGB uniform [0,1] (albedo = colour), roughness 1, metallic 0.
    """
    rng = np.random.default_rng(seed)
    k_s, k_p = _alloc(n, [4 * np.pi, 16.0])
    p1, n1 = _sphere(rng, k_s, (0, 0, 0), 1.0)
    p2, n2 = _plane_y(rng, k_p, -1.0, 2.0, 2.0)
    pos = np.concatenate([p1, p2]); nrm = np.concatenate([n1, n2])
    return _finish(rng, pos, nrm, 0.01, 0.05, 3, rgb_albedo=True,
                   rough=np.ones(n, np.float32), metal=np.zeros(n, np.float32))


def _place_objects(rng, specs, lim, floor_y):
    """Seeded rejection placement of bounding circles (x,z) without overlap."""
    placed = []
    for rad in specs:
        for _ in range(10000):
            c = rng.uniform(-lim + rad, lim - rad, 2)
            if all(np.hypot(*(c - p)) > rad + pr + 0.02 for p, pr in placed):
                placed.append((c, rad))
                break
        else:
            placed.append((rng.uniform(-lim, lim, 2), rad))
    return [np.array([c[0], floor_y, c[1]]) for c, _ in placed]


def scene_objects(n: int = 300_000, seed: int = 2607, color_dim: int = 48) -> Scene:
    """300k surfels: 3 spheres, 2 tori, a box and an 8x8 ground plane.

    Sphere radii U[0.3,0.6]; tori R=0.5, r=0.15 with random axes; box side 0.6;
    objects rest on the plane y=-1 inside |x|,|z| <= 2 without overlap.  Surfels
    are allocated by area; scales log-uniform [0.002, 0.02]; SH degree 3 with
    coefficients N(0, 0.3); albedo U[0,1]^3; roughness U[0.05,1]; metallic
    Bernoulli(0.3).
    """
    rng = np.random.default_rng(seed)
    radii = rng.uniform(0.3, 0.6, 3)
    Rt, rt = 0.5, 0.15
    half = 0.3
    foot = list(radii) + [Rt + rt, Rt + rt, half * np.sqrt(2)]
    centres = _place_objects(rng, foot, 2.0, -1.0)
    axes = [rng.normal(size=3) for _ in range(2)]
    areas = [4 * np.pi * r * r for r in radii] + [4 * np.pi ** 2 * Rt * rt] * 2 + \
        [6 * (2 * half) ** 2, 64.0]
    cnt = _alloc(n, areas)
    parts = []
    for i in range(3):
        parts.append(_sphere(rng, cnt[i], centres[i] + [0, radii[i], 0], radii[i]))
    for j in range(2):
        parts.append(_torus(rng, cnt[3 + j], centres[3 + j] + [0, Rt + rt, 0], Rt, rt, axes[j]))
    parts.append(_box(rng, cnt[5], centres[5] + [0, half, 0], half))
    parts.append(_plane_y(rng, cnt[6], -1.0, 4.0, 4.0))
    pos = np.concatenate([p for p, _ in parts]); nrm = np.concatenate([q for _, q in parts])
    return _finish(rng, pos, nrm, 0.002, 0.02, color_dim)


@dataclasses.dataclass
class Mesh:
    """Triangle mesh with per-vertex attributes (float32 / int32, contiguous)."""
    pos: np.ndarray      # [V, 3]
    tri: np.ndarray      # [T, 3] vertex indices
    normal: np.ndarray   # [V, 3] unit
    albedo: np.ndarray   # [V, 3]
    rough: np.ndarray    # [V]
    metal: np.ndarray    # [V]


def _rot_y_to(axis):
    ax = np.asarray(axis, np.float64); ax = ax / np.linalg.norm(ax)
    y = np.array([0.0, 1.0, 0.0])
    c = float(np.dot(y, ax)); w = np.cross(y, ax); s = np.linalg.norm(w)
    if s < 1e-12:
        return np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    w /= s
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    return np.eye(3) + s * K + (1 - c) * K @ K


def _grid_tris(nu, nv, wrap_u, wrap_v, base):
    """Two triangles per cell of an nu x nv vertex grid (index u * nv + v)."""
    cu = nu if wrap_u else nu - 1
    cv = nv if wrap_v else nv - 1
    u, v = np.meshgrid(np.arange(cu), np.arange(cv), indexing="ij")
    u1 = (u + 1) % nu; v1 = (v + 1) % nv
    a = u * nv + v; b = u1 * nv + v; c = u1 * nv + v1; d = u * nv + v1
    return np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)]) + base


def mesh_objects(seed: int = 2607, res: int = 64) -> Mesh:
    """The layout of ``scene_objects`` (same seed: same radii, positions and torus axes) as a
    triangle mesh: UV spheres and tori of res x 2 res vertices, cube faces and the 8x8 ground
    plane as res x res grids.  Per vertex: analytic normal, albedo U[0,1]^3, roughness
    U[0.05,1], metallic Bernoulli(0.3)."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(0.3, 0.6, 3)
    Rt, rt = 0.5, 0.15
    half = 0.3
    foot = list(radii) + [Rt + rt, Rt + rt, half * np.sqrt(2)]
    centres = _place_objects(rng, foot, 2.0, -1.0)
    axes = [rng.normal(size=3) for _ in range(2)]
    P, N, T = [], [], []
    nv_ = 0

    def add(pos, nrm, tris):
        nonlocal nv_
        P.append(pos); N.append(nrm); T.append(tris + nv_)
        nv_ += pos.shape[0]

    nl, nlon = res, 2 * res
    for i in range(3):
        th = np.pi * (np.arange(nl) + 0.5) / nl
        ph = 2 * np.pi * np.arange(nlon) / nlon
        TH, PH = np.meshgrid(th, ph, indexing="ij")
        d = np.stack([np.sin(TH) * np.sin(PH), np.cos(TH), np.sin(TH) * np.cos(PH)], -1).reshape(-1, 3)
        c = centres[i] + [0, radii[i], 0]
        # poles closed by the first and last rings' fans
        top = c + [0, radii[i], 0]; bot = c - [0, radii[i], 0]
        pos = np.concatenate([c + radii[i] * d, [top, bot]])
        nrm = np.concatenate([d, [[0, 1.0, 0], [0, -1.0, 0]]])
        tris = _grid_tris(nl, nlon, False, True, 0)
        k = np.arange(nlon)
        ti, bi = nl * nlon, nl * nlon + 1
        fan_t = np.stack([np.full(nlon, ti), k, (k + 1) % nlon], -1)
        fan_b = np.stack([np.full(nlon, bi), (nl - 1) * nlon + (k + 1) % nlon, (nl - 1) * nlon + k], -1)
        add(pos, nrm, np.concatenate([tris, fan_t, fan_b]))
    for j in range(2):
        u = 2 * np.pi * np.arange(2 * res) / (2 * res)
        v = 2 * np.pi * np.arange(res) / res
        U, Vv = np.meshgrid(u, v, indexing="ij")
        loc = np.stack([(Rt + rt * np.cos(Vv)) * np.cos(U), rt * np.sin(Vv), (Rt + rt * np.cos(Vv)) * np.sin(U)], -1)
        nn = np.stack([np.cos(Vv) * np.cos(U), np.sin(Vv), np.cos(Vv) * np.sin(U)], -1)
        Rm = _rot_y_to(axes[j])
        c = centres[3 + j] + [0, Rt + rt, 0]
        add(loc.reshape(-1, 3) @ Rm.T + c, nn.reshape(-1, 3) @ Rm.T, _grid_tris(2 * res, res, True, True, 0))
    g = np.linspace(-1.0, 1.0, res)
    A, B = np.meshgrid(g, g, indexing="ij")
    cb = centres[5] + [0, half, 0]
    for d in range(3):
        o1, o2 = [e for e in range(3) if e != d]
        for sgn in (1.0, -1.0):
            pos = np.zeros((res * res, 3))
            pos[:, d] = sgn * half
            pos[:, o1] = half * A.reshape(-1)
            pos[:, o2] = half * B.reshape(-1)
            nrm = np.zeros((res * res, 3)); nrm[:, d] = sgn
            add(pos + cb, nrm, _grid_tris(res, res, False, False, 0))
    pos = np.zeros((res * res, 3))
    pos[:, 0] = 4.0 * A.reshape(-1); pos[:, 1] = -1.0; pos[:, 2] = 4.0 * B.reshape(-1)
    nrm = np.tile([0.0, 1.0, 0.0], (res * res, 1))
    add(pos, nrm, _grid_tris(res, res, False, False, 0))
    pos = np.concatenate(P); nrm = np.concatenate(N); tri = np.concatenate(T)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    V = pos.shape[0]
    return Mesh(pos=np.ascontiguousarray(pos, np.float32), tri=np.ascontiguousarray(tri, np.int32),
                normal=np.ascontiguousarray(nrm, np.float32),
                albedo=rng.uniform(0.0, 1.0, (V, 3)).astype(np.float32),
                rough=rng.uniform(0.05, 1.0, V).astype(np.float32),
                metal=(rng.uniform(size=V) < 0.3).astype(np.float32))


def scene_large(n: int = 2_000_000, seed: int = 2607, color_dim: int = 48) -> Scene:
    """Large unbounded scene: 40x40 plane (45%), 50 primitives (35%), r=50 shell (20%).

    Primitives are spheres, boxes and tori with size U[0.2,2] inside
    |x|,|z| <= 18; the background shell has inward normals.  Scales log-uniform
    [0.001, 0.1]; appearance and materials as in ``scene_objects``.
    """
    rng = np.random.default_rng(seed)
    n_plane = int(0.45 * n); n_shell = int(0.20 * n); n_obj = n - n_plane - n_shell
    kinds = rng.integers(0, 3, 50)
    sizes = rng.uniform(0.2, 2.0, 50)
    areas = np.where(kinds == 0, 4 * np.pi * sizes ** 2,
                     np.where(kinds == 1, 6 * (2 * sizes) ** 2, 4 * np.pi ** 2 * sizes * 0.3 * sizes))
    cnt = _alloc(n_obj, areas)
    parts = [_plane_y(rng, n_plane, -1.0, 20.0, 20.0)]
    for i in range(50):
        c = np.array([rng.uniform(-18, 18), -1.0 + sizes[i], rng.uniform(-18, 18)])
        if kinds[i] == 0:
            parts.append(_sphere(rng, cnt[i], c, sizes[i]))
        elif kinds[i] == 1:
            parts.append(_box(rng, cnt[i], c, sizes[i]))
        else:
            parts.append(_torus(rng, cnt[i], c, sizes[i], 0.3 * sizes[i], rng.normal(size=3)))
    parts.append(_sphere(rng, n_shell, (0, 0, 0), 50.0, inward=True))
    pos = np.concatenate([p for p, _ in parts]); nrm = np.concatenate([q for _, q in parts])
    return _finish(rng, pos, nrm, 0.001, 0.1, color_dim)


def scene_random_soup(n: int, seed: int, extent: float = 1.0, scale_lo: float = 0.05,
                      scale_hi: float = 0.3, color_dim: int = 3) -> Scene:
    """Small randomly oriented surfels in a cube: used for gradient checks.

    Normals are uniform on the sphere, so no two surfels are coplanar and depth
    order is unambiguous almost surely.
    """
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-extent, extent, size=(n, 3))
    nrm = rng.normal(size=(n, 3))
    return _finish(rng, pos, nrm, scale_lo, scale_hi, color_dim)


# ----------------------------------------------------------------------------- lighting

def envmap_constant(value: float = 1.0, width: int = 16, height: int = 8) -> np.ndarray:
    """Constant environment map [H, W, 3]."""
    return np.full((height, width, 3), value, np.float32)


def envmap_hdr(seed: int, width: int = 512, height: int = 256, sigma: float = 1.5,
               sun_gain: float = 200.0, sun_width: float = 0.002) -> np.ndarray:
    """Log-normal HDR equirectangular map [H, W, 3] with one sun lobe.

    Texel (row, col) covers polar angle theta in [pi*row/H, pi*(row+1)/H] from
    +y and azimuth phi in [2*pi*col/W, 2*pi*(col+1)/W] with direction
    (sin t sin p, cos t, sin t cos p).  Log-luminance N(0, sigma) i.i.d. per
    texel, grey times a per-texel tint U[0.9,1.1]^3, plus a sun with
    elevation U[20,70] degrees adding sun_gain*exp((cos g - 1)/sun_width).
    """
    rng = np.random.default_rng(seed)
    grey = np.exp(rng.normal(0.0, sigma, size=(height, width, 1)))
    tint = rng.uniform(0.9, 1.1, size=(height, width, 3))
    env = grey * tint
    elev = np.deg2rad(rng.uniform(20.0, 70.0)); az = rng.uniform(0, 2 * np.pi)
    sun = np.array([np.cos(elev) * np.sin(az), np.sin(elev), np.cos(elev) * np.cos(az)])
    th = np.pi * (np.arange(height) + 0.5) / height
    ph = 2 * np.pi * (np.arange(width) + 0.5) / width
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.sin(P), np.cos(T), np.sin(T) * np.cos(P)], -1)
    cosg = d @ sun
    env = env + (sun_gain * np.exp((cosg - 1.0) / sun_width))[..., None]
    return np.ascontiguousarray(env, np.float32)


# ----------------------------------------------------------------------------- cameras

def camera_c1(width: int = 64, height: int = 64) -> Camera:
    """Pinhole at distance 3, 20 degrees above the horizon, 60 degree vertical fov."""
    e = math.radians(20.0)
    return Camera(eye=(0.0, 3 * math.sin(e), 3 * math.cos(e)), target=(0.0, 0.0, 0.0),
                  up=(0.0, 1.0, 0.0), tan_half_fovy=math.tan(math.radians(30.0)),
                  width=width, height=height)


def camera_orbit(seed: int, width: int, height: int, distance: float = 3.0,
                 fovy_deg: float = 60.0, target=(0.0, -0.3, 0.0)) -> Camera:
    """Seeded camera on a sphere of given distance, elevation U[15,45] degrees."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0, 2 * np.pi); el = np.deg2rad(rng.uniform(15.0, 45.0))
    t = np.asarray(target, np.float64)
    eye = t + distance * np.array([np.cos(el) * np.sin(az), np.sin(el), np.cos(el) * np.cos(az)])
    return Camera(eye=tuple(float(x) for x in eye), target=tuple(float(x) for x in t),
                  up=(0.0, 1.0, 0.0), tan_half_fovy=math.tan(math.radians(fovy_deg / 2)),
                  width=width, height=height)


def target_image(seed: int, height: int, width: int) -> np.ndarray:
    """Seeded U[0,1]^3 target image for the L2 loss."""
    return np.random.default_rng(seed).uniform(0, 1, size=(height, width, 3)).astype(np.float32)
