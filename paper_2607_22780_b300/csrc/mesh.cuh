// mesh.cuh -- mesh backend of the relighting query (Sec. III-E): closest triangle hit in the
// 4-wide LBVH built by grt_build_mesh_bvh, and the barycentric attributes of Eq. 14.
//
// Leaf records (64 bytes, one triangle): (v0, triangle id), (v1 - v0), (v2 - v0), unused.
// Intersection by the Moeller-Trumbore test; the nearest t in (t_min, t_max) wins, equal t
// by triangle index.  The walk visits children near to far and culls every box beyond the
// nearest hit found so far.
#pragma once

#include "relight.cuh"
#include "trace.cuh"

namespace grt {

struct MeshDev {
    const int* tri;
    const float *normal, *albedo, *rough, *metal;
    int nv;
};

struct MeshHit {
    int id;       // triangle index, -1 for a miss
    float u, v;   // barycentrics of v1 and v2
};

__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ void mesh_test_leaf(const DevBvh& bvh, int ref, const RayState& r, float tmin, float tmax,
                                               float& best, MeshHit& h) {
    const int first = leaf_first(ref), count = leaf_count(ref);
    if (first + count > bvh.n) {
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        return;
    }
    for (int i = 0; i < count; ++i) {
        const float4* R = bvh.records + 4 * (size_t)(first + i);
        const float4 r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2);
        const f3 e1 = mk3(r1.x, r1.y, r1.z), e2 = mk3(r2.x, r2.y, r2.z);
        const f3 pv = cross3(r.d, e2);
        const float det = dot3(e1, pv);
        if (!(fabsf(det) >= 1e-12f * sqrtf(dot3(e1, e1) * dot3(e2, e2)))) continue;
        const float inv = 1.f / det;
        const f3 sv = mk3(r.o.x - r0.x, r.o.y - r0.y, r.o.z - r0.z);
        const float u = dot3(sv, pv) * inv;
        if (u < 0.f || u > 1.f) continue;
        const f3 qv = cross3(sv, e1);
        const float v = dot3(r.d, qv) * inv;
        if (v < 0.f || u + v > 1.f) continue;
        const float t = dot3(e2, qv) * inv;
        if (!(t > tmin && t < tmax)) continue;
        const int id = __float_as_int(r0.w);
        if (t < best || (t == best && id < h.id)) {
            best = t;
            h.id = id;
            h.u = u;
            h.v = v;
        }
    }
}

// Closest hit of the ray (o, d) with t in (tmin, tmax).
__device__ __forceinline__ MeshHit mesh_closest(const DevBvh& bvh, f3 o, f3 d, float tmin, float tmax) {
    MeshHit h{-1, 0.f, 0.f};
    if (bvh.n == 0 || bvh.root == kRefEmpty) return h;
    const RayState r = make_ray(o, d);
    float best = tmax;
    if (bvh.root < 0) {  // a single triangle
        mesh_test_leaf(bvh, bvh.root, r, tmin, tmax, best, h);
        return h;
    }
    int2 stack[kStackDepth];
    int sp = 0, node = bvh.root, budget = bvh.cap + 8;
    const float tlo = fmaf(tmin, 0.99999f, -r.eps);
    const int ox = r.inv.x >= 0.f ? 0 : 3, oy = r.inv.y >= 0.f ? 1 : 4, oz = r.inv.z >= 0.f ? 2 : 5;
    while (true) {
        if ((unsigned)node >= (unsigned)bvh.cap || --budget < 0) {
            atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
            return h;
        }
        const float4* N = bvh.nodes + 8 * (size_t)node;
        const float4 nx = __ldg(N + ox), ny = __ldg(N + oy), nz = __ldg(N + oz);
        const float4 fx = __ldg(N + (3 - ox)), fy = __ldg(N + (5 - oy)), fz = __ldg(N + (7 - oz));
        const int4 ref = __ldg(reinterpret_cast<const int4*>(N + 6));
        const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, nys[4] = {ny.x, ny.y, ny.z, ny.w},
                    nzs[4] = {nz.x, nz.y, nz.z, nz.w};
        const float fxs[4] = {fx.x, fx.y, fx.z, fx.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w},
                    fzs[4] = {fz.x, fz.y, fz.z, fz.w};
        const int refs[4] = {ref.x, ref.y, ref.z, ref.w};
        float tn[4];
        bool hit[4];
        const float thi0 = fmaf(best, 1.00001f, r.eps);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float t0 = fmaxf(fmaxf(fmaf(nxs[c], r.inv.x, r.oinv.x), fmaf(nys[c], r.inv.y, r.oinv.y)),
                                   fmaxf(fmaf(nzs[c], r.inv.z, r.oinv.z), tlo));
            const float t1 = fminf(fminf(fmaf(fxs[c], r.inv.x, r.oinv.x), fmaf(fys[c], r.inv.y, r.oinv.y)),
                                   fminf(fmaf(fzs[c], r.inv.z, r.oinv.z), thi0));
            tn[c] = t0;
            hit[c] = t0 <= t1 && refs[c] != kRefEmpty;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (hit[c] && refs[c] < 0) {
                mesh_test_leaf(bvh, refs[c], r, tmin, tmax, best, h);
                hit[c] = false;
            }
        const float thi = fmaf(best, 1.00001f, r.eps);
        const float inf = __int_as_float(0x7f800000);
        float dd[4];
        int e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            dd[c] = (hit[c] && tn[c] <= thi) ? tn[c] : inf;
            e[c] = refs[c];
        }
#define GRT_CSWAP(i, j)              \
    if (dd[j] < dd[i]) {             \
        float td = dd[i];            \
        dd[i] = dd[j];               \
        dd[j] = td;                  \
        int te = e[i];               \
        e[i] = e[j];                 \
        e[j] = te;                   \
    }
        GRT_CSWAP(0, 1) GRT_CSWAP(2, 3) GRT_CSWAP(0, 2) GRT_CSWAP(1, 3) GRT_CSWAP(1, 2)
#undef GRT_CSWAP
        if (dd[0] != inf) {
#pragma unroll
            for (int c = 3; c >= 1; --c) {
                if (dd[c] != inf) {
                    if (sp < kStackDepth)
                        stack[sp++] = make_int2(e[c], __float_as_int(dd[c]));
                    else
                        atomicOr(bvh.status, GRT_STATUS_STACK_OVERFLOW);
                }
            }
            node = e[0];
            continue;
        }
        bool found = false;
        while (sp > 0) {
            const int2 t = stack[--sp];
            if (__int_as_float(t.y) <= fmaf(best, 1.00001f, r.eps)) {
                node = t.x;
                found = true;
                break;
            }
        }
        if (!found) return h;
    }
}

// Barycentric material state of a hit (Eq. 14, mesh backend); the normal faces the ray origin.
__device__ __forceinline__ void mesh_attr(const MeshDev& M, const MeshHit& h, f3 d, int* status, float a[3], float* r,
                                          float* m, f3* n) {
    const float w[3] = {1.f - h.u - h.v, h.u, h.v};
    float na[3] = {0.f, 0.f, 0.f};
    a[0] = a[1] = a[2] = 0.f;
    *r = 0.f;
    *m = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int vi = __ldg(M.tri + 3 * (size_t)h.id + k);
        if ((unsigned)vi >= (unsigned)M.nv) {
            atomicOr(status, GRT_STATUS_BAD_INDEX);
            vi = 0;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c] = fmaf(w[k], __ldg(M.albedo + 3 * (size_t)vi + c), a[c]);
            na[c] = fmaf(w[k], __ldg(M.normal + 3 * (size_t)vi + c), na[c]);
        }
        *r = fmaf(w[k], __ldg(M.rough + vi), *r);
        *m = fmaf(w[k], __ldg(M.metal + vi), *m);
    }
    const float nl = sqrtf(na[0] * na[0] + na[1] * na[1] + na[2] * na[2]);
    const float s = (na[0] * d.x + na[1] * d.y + na[2] * d.z) > 0.f ? -1.f : 1.f;
    const float in = nl > 0.f ? s / nl : 0.f;
    *n = mk3(na[0] * in, na[1] * in, na[2] * in);
}

}  // namespace grt
