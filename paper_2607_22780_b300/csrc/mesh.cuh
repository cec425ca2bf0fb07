// mesh.cuh -- mesh backend of the relighting query (Sec. III-E): closest triangle hit in the
// 4-wide LBVH built by grt_build_mesh_bvh, and the barycentric attributes of Eq. 14.
//
// Leaf records (64 bytes, one triangle): (v0, triangle id), (v1, 0), (v2, 0), unused.
// Which triangle a ray hits is decided in FP32 by the watertight ray/triangle test of Woop,
// Benthin and Wald (JCGT 2(1), 2013), two-sided, through one fixed sequence of correctly
// rounded operations (no contraction into FMA):
//   kz = the axis of the largest |d| (the first on ties), kx = kz+1 mod 3, ky = kx+1 mod 3;
//   Sx = d[kx]/d[kz], Sy = d[ky]/d[kz], Sz = 1/d[kz];
//   A = v0 - o, B = v1 - o, C = v2 - o;  Px = P[kx] - Sx P[kz], Py = P[ky] - Sy P[kz];
//   U = Cx By - Cy Bx, V = Ax Cy - Ay Cx, W = Bx Ay - By Ax, recomputed when one of them is
//   0 by Kahan's difference of products with fused multiply-adds (relative error below
//   2 ulp, Jeannerod, Louvet and Muller 2013: exact sign and zeros), FP32 throughout;
//   hit iff U, V, W share a sign (zeros allowed) and det = (U + V) + W != 0, and
//   t = ((U (Sz A[kz]) + V (Sz B[kz])) + W (Sz C[kz])) / det lies in (t_min, t_max).
// A shared edge gives the two triangles edge functions of equal magnitude and opposite
// sign, and when it is 0 in one it is 0 in both and both take the exact-sign difference,
// so no ray passes between neighbours.  The nearest t wins, equal t by triangle
// index; the weights of (v0, v1, v2) are (U, V, W) / det.  The walk visits children near to
// far and culls every box beyond the nearest hit found so far.
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
    int id;        // triangle index, -1 for a miss
    float w[3];    // barycentric weights of v0, v1, v2
};

// The ray's shear for the watertight test.
struct ShearRay {
    f3 o;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

// a b - c d by Kahan's algorithm (exact sign).
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

__device__ __forceinline__ float comp(f3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

__device__ __forceinline__ ShearRay shear_ray(f3 o, f3 d) {
    ShearRay r;
    r.o = o;
    int kz = 0;
    if (fabsf(d.y) > fabsf(comp(d, kz))) kz = 1;
    if (fabsf(d.z) > fabsf(comp(d, kz))) kz = 2;
    r.kz = kz;
    r.kx = kz == 2 ? 0 : kz + 1;
    r.ky = r.kx == 2 ? 0 : r.kx + 1;
    const float dz = comp(d, kz);
    r.Sx = __fdiv_rn(comp(d, r.kx), dz);
    r.Sy = __fdiv_rn(comp(d, r.ky), dz);
    r.Sz = __fdiv_rn(1.f, dz);
    return r;
}

__device__ __forceinline__ void mesh_test_leaf(const DevBvh& bvh, int ref, const ShearRay& r, float tmin, float& best,
                                               MeshHit& h) {
    const int first = leaf_first(ref), count = leaf_count(ref);
    if (first + count > bvh.n) {
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        return;
    }
    for (int i = 0; i < count; ++i) {
        const float4* R = bvh.records + 4 * (size_t)(first + i);
        const float4 r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2);
        const f3 A = mk3(__fsub_rn(r0.x, r.o.x), __fsub_rn(r0.y, r.o.y), __fsub_rn(r0.z, r.o.z));
        const f3 B = mk3(__fsub_rn(r1.x, r.o.x), __fsub_rn(r1.y, r.o.y), __fsub_rn(r1.z, r.o.z));
        const f3 C = mk3(__fsub_rn(r2.x, r.o.x), __fsub_rn(r2.y, r.o.y), __fsub_rn(r2.z, r.o.z));
        const float Az = comp(A, r.kz), Bz = comp(B, r.kz), Cz = comp(C, r.kz);
        const float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Az)), Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Az));
        const float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bz)), By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bz));
        const float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Cz)), Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Cz));
        float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
        float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
        float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
        if (U == 0.f || V == 0.f || W == 0.f) {
            U = diff_prod(Cx, By, Cy, Bx);
            V = diff_prod(Ax, Cy, Ay, Cx);
            W = diff_prod(Bx, Ay, By, Ax);
        }
        if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) continue;
        const float det = __fadd_rn(__fadd_rn(U, V), W);
        if (det == 0.f) continue;
        const float T = __fadd_rn(__fadd_rn(__fmul_rn(U, __fmul_rn(r.Sz, Az)), __fmul_rn(V, __fmul_rn(r.Sz, Bz))),
                                  __fmul_rn(W, __fmul_rn(r.Sz, Cz)));
        const float t = __fdiv_rn(T, det);
        if (!(t > tmin && t <= best)) continue;
        const int id = __float_as_int(r0.w);
        if (h.id < 0 || t < best || id < h.id) {
            best = t;
            h.id = id;
            const float inv = 1.f / det;
            h.w[0] = U * inv;
            h.w[1] = V * inv;
            h.w[2] = W * inv;
        }
    }
}

// Closest hit of the ray (o, d) with t in (tmin, tmax).
__device__ __forceinline__ MeshHit mesh_closest(const DevBvh& bvh, f3 o, f3 d, float tmin, float tmax) {
    MeshHit h{-1, {0.f, 0.f, 0.f}};
    if (bvh.n == 0 || bvh.root == kRefEmpty) return h;
    const RayState r = make_ray(o, d);
    const ShearRay sr = shear_ray(o, d);
    // best starts just below t_max: a hit needs t < t_max, and t <= best afterwards keeps
    // equal-t hits for the index tie-break
    float best = __int_as_float(__float_as_int(tmax) - 1);
    if (bvh.root < 0) {  // a single triangle
        mesh_test_leaf(bvh, bvh.root, sr, tmin, best, h);
        return h;
    }
    int2 stack[kStackDepth];
    int sp = 0, node = bvh.root, budget = bvh.cap + 8;
    const float tlo = fmaf(tmin, 0.99999f, -r.eps);
    const int ox = r.inv.x >= 0.f ? 0 : 3, oy = r.inv.y >= 0.f ? 1 : 4, oz = r.inv.z >= 0.f ? 2 : 5;
    // Conservative slabs.  fmaf(plane, inv, oinv) differs from (plane - o) / d by at most
    // 4 * 2^-24 (C + |o|) |inv| on an axis whose planes satisfy |plane| <= C; every slab is
    // widened by 2^-20 (C + |o|) |inv|, C the largest |coordinate| of the root's boxes, so
    // that no box whose exact slab interval meets the ray is culled.  Triangles in an
    // axis-aligned plane have boxes of zero thickness, where an unwidened test drops hits
    // near the box edges at grazing incidence.
    f3 oN, oF;
    {
        const float4* N = bvh.nodes + 8 * (size_t)bvh.root;
        const int4 ref = __ldg(reinterpret_cast<const int4*>(N + 6));
        const int refs[4] = {ref.x, ref.y, ref.z, ref.w};
        float C[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float4 lo = __ldg(N + a), hi = __ldg(N + 3 + a);
            const float los[4] = {lo.x, lo.y, lo.z, lo.w}, his[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (refs[c] != kRefEmpty) C[a] = fmaxf(C[a], fmaxf(fabsf(los[c]), fabsf(his[c])));
        }
        const float sx = 0x1p-20f * (C[0] + fabsf(o.x)) * fabsf(r.inv.x);
        const float sy = 0x1p-20f * (C[1] + fabsf(o.y)) * fabsf(r.inv.y);
        const float sz = 0x1p-20f * (C[2] + fabsf(o.z)) * fabsf(r.inv.z);
        oN = mk3(r.oinv.x - sx, r.oinv.y - sy, r.oinv.z - sz);
        oF = mk3(r.oinv.x + sx, r.oinv.y + sy, r.oinv.z + sz);
    }
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
            const float t0 = fmaxf(fmaxf(fmaf(nxs[c], r.inv.x, oN.x), fmaf(nys[c], r.inv.y, oN.y)),
                                   fmaxf(fmaf(nzs[c], r.inv.z, oN.z), tlo));
            const float t1 = fminf(fminf(fmaf(fxs[c], r.inv.x, oF.x), fmaf(fys[c], r.inv.y, oF.y)),
                                   fminf(fmaf(fzs[c], r.inv.z, oF.z), thi0));
            tn[c] = t0;
            hit[c] = t0 <= t1 && refs[c] != kRefEmpty;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (hit[c] && refs[c] < 0) {
                mesh_test_leaf(bvh, refs[c], sr, tmin, best, h);
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
    const float* w = h.w;
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
