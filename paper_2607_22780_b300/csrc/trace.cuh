// trace.cuh -- per-ray 2DGRT (Sec. III-B): LBVH traversal, ray-surfel test (Eq. 7),
// k-buffer of the nearest admitted hits, front-to-back compositing (Eq. 8).
//
// One thread traces one ray.  A round traverses the whole BVH collecting, in a register
// k-buffer, the K smallest keys (tau bits << 32 | surfel id) larger than the last key
// composited; the round then composites them in order.  While collecting, the buffer
// knows the transmittance its entries would leave: once the product of (1 - alpha) over
// a prefix drops below T_min, entries after that prefix can never be composited, so they
// are dropped and every node entered beyond the cut depth is culled.  A ray that filled
// the buffer without terminating traverses again from its last key.  The composited
// sequence is therefore exactly the (tau, id)-sorted admitted hits up to termination,
// whatever K is.
#pragma once

#include "grt_internal.cuh"

namespace grt {

struct TraceParams {
    float alpha_min, alpha_max, t_min, t_max, T_min, eps_nd;
};

__host__ __forceinline__ TraceParams to_params(const grt_trace_params& p) {
    return TraceParams{p.alpha_min, p.alpha_max, p.t_min, p.t_max, p.T_min, p.eps_nd};
}

constexpr int kStackDepth = 64;  // >= tree depth: at most 30 code bits + 34 position bits
constexpr uint64_t kNoKey = ~0ull;

struct RayState {
    f3 o, d;     // origin, direction (decision values)
    f3 inv;      // 1/d with zeros replaced by +-1e-20
    f3 oinv;     // -o * inv
    float eps;   // absolute slack of box tests
};

__device__ __forceinline__ RayState make_ray(f3 o, f3 d) {
    RayState r;
    r.o = o;
    r.d = d;
    float dx = fabsf(d.x) < 1e-20f ? copysignf(1e-20f, d.x) : d.x;
    float dy = fabsf(d.y) < 1e-20f ? copysignf(1e-20f, d.y) : d.y;
    float dz = fabsf(d.z) < 1e-20f ? copysignf(1e-20f, d.z) : d.z;
    r.inv = mk3(1.f / dx, 1.f / dy, 1.f / dz);
    r.oinv = mk3(-o.x * r.inv.x, -o.y * r.inv.y, -o.z * r.inv.z);
    r.eps = 1e-6f * (fmaxf(fabsf(o.x), fmaxf(fabsf(o.y), fabsf(o.z))) + 1.f);
    return r;
}

// Slab test of a box against [tlo, thi]; returns the entry distance in *tn.
__device__ __forceinline__ bool slab(const RayState& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                     float tlo, float thi, float* tn) {
    float x0 = fmaf(lx, r.inv.x, r.oinv.x), x1 = fmaf(hx, r.inv.x, r.oinv.x);
    float y0 = fmaf(ly, r.inv.y, r.oinv.y), y1 = fmaf(hy, r.inv.y, r.oinv.y);
    float z0 = fmaf(lz, r.inv.z, r.oinv.z), z1 = fmaf(hz, r.inv.z, r.oinv.z);
    float tmin = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tlo));
    float tmax = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), thi));
    *tn = tmin;
    return tmin <= tmax;
}

// Eq. 7 on a packed record.  The plane test (|n.d| >= eps_nd, tau in (t_min, t_max)) is
// a decision computation; the Gaussian test needs u^2 + v^2 <= 2 ln(o/alpha_min).
__device__ __forceinline__ bool intersect(const float4* __restrict__ records, int rec, const RayState& r,
                                          const TraceParams& P, float* tau, float* alpha, int* id) {
    const float4* R = records + 4 * (size_t)rec;
    float4 r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2), r3 = __ldg(R + 3);
    f3 n = mk3(r1.x, r1.y, r1.z);
    f3 w = mk3(sub_d(r0.x, r.o.x), sub_d(r0.y, r.o.y), sub_d(r0.z, r.o.z));
    float num = dot_d(n, w), den = dot_d(n, r.d);
    if (!(fabsf(den) >= P.eps_nd)) return false;
    float t = div_d(num, den);
    if (!(t > P.t_min && t < P.t_max)) return false;
    f3 dp = mk3(fmaf(t, r.d.x, -w.x), fmaf(t, r.d.y, -w.y), fmaf(t, r.d.z, -w.z));
    float u = fmaf(r2.x, dp.x, fmaf(r2.y, dp.y, r2.z * dp.z));
    float v = fmaf(r3.x, dp.x, fmaf(r3.y, dp.y, r3.z * dp.z));
    float q = fmaf(u, u, v * v);
    if (!(q <= r2.w)) return false;
    *alpha = fminf(r0.w * __expf(-0.5f * q), P.alpha_max);
    *tau = t;
    *id = __float_as_int(r1.w);
    return true;
}

__device__ __forceinline__ uint64_t make_key(float tau, int id) {
    return ((uint64_t)__float_as_uint(tau) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_tau(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int key_id(uint64_t k) { return (int)(uint32_t)k; }

struct Counters {
    long long nodes, tests, comp;
};

template <int K>
struct KBuf {
    uint64_t key[K];
    float a[K];
    uint64_t cut;   // keys >= cut cannot be composited this round
    float thi;      // node culling distance derived from cut

    __device__ __forceinline__ void reset(float t_max) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            key[j] = kNoKey;
            a[j] = 0.f;
        }
        cut = kNoKey;
        thi = t_max;
    }

    // Insert (k, al); keep ascending order; recompute the termination cut from the
    // transmittance T0 at the start of the round, with the compositing arithmetic.
    __device__ __forceinline__ void insert(uint64_t k, float al, float T0, float T_min, float t_max, float eps) {
        uint64_t ck = k;
        float ca = al;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            bool sw = ck < key[j];
            uint64_t tk = key[j];
            float ta = a[j];
            key[j] = sw ? ck : tk;
            a[j] = sw ? ca : ta;
            ck = sw ? tk : ck;
            ca = sw ? ta : ca;
        }
        float T = T0;
        bool dead = false;
        uint64_t nc = key[K - 1];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (dead) {
                key[j] = kNoKey;
            } else if (key[j] != kNoKey) {
                T = mul_d(T, sub_d(1.0f, a[j]));
                if (T < T_min) {
                    dead = true;
                    nc = key[j];
                }
            }
        }
        cut = nc;
        thi = nc == kNoKey ? t_max : fmaf(key_tau(nc), 1.00001f, eps);
    }
};

// Traverse the BVH once, feeding admitted hits with key in (last, cut) to the buffer.
template <int K, bool COUNT>
__device__ __forceinline__ void traverse(const DevBvh& bvh, const RayState& r, const TraceParams& P, uint64_t last,
                                         float T0, KBuf<K>& kb, Counters& cnt) {
    int2 stack[kStackDepth];
    int sp = 0;
    float tlo = fmaf(P.t_min, 0.99999f, -r.eps);
    auto test = [&](int rec) {
        if (COUNT) ++cnt.tests;
        float tau, al;
        int id;
        if (intersect(bvh.records, rec, r, P, &tau, &al, &id)) {
            uint64_t k = make_key(tau, id);
            if (k > last && k < kb.cut) kb.insert(k, al, T0, P.T_min, P.t_max, r.eps);
        }
    };
    int node = bvh.root;
    if (node == kRefEmpty) return;
    if (node < 0) {
        test(~node);
        return;
    }
    // every internal node is entered at most once per traversal; a longer walk means a
    // corrupt hierarchy, which is reported instead of looping
    int budget = bvh.n + 8;
    while (true) {
        if (COUNT) ++cnt.nodes;
        if ((unsigned)node >= (unsigned)(bvh.n - 1) || --budget < 0) {
            atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
            return;
        }
        const float4* N = bvh.nodes + 4 * (size_t)node;
        float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
        int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        float t0, t1;
        bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, tlo, kb.thi, &t0);
        bool h1 = slab(r, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, tlo, kb.thi, &t1);
        if (h0 && c0 < 0) {
            if (~c0 < bvh.n) test(~c0);
            else atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
            h0 = false;
        }
        if (h1 && c1 < 0) {
            if (~c1 < bvh.n) test(~c1);
            else atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
            h1 = false;
        }
        h0 = h0 && t0 <= kb.thi;
        h1 = h1 && t1 <= kb.thi;
        if (h0 && h1) {
            bool swap = t1 < t0;
            int near = swap ? c1 : c0, far = swap ? c0 : c1;
            float tf = swap ? t0 : t1;
            if (sp < kStackDepth) {
                stack[sp++] = make_int2(far, __float_as_int(tf));
            } else {
                atomicOr(bvh.status, GRT_STATUS_STACK_OVERFLOW);
            }
            node = near;
            continue;
        }
        if (h0) {
            node = c0;
            continue;
        }
        if (h1) {
            node = c1;
            continue;
        }
        bool found = false;
        while (sp > 0) {
            int2 e = stack[--sp];
            if (__int_as_float(e.y) <= kb.thi) {
                node = e.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}

// Trace one ray through all rounds.  `vis` receives composite(k, id, tau, alpha, T)
// for each composited hit in order (T = transmittance before the hit) and returns the
// final transmittance via vis.finish(T).  Returns the number of rounds.
template <int K, bool COUNT, class Visitor>
__device__ __forceinline__ int trace_ray(const DevBvh& bvh, const RayState& r, const TraceParams& P, Visitor& vis,
                                         Counters& cnt) {
    float T = 1.f;
    uint64_t last = 0ull;
    int k = 0, rounds = 0;
    KBuf<K> kb;
    while (true) {
        if (++rounds > bvh.n + 1) {  // each full round composites K new hits
            atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
            break;
        }
        kb.reset(P.t_max);
        traverse<K, COUNT>(bvh, r, P, last, T, kb, cnt);
        bool term = false;
        int filled = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!term && kb.key[j] != kNoKey) {
                vis.composite(k++, key_id(kb.key[j]), key_tau(kb.key[j]), kb.a[j], T);
                T = mul_d(T, sub_d(1.0f, kb.a[j]));
                ++filled;
                if (T < P.T_min) term = true;
            }
        }
        if (COUNT) cnt.comp += filled;
        if (term || filled < K) break;
        last = kb.key[K - 1];
    }
    vis.finish(T);
    return rounds;
}

// ----------------------------------------------------------------------------- colour

// Real SH basis to degree 3 at unit direction (x,y,z), constants sqrt((2l+1)/(4pi)...).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    const float c0 = 0.28209479177387814f, c1 = 0.48860251190291992f;
    const float c2a = 1.0925484305920790f, c2b = 0.31539156525252005f, c2c = 0.54627421529603959f;
    const float c3a = 0.59004358992664352f, c3b = 2.8906114426405538f, c3c = 0.45704579946446572f;
    const float c3d = 0.37317633259011540f, c3e = 1.4453057213202769f;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.f * zz - xx - yy);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (xx - yy);
    Y[9] = -c3a * y * (3.f * xx - yy);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.f * zz - xx - yy);
    Y[12] = c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -c3c * x * (4.f * zz - xx - yy);
    Y[14] = c3e * z * (xx - yy);
    Y[15] = -c3a * x * (xx - 3.f * yy);
}

// Surfel colour toward direction d: RGB, or max(0, SH(d) + 0.5) per channel.
__device__ __forceinline__ void surfel_colour(const float* __restrict__ color, int cdim, int id, f3 d, float c[3]) {
    if (cdim == 3) {
        c[0] = __ldg(color + 3 * (size_t)id);
        c[1] = __ldg(color + 3 * (size_t)id + 1);
        c[2] = __ldg(color + 3 * (size_t)id + 2);
        return;
    }
    float Y[16];
    sh_basis(d.x, d.y, d.z, Y);
    const float4* s = reinterpret_cast<const float4*>(color + 48 * (size_t)id);
    float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        float4 v = __ldg(s + q);
        float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int idx = 4 * q + t;
            acc[idx % 3] = fmaf(e[t], Y[idx / 3], acc[idx % 3]);
        }
    }
    c[0] = fmaxf(acc[0], 0.f);
    c[1] = fmaxf(acc[1], 0.f);
    c[2] = fmaxf(acc[2], 0.f);
}

// Forward visitor: c_rt, o_rt = 1 - T (Eq. 8), optional hit list.
struct ColourVisitor {
    const float* color;
    int cdim;
    f3 d;
    float c[3];
    float T;
    int* hits;
    int max_hits;
    int nh;
    __device__ __forceinline__ ColourVisitor(const float* col, int cd, f3 dir, int* h, int mh)
        : color(col), cdim(cd), d(dir), T(1.f), hits(h), max_hits(mh), nh(0) {
        c[0] = c[1] = c[2] = 0.f;
    }
    __device__ __forceinline__ void composite(int k, int id, float, float alpha, float Tb) {
        float ck[3];
        surfel_colour(color, cdim, id, d, ck);
        float w = Tb * alpha;
        c[0] = fmaf(w, ck[0], c[0]);
        c[1] = fmaf(w, ck[1], c[1]);
        c[2] = fmaf(w, ck[2], c[2]);
        if (hits && k < max_hits) hits[k] = id;
        nh = k + 1;
    }
    __device__ __forceinline__ void finish(float Tf) { T = Tf; }
};

}  // namespace grt
