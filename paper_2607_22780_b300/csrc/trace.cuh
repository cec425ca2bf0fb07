// trace.cuh -- per-ray 2DGRT (Sec. III-B): 4-wide BVH traversal, ray-surfel test (Eq. 7),
// k-buffer of the nearest admitted hits, front-to-back compositing (Eq. 8).
//
// One thread traces one ray.  A round traverses the BVH collecting, in a register
// k-buffer, the K smallest keys (tau bits << 32 | surfel id) larger than the last key
// composited, then composites them in order.  The buffer also tracks the product of
// (1 - alpha) over its entries; once the round-start transmittance times that product is
// below T_min (with a margin far wider than FP32 rounding of K factors), compositing is
// certain to stop at or before the buffer's largest key, so hits beyond it -- and every
// node entered beyond its depth -- are culled, as they are when the buffer is full.  A
// ray that filled the buffer without terminating traverses again from its last key.  The
// composited sequence is exactly the (tau, id)-sorted admitted hits up to termination,
// whatever K and the tree shape are.
#pragma once

#include <type_traits>
#include <utility>

#include "grt_internal.cuh"

namespace grt {

struct TraceParams {
    float alpha_min, alpha_max, t_min, t_max, T_min, eps_nd;
};

__host__ __forceinline__ TraceParams to_params(const grt_trace_params& p) {
    return TraceParams{p.alpha_min, p.alpha_max, p.t_min, p.t_max, p.T_min, p.eps_nd};
}

// Ordered traversal keeps at most kWide - 1 entries per level of the current path.
constexpr int kStackDepth = 96;
constexpr uint64_t kNoKey = ~0ull;

// Traversal stack of one lane.  LocalStack lives in local memory; SplitStack keeps its
// first kSharedStack entries in shared memory (slot i of lane t at sh[i * stride]) and
// only deeper ones in local memory, so the hot top of the stack does not compete with
// node and record lines for L1 (16 shared entries: 328.5 -> 339.8 M rays/s on the
// 300k-surfel 800x800 workload; 8 or 32 gained less).
#ifndef GRT_SMEM_STACK
#define GRT_SMEM_STACK 8
#endif
constexpr int kSharedStack = GRT_SMEM_STACK;

struct LocalStack {
    int2 e[kStackDepth];
    __device__ __forceinline__ void put(int i, int2 v) { e[i] = v; }
    __device__ __forceinline__ int2 get(int i) const { return e[i]; }
};

struct SplitStack {
    int2* sh;
    int stride;
    int2 e[kStackDepth - kSharedStack > 0 ? kStackDepth - kSharedStack : 1];
    __device__ __forceinline__ void put(int i, int2 v) {
        if (i < kSharedStack)
            sh[i * stride] = v;
        else
            e[i - kSharedStack] = v;
    }
    __device__ __forceinline__ int2 get(int i) const { return i < kSharedStack ? sh[i * stride] : e[i - kSharedStack]; }
};

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

// 32-byte read-only loads (PTX ld.global.nc.v8.f32, sm_100 and later; the address must be
// 32-byte aligned).  A divergent warp-wide load costs one L1 wavefront per distinct line
// it touches, so halving the load instructions of a node visit, a record test and an SH
// evaluation halves their share of the L1 data pipe, which bounds the walk.
#ifndef GRT_V8
#define GRT_V8 1
#endif
struct F8 {
    float4 a, b;
};
__device__ __forceinline__ F8 ld_v8(const float4* p) {
#if GRT_V8
    F8 r;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y), "=f"(r.b.z), "=f"(r.b.w)
        : "l"(p));
    return r;
#else
    return F8{__ldg(p), __ldg(p + 1)};
#endif
}

// Eq. 7 on a packed record.  The plane test (|n.d| >= eps_nd, tau in (t_min, t_max)) is
// a decision computation; the Gaussian test needs u^2 + v^2 <= 2 ln(o/alpha_min).
__device__ __forceinline__ bool intersect(const float4* __restrict__ records, int rec, const RayState& r,
                                          const TraceParams& P, float* tau, float* alpha, int* id) {
    const float4* R = records + 4 * (size_t)rec;
    const F8 r01 = ld_v8(R), r23 = ld_v8(R + 2);  // records are 64-byte aligned
    const float4 r0 = r01.a, r1 = r01.b, r2 = r23.a, r3 = r23.b;
    f3 n = mk3(r1.x, r1.y, r1.z);
    f3 w = mk3(sub_d(r0.x, r.o.x), sub_d(r0.y, r.o.y), sub_d(r0.z, r.o.z));
    float num = dot_d(n, w), den = dot_d(n, r.d);
    // every test runs the whole of Eq. 7 and decides once at the end: a hit computes the same
    // values, a miss may divide by a tiny |n.d| (inf or NaN, which fail the checks).  Exiting
    // at the plane and depth checks split the lanes of a warp three ways: walk 11.07 -> 10.74
    // ms on 300k surfels at 800x800, G-buffer 1.12 -> 1.05 ms, 2M-surfel 1080p forward 65.1 ->
    // 63.2 ms.
    float t = div_d(num, den);
    f3 dp = mk3(fmaf(t, r.d.x, -w.x), fmaf(t, r.d.y, -w.y), fmaf(t, r.d.z, -w.z));
    float u = fmaf(r2.x, dp.x, fmaf(r2.y, dp.y, r2.z * dp.z));
    float v = fmaf(r3.x, dp.x, fmaf(r3.y, dp.y, r3.z * dp.z));
    float q = fmaf(u, u, v * v);
    const bool ok = (fabsf(den) >= P.eps_nd) & (t > P.t_min) & (t < P.t_max) & (q <= r2.w);
    if (!ok) return false;
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
    static constexpr bool kShared = false;
    uint64_t key[K];
    float a[K];
    int cnt;         // valid entries, a prefix of key[]
    float Tall;      // product of (1 - a) over the entries (any order)
    uint64_t maxk;   // largest valid key
    uint64_t cut;    // keys >= cut cannot be composited this round
    float thi;       // node culling distance derived from cut

    __device__ __forceinline__ void reset(float t_max) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            key[j] = kNoKey;
            a[j] = 0.f;
        }
        cnt = 0;
        Tall = 1.f;
        maxk = 0ull;
        cut = kNoKey;
        thi = t_max;
    }

    // Branch-free insertion (one compare-swap pass over the buffer).  An append branch for
    // keys beyond the current maximum (the common case front to back) measured slower:
    // 431 -> 368 M rays/s, lanes of a warp split between the two paths.
    __device__ __forceinline__ void insert(uint64_t k, float al, float T0, float T_min, float t_max, float eps) {
        const bool full = cnt == K;
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
        if (full) {
            // the old maximum was evicted: recompute the product, no division drift
            float t = 1.f;
#pragma unroll
            for (int j = 0; j < K; ++j) t *= sub_d(1.0f, a[j]);
            Tall = t;
            maxk = key[K - 1];
        } else {
            ++cnt;
            Tall *= sub_d(1.0f, al);
            maxk = k > maxk ? k : maxk;
        }
        // T0 * Tall rounds within 2K ulps of the sequential product the compositor forms
        bool terminates = T0 * Tall < T_min * 0.9999f;
        cut = (cnt == K || terminates) ? maxk : kNoKey;
        thi = cut == kNoKey ? t_max : fmaf(key_tau(cut), 1.00001f, eps);
    }
};

// The same k-buffer for the persistent walks, kept in shared memory as a sorted array
// instead of registers: entry j of the lane whose column starts at key/a sits at
// key[j * kKbufThreads] (one 8-byte key and one 4-byte alpha word per lane and
// entry, bank-conflict free across a warp).  A hit is placed by shifting the larger keys
// up by one; hits mostly arrive near to far, so the shift is short, where the register
// buffer pays a compare-swap over all K entries for every hit.  When the buffer is full
// the largest entry drops off its end.  The cut and termination rules are those of KBuf,
// so the composited sequence is the same.
constexpr int kKbufThreads = 128;  // lanes of a block sharing the k-buffer arrays

template <int K>
struct KBufShared {
    static constexpr bool kShared = true;
    uint64_t* key;   // this lane's column: key[j * kKbufThreads]
    float* a;
    int cnt;
    float Tall;      // product of (1 - a) over the entries while the buffer is not full
    uint64_t cut;
    float thi;

    __device__ __forceinline__ uint64_t key_at(int j) const { return key[j * kKbufThreads]; }
    __device__ __forceinline__ float a_at(int j) const { return a[j * kKbufThreads]; }

    __device__ __forceinline__ void reset(float t_max) {
        cnt = 0;
        Tall = 1.f;
        cut = kNoKey;
        thi = t_max;
    }

    __device__ __forceinline__ void insert(uint64_t k, float al, float T0, float T_min, float t_max, float eps) {
        int pos = cnt < K ? cnt : K - 1;  // a full buffer loses its largest entry
        while (pos > 0) {
            const uint64_t kp = key[(pos - 1) * kKbufThreads];
            if (kp < k) break;  // keys are distinct: (tau, id) with distinct ids
            key[pos * kKbufThreads] = kp;
            a[pos * kKbufThreads] = a[(pos - 1) * kKbufThreads];
            --pos;
        }
        key[pos * kKbufThreads] = k;
        a[pos * kKbufThreads] = al;
        if (cnt < K) {
            ++cnt;
            Tall *= sub_d(1.0f, al);  // once full the product is no longer needed this round
        }
        // T0 * Tall rounds within 2K ulps of the sequential product the compositor forms
        if (cnt == K || T0 * Tall < T_min * 0.9999f) {
            cut = key[(cnt - 1) * kKbufThreads];
            thi = fmaf(key_tau(cut), 1.00001f, eps);
        }
    }
};

// Per-ray traversal state, advanced one wide node at a time so that a warp can refill
// lanes whose rays have finished while others are still walking the tree.
template <int K, class KB = KBuf<K>>
struct TraceState {
    using KBT = KB;
    static constexpr int kK = K;
    RayState r;
    KB kb;
    float T;         // transmittance before the next composited hit
    uint64_t last;   // largest key composited so far
    int node;        // next wide node, or -1 when the round's walk is over
    int sp;          // stack depth
    int budget;      // node visits left in this round
    int rounds;
    int ncomp;       // hits composited so far
};

// State of a ray in the persistent walks (k-buffer in shared memory).
template <int K>
using WalkState = TraceState<K, KBufShared<K>>;

template <class TS>
__device__ __forceinline__ void round_begin(const DevBvh& bvh, TS& s, const TraceParams& P) {
    s.kb.reset(P.t_max);
    s.sp = 0;
    s.budget = bvh.cap + 8;
    s.node = (bvh.root >= 0) ? bvh.root : -1;
}

template <class TS>
__device__ __forceinline__ void trace_begin(const DevBvh& bvh, TS& s, f3 o, f3 d, const TraceParams& P) {
    s.r = make_ray(o, d);
    s.T = 1.f;
    s.last = 0ull;
    s.rounds = 1;
    s.ncomp = 0;
    round_begin(bvh, s, P);
    // a NaN or infinite origin or direction is reported and traced as a miss
    if (!(isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) && isfinite(d.z))) {
        atomicOr(bvh.status, GRT_STATUS_NONFINITE);
        s.node = -2;
        s.budget = 0;
    }
}

// Continue a ray after `ncomp` hits already composited (the last one with key `last`),
// with transmittance T in front of the next hit: the next round collects keys > last.
template <class TS>
__device__ __forceinline__ void trace_resume(const DevBvh& bvh, TS& s, f3 o, f3 d, const TraceParams& P,
                                             uint64_t last, float T, int ncomp) {
    trace_begin(bvh, s, o, d, P);
    if (s.node == -2) return;  // non-finite ray
    s.last = last;
    s.T = T;
    s.ncomp = ncomp;
}

template <bool COUNT, class TS>
__device__ __forceinline__ void test_leaf(const DevBvh& bvh, TS& s, int ref, const TraceParams& P, Counters& cnt) {
    int first = leaf_first(ref), count = leaf_count(ref);
    if (first + count > bvh.n) {
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        return;
    }
    for (int i = 0; i < count; ++i) {
        if (COUNT) ++cnt.tests;
        float tau, al;
        int id;
        if (intersect(bvh.records, first + i, s.r, P, &tau, &al, &id)) {
            uint64_t k = make_key(tau, id);
            if (k > s.last && k < s.kb.cut) s.kb.insert(k, al, s.T, P.T_min, P.t_max, s.r.eps);
        }
    }
}

// One step of the round's walk: visit one wide node (testing its leaf children) and pick
// the next node.  Returns false once the walk of this round is over.
template <bool COUNT, class TS, class Stack>
__device__ __forceinline__ bool trav_step(const DevBvh& bvh, TS& s, Stack& stack, const TraceParams& P,
                                          Counters& cnt) {
    int node = s.node;
    if (node < 0) {
        // root that is a single leaf (n == 1), or an empty scene
        if (node == -1 && bvh.root != kRefEmpty && bvh.root < 0 && s.budget > 0) {
            s.budget = 0;
            test_leaf<COUNT>(bvh, s, bvh.root, P, cnt);
        }
        return false;
    }
    if (COUNT) ++cnt.nodes;
    if ((unsigned)node >= (unsigned)bvh.cap || --s.budget < 0) {
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        s.node = -2;
        return false;
    }
    const RayState& r = s.r;
    // near cull: t_min, and in later rounds the last composited depth (a node ending before
    // it holds only keys <= last), with the far cull's slack
    const float tlo = fmaf(fmaxf(P.t_min, key_tau(s.last)), 0.99999f, -r.eps);
    // the six child-plane float4 in three 32-byte loads (nodes are 128-byte aligned), the
    // near plane of each axis chosen by the direction's sign (lo for a positive direction)
    const float4* N = bvh.nodes + 8 * (size_t)node;
    const F8 xy = ld_v8(N), zx = ld_v8(N + 2), yz = ld_v8(N + 4);  // (lo.x lo.y) (lo.z hi.x) (hi.y hi.z)
    const int4 ref = __ldg(reinterpret_cast<const int4*>(N + 6));
    const bool px = r.inv.x >= 0.f, py = r.inv.y >= 0.f, pz = r.inv.z >= 0.f;
    const float4 nx = px ? xy.a : zx.b, fx = px ? zx.b : xy.a;
    const float4 ny = py ? xy.b : yz.a, fy = py ? yz.a : xy.b;
    const float4 nz = pz ? zx.a : yz.b, fz = pz ? yz.b : zx.a;
    const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, nys[4] = {ny.x, ny.y, ny.z, ny.w}, nzs[4] = {nz.x, nz.y, nz.z, nz.w};
    const float fxs[4] = {fx.x, fx.y, fx.z, fx.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
    const int refs[4] = {ref.x, ref.y, ref.z, ref.w};
    float tn[4];
    bool hit[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float t0 = fmaxf(fmaxf(fmaf(nxs[c], r.inv.x, r.oinv.x), fmaf(nys[c], r.inv.y, r.oinv.y)),
                         fmaxf(fmaf(nzs[c], r.inv.z, r.oinv.z), tlo));
        float t1 = fminf(fminf(fmaf(fxs[c], r.inv.x, r.oinv.x), fmaf(fys[c], r.inv.y, r.oinv.y)),
                         fminf(fmaf(fzs[c], r.inv.z, r.oinv.z), s.kb.thi));
        tn[c] = t0;
        hit[c] = t0 <= t1;
    }
    // leaves in slot order (the k-buffer sorts), one copy of the leaf code for all slots,
    // then internal children near to far
    unsigned leaves = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (hit[c] && refs[c] < 0) {
            leaves |= 1u << c;
            hit[c] = false;
        }
    }
#pragma unroll 1
    while (leaves) {
        int c = __ffs(leaves) - 1;
        leaves &= leaves - 1;
        int lr = c == 0 ? ref.x : (c == 1 ? ref.y : (c == 2 ? ref.z : ref.w));
        test_leaf<COUNT>(bvh, s, lr, P, cnt);
    }
    const float inf = __int_as_float(0x7f800000);
    float d[4];
    int e[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        bool h = hit[c] && tn[c] <= s.kb.thi;
        d[c] = h ? tn[c] : inf;
        e[c] = refs[c];
    }
#define GRT_CSWAP(i, j)              \
    if (d[j] < d[i]) {               \
        float td = d[i];             \
        d[i] = d[j];                 \
        d[j] = td;                   \
        int te = e[i];               \
        e[i] = e[j];                 \
        e[j] = te;                   \
    }
    GRT_CSWAP(0, 1) GRT_CSWAP(2, 3) GRT_CSWAP(0, 2) GRT_CSWAP(1, 3) GRT_CSWAP(1, 2)
#undef GRT_CSWAP
    if (d[0] != inf) {
#pragma unroll
        for (int c = 3; c >= 1; --c) {
            if (d[c] != inf) {
                if (s.sp < kStackDepth) {
                    stack.put(s.sp++, make_int2(e[c], __float_as_int(d[c])));
                } else {
                    atomicOr(bvh.status, GRT_STATUS_STACK_OVERFLOW);
                }
            }
        }
        s.node = e[0];
        return true;
    }
    while (s.sp > 0) {
        int2 t = stack.get(--s.sp);
        if (__int_as_float(t.y) <= s.kb.thi) {
            s.node = t.x;
            return true;
        }
    }
    s.node = -2;
    return false;
}

// Node visit of the two-phase walk: hit leaf children are queued (tested later by the
// whole warp together) instead of being tested here; hit internal children go near to far
// on the stack as in trav_step.  The queue lives in shared memory, q[slot * stride].
template <bool COUNT, class TS, class Stack>
__device__ __forceinline__ void node_step_q(const DevBvh& bvh, TS& s, Stack& stack, const TraceParams& P, int* q,
                                            int stride, int& nq, Counters& cnt) {
    int node = s.node;
    if (node < 0) {
        if (node == -1 && bvh.root != kRefEmpty && bvh.root < 0) q[stride * nq++] = bvh.root;
        s.node = -2;
        return;
    }
    if (COUNT) ++cnt.nodes;
    if ((unsigned)node >= (unsigned)bvh.cap || --s.budget < 0) {
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        s.node = -2;
        s.sp = 0;
        return;
    }
    const RayState& r = s.r;
    // near cull: t_min, and in later rounds the last composited depth (a node ending before
    // it holds only keys <= last), with the far cull's slack
    const float tlo = fmaf(fmaxf(P.t_min, key_tau(s.last)), 0.99999f, -r.eps);
    // the six child-plane float4 in three 32-byte loads (nodes are 128-byte aligned), the
    // near plane of each axis chosen by the direction's sign (lo for a positive direction)
    const float4* N = bvh.nodes + 8 * (size_t)node;
    const F8 xy = ld_v8(N), zx = ld_v8(N + 2), yz = ld_v8(N + 4);  // (lo.x lo.y) (lo.z hi.x) (hi.y hi.z)
    const int4 ref = __ldg(reinterpret_cast<const int4*>(N + 6));
    const bool px = r.inv.x >= 0.f, py = r.inv.y >= 0.f, pz = r.inv.z >= 0.f;
    const float4 nx = px ? xy.a : zx.b, fx = px ? zx.b : xy.a;
    const float4 ny = py ? xy.b : yz.a, fy = py ? yz.a : xy.b;
    const float4 nz = pz ? zx.a : yz.b, fz = pz ? yz.b : zx.a;
    const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, nys[4] = {ny.x, ny.y, ny.z, ny.w}, nzs[4] = {nz.x, nz.y, nz.z, nz.w};
    const float fxs[4] = {fx.x, fx.y, fx.z, fx.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
    const int refs[4] = {ref.x, ref.y, ref.z, ref.w};
    const float inf = __int_as_float(0x7f800000);
    float d[4];
    int e[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float t0 = fmaxf(fmaxf(fmaf(nxs[c], r.inv.x, r.oinv.x), fmaf(nys[c], r.inv.y, r.oinv.y)),
                         fmaxf(fmaf(nzs[c], r.inv.z, r.oinv.z), tlo));
        float t1 = fminf(fminf(fmaf(fxs[c], r.inv.x, r.oinv.x), fmaf(fys[c], r.inv.y, r.oinv.y)),
                         fminf(fmaf(fzs[c], r.inv.z, r.oinv.z), s.kb.thi));
        bool h = t0 <= t1;
        if (h && refs[c] < 0) {
            q[stride * nq++] = refs[c];
            h = false;
        }
        d[c] = h ? t0 : inf;
        e[c] = refs[c];
    }
#define GRT_CSWAP(i, j)              \
    if (d[j] < d[i]) {               \
        float td = d[i];             \
        d[i] = d[j];                 \
        d[j] = td;                   \
        int te = e[i];               \
        e[i] = e[j];                 \
        e[j] = te;                   \
    }
    GRT_CSWAP(0, 1) GRT_CSWAP(2, 3) GRT_CSWAP(0, 2) GRT_CSWAP(1, 3) GRT_CSWAP(1, 2)
#undef GRT_CSWAP
    if (d[0] != inf) {
#pragma unroll
        for (int c = 3; c >= 1; --c) {
            if (d[c] != inf) {
                if (s.sp < kStackDepth) {
                    stack.put(s.sp++, make_int2(e[c], __float_as_int(d[c])));
                } else {
                    atomicOr(bvh.status, GRT_STATUS_STACK_OVERFLOW);
                }
            }
        }
        s.node = e[0];
        return;
    }
    while (s.sp > 0) {
        int2 t = stack.get(--s.sp);
        if (__int_as_float(t.y) <= s.kb.thi) {
            s.node = t.x;
            return;
        }
    }
    s.node = -2;
}

// End of a round: composite the buffer in order (Eq. 8).  Returns true when the ray is
// finished; otherwise the next round starts after the last composited key.
template <bool COUNT, class TS, class Visitor>
__device__ __forceinline__ bool round_end(const DevBvh& bvh, TS& s, const TraceParams& P, Visitor& vis,
                                          Counters& cnt) {
    constexpr int K = TS::kK;
    bool term = false;
    int filled = 0;
    float T = s.T;
    uint64_t lastk;
    if constexpr (TS::KBT::kShared) {
        // entries in order from shared memory; stop at termination
        for (int j = 0; j < s.kb.cnt; ++j) {
            const uint64_t k = s.kb.key_at(j);
            const float al = s.kb.a_at(j);
            vis.composite(s.ncomp + filled, key_id(k), key_tau(k), al, T);
            T = mul_d(T, sub_d(1.0f, al));
            ++filled;
            if (T < P.T_min) {
                term = true;
                break;
            }
        }
        lastk = s.kb.cnt == K ? s.kb.key_at(K - 1) : 0ull;
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!term && j < s.kb.cnt) {
                vis.composite(s.ncomp + filled, key_id(s.kb.key[j]), key_tau(s.kb.key[j]), s.kb.a[j], T);
                T = mul_d(T, sub_d(1.0f, s.kb.a[j]));
                ++filled;
                if (T < P.T_min) term = true;
            }
        }
        lastk = s.kb.key[K - 1];
    }
    s.T = T;
    s.ncomp += filled;
    if (COUNT) cnt.comp += filled;
    if (term || s.kb.cnt < K) return true;
    if (++s.rounds > bvh.n + 1) {  // each full round composites K new hits
        atomicOr(bvh.status, GRT_STATUS_BAD_TREE);
        return true;
    }
    s.last = lastk;
    round_begin(bvh, s, P);
    return false;
}

// Trace one ray through all rounds.  `vis` receives composite(k, id, tau, alpha, T)
// for each composited hit in order (T = transmittance before the hit) and the final
// transmittance via vis.finish(T).  Returns the number of rounds.
template <int K, bool COUNT, class Visitor>
__device__ __forceinline__ int trace_ray(const DevBvh& bvh, const RayState& r, const TraceParams& P, Visitor& vis,
                                         Counters& cnt) {
    LocalStack stack;
    TraceState<K> s;
    trace_begin(bvh, s, r.o, r.d, P);
    while (true) {
        while (trav_step<COUNT>(bvh, s, stack, P, cnt)) {
        }
        if (round_end<COUNT>(bvh, s, P, vis, cnt)) break;
    }
    vis.finish(s.T);
    return s.rounds;
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
#ifndef GRT_SH_INLINE
#define GRT_SH_INLINE 1
#endif
#if GRT_SH_INLINE
#define GRT_SH_ATTR __forceinline__
#else
#define GRT_SH_ATTR __noinline__
#endif
static __device__ GRT_SH_ATTR void surfel_colour_sh(const float* __restrict__ color, int id, f3 d, float c[3]);

__device__ __forceinline__ void surfel_colour(const float* __restrict__ color, int cdim, int id, f3 d, float c[3]) {
    if (cdim == 3) {
        c[0] = __ldg(color + 3 * (size_t)id);
        c[1] = __ldg(color + 3 * (size_t)id + 1);
        c[2] = __ldg(color + 3 * (size_t)id + 2);
        return;
    }
    surfel_colour_sh(color, id, d, c);
}

// SH colour: inline where its callers have one call site (the walks' in-order compositing
// loop), out of line otherwise.
static __device__ GRT_SH_ATTR void surfel_colour_sh(const float* __restrict__ color, int id, f3 d, float c[3]) {
    float Y[16];
    sh_basis(d.x, d.y, d.z, Y);
    const float4* s = reinterpret_cast<const float4*>(color + 48 * (size_t)id);
    float4 sv[12];
    if ((reinterpret_cast<uintptr_t>(color) & 31) == 0) {  // 192-byte rows: 32-byte loads
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const F8 v = ld_v8(s + 2 * q);
            sv[2 * q] = v.a;
            sv[2 * q + 1] = v.b;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 12; ++q) sv[q] = __ldg(s + q);
    }
    float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const float4 v = sv[q];
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

// Lean forward visitor of the shading rays: c_rt only (T comes from the trace state).
// c_rt accumulates w c_k, w = T_k a_k, in compositing order.
__device__ __forceinline__ void accumulate_colour(float c[3], float w, const float ck[3]) {
    c[0] = fmaf(w, ck[0], c[0]);
    c[1] = fmaf(w, ck[1], c[1]);
    c[2] = fmaf(w, ck[2], c[2]);
}

struct RadianceVisitor {
    const float* color;
    int cdim;
    f3 d;
    float c[3];
    __device__ __forceinline__ RadianceVisitor() {}
    __device__ __forceinline__ RadianceVisitor(const float* col, int cd, f3 dir) : color(col), cdim(cd), d(dir) {
        c[0] = c[1] = c[2] = 0.f;
    }

    __device__ __forceinline__ void composite(int, int id, float, float alpha, float Tb) {
        float ck[3];
        surfel_colour(color, cdim, id, d, ck);
        accumulate_colour(c, Tb * alpha, ck);
    }
    __device__ __forceinline__ void finish(float) {}
};

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
    __device__ __forceinline__ ColourVisitor() : color(nullptr), cdim(3), d(mk3(0.f, 0.f, 0.f)), T(1.f),
                                                  hits(nullptr), max_hits(0), nh(0) {
        c[0] = c[1] = c[2] = 0.f;
    }
    __device__ __forceinline__ ColourVisitor(const float* col, int cd, f3 dir, int* h, int mh)
        : color(col), cdim(cd), d(dir), T(1.f), hits(h), max_hits(mh), nh(0) {
        c[0] = c[1] = c[2] = 0.f;
    }
    __device__ __forceinline__ void composite(int k, int id, float, float alpha, float Tb) {
        float ck[3];
        surfel_colour(color, cdim, id, d, ck);
        accumulate_colour(c, Tb * alpha, ck);
        if (hits && k < max_hits) hits[k] = id;
        nh = k + 1;
    }
    __device__ __forceinline__ void finish(float Tf) { T = Tf; }
};


// ----------------------------------------------------------------------------- persistent walk
// Generic persistent two-phase walk over a flat list of `total` rays.  Warps stay resident;
// once kRefill lanes are idle they claim that many rays from *next (a global counter);
// then the warp alternates (A) internal-node visits with hit leaves queued in shared memory,
// until every active lane has kLeafBatch leaves queued or has finished its walk, (B) the queued surfel
// tests of all lanes, (C) compositing of finished walks, once kCompositeBatch of them (or
// all active lanes) are waiting.  Task supplies
//   bool begin(long long ray, WalkState<K>&, Visitor&, const DevBvh*&)  -- false: no ray
//   void end(long long ray, const WalkState<K>&, Visitor&)              -- ray finished
// and the Visitor type receiving composite() calls.
#ifndef GRT_REFILL
#define GRT_REFILL 4
#endif
#ifndef GRT_QUEUE
#define GRT_QUEUE 12
#endif
#ifndef GRT_LEAF_BATCH
#define GRT_LEAF_BATCH 2
#endif
#ifndef GRT_COMPOSITE_BATCH
#define GRT_COMPOSITE_BATCH 12
#endif
// Scheduling of the walk, measured on the 300k-surfel 800x800 workload (M rays/s):
// queue 8 / 12 / 16 / 24 leaves: 339 / 364 / 351 / 333; leaf batch 1 / 2 / 4: 339 / 328 /
// 307; composite batch 1 / 4 / 8 / 16 / 24: 364 / 389 / 394 / 377 / 323 (compositing runs
// the SH colour of each hit, 22 % of the trace time, at 19 % lane use when unbatched);
// refill at 4 / 8 / 12 idle lanes: 397 / 394 / 385.  With rays in bucket order (coherent
// warps): queue 12 / 16 / 20 / 24: 424 / 430 / 429 / 427; refill 2 / 4 / 8: 424 / 424 / 421;
// composite batch 4 / 8 / 12: 417 / 424 / 425; shared stack 8 / 16 / 24 entries: 418 / 424 /
// 424; at least 3 / 4 / 5 blocks per SM: 377 / 424 / 333.  On the current walk (k-buffer in
// shared memory, near cull, restructured tree, 32-byte loads), walk ms with composite batch
// 4 / 8 / 12 / 16: 12.01 / 11.78 / 11.64 / 11.72; leaf batch 1 / 2 / 3: 11.78 / 11.72 / 11.76;
// refill at 2 / 4 / 8: 11.78 / 11.78 / 11.82; composite batch 12 with leaf batch 2: 11.57
// (G-buffer 1.25 -> 1.24 ms, 2M-surfel forward unchanged at 66.7 ms).  With those: queue
// 10 / 12 / 14 leaves: 11.81 / 11.53 / 11.92; shared stack 6 / 8 / 12 entries: 11.78 / 11.53 /
// 11.88; leaf batch 3: 11.59 (2M forward 66.5 ms at the defaults, 67.3-70.1 otherwise).
constexpr int kRefill = GRT_REFILL;         // idle lanes that trigger a refill
constexpr int kQueue = GRT_QUEUE;           // queued leaves per lane
constexpr int kLeafBatch = GRT_LEAF_BATCH;  // leaves every walking lane queues before the tests
constexpr int kCompositeBatch = GRT_COMPOSITE_BATCH;  // finished walks composited together
constexpr int kPersistentThreads = 128;  // block size of every persistent_trace kernel
// Blocks per SM the walk kernels are compiled for (launch bounds): 128 threads x 5 blocks
// leaves at most 96 registers per thread; with the k-buffer in shared memory the walk
// state fits without spills (4 blocks at 111 registers: walk 18.05 ms, 5 blocks with an
// 8-entry shared stack top and 12-leaf queues: 17.08 ms on the 300k-surfel 800x800 frame).
#ifndef GRT_TRACE_MIN_BLOCKS
#define GRT_TRACE_MIN_BLOCKS 5
#endif

static_assert(kPersistentThreads == kKbufThreads, "k-buffer columns are laid out for the persistent block");

// Dynamic shared memory of a persistent walk kernel: its lanes' k-buffers.
template <int K>
constexpr size_t walk_smem_bytes() {
    return (size_t)K * (sizeof(uint64_t) + sizeof(float)) * kPersistentThreads;
}

// A task with a `pos` member learns each ray's position in the walk order before begin().
template <class T, class = void>
struct wants_pos : std::false_type {};
template <class T>
struct wants_pos<T, std::void_t<decltype(std::declval<T&>().pos)>> : std::true_type {};

template <int K, class Task>
__device__ __forceinline__ void persistent_trace(Task& task, const TraceParams& P, unsigned long long* next,
                                                 long long total, int* q, int qstride,
                                                 const unsigned* __restrict__ order = nullptr) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    SplitStack stack;
    if constexpr (kSharedStack > 0) {
        __shared__ int2 shared_stack[kSharedStack * kPersistentThreads];
        stack.sh = shared_stack + threadIdx.x;
        stack.stride = kPersistentThreads;
    }
    extern __shared__ __align__(16) unsigned char walk_smem[];
    WalkState<K> ts;
    ts.kb.key = reinterpret_cast<uint64_t*>(walk_smem) + threadIdx.x;
    ts.kb.a = reinterpret_cast<float*>(reinterpret_cast<uint64_t*>(walk_smem) + K * kPersistentThreads) + threadIdx.x;
    ts.node = -2;
    typename Task::Visitor vis;
    const DevBvh* bvh = nullptr;
    long long ray = -1;
    bool act = false, drained = false;
    int nq = 0;
    Counters cnt{0, 0, 0};
    while (true) {
        unsigned idle = __ballot_sync(0xffffffffu, !act);
        int nidle = __popc(idle);
        if (!drained && (nidle >= kRefill || nidle == 32)) {
            // consecutive rays of the (coherent) walk order from one global counter; per-block
            // chunks of 256 / 1,024 / 4,096 consecutive rays, for L1 reuse within an SM, measured
            // slower (walk 17.08 -> 17.25 / 18.09 / 24.69 ms on the 300k-surfel 800x800 frame)
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(next, (unsigned long long)nidle);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + nidle >= (unsigned long long)total) drained = true;
            if (!act) {
                long long r = (long long)base + __popc(idle & lt);
                if (r < total) {
                    ray = order ? (long long)__ldg(order + r) : r;
                    if constexpr (wants_pos<Task>::value) task.pos = r;
                    act = task.begin(ray, ts, vis, bvh);
                    nq = 0;
                }
            }
        }
        if (!__any_sync(0xffffffffu, act)) {
            if (drained) break;
            continue;
        }
        while (true) {
            bool walking = act && ts.node != -2 && nq <= kQueue - kWide;
            if (!__any_sync(0xffffffffu, walking)) break;
            if (walking) node_step_q<false>(*bvh, ts, stack, P, q, qstride, nq, cnt);
            if (__all_sync(0xffffffffu, !act || nq >= kLeafBatch || ts.node == -2)) break;
        }
        // (an L1 prefetch of every queued record before the tests measured slower: 16.84 ->
        // 17.20 ms; so did one of the buffered hits' SH lines before compositing)
        for (int i = 0; i < nq; ++i) test_leaf<false>(*bvh, ts, q[i * qstride], P, cnt);
        nq = 0;
        // finished walks wait until kCompositeBatch of them (or every active lane) can
        // composite in the same pass
        const bool fin = act && ts.node == -2;
        bool go = fin;
        if (kCompositeBatch > 1) {
            const unsigned fm = __ballot_sync(0xffffffffu, fin);
            const unsigned am = __ballot_sync(0xffffffffu, act);
            go = fin && (__popc(fm) >= kCompositeBatch || fm == am);
        }
        // Evaluating the batch's colours with the whole warp (hits pooled across lanes, owners
        // adding their products in order) measured slower: walk 17.05 -> 17.60 ms.
        if (go) {
            if (round_end<false>(*bvh, ts, P, vis, cnt)) {
                vis.finish(ts.T);
                task.end(ray, ts, vis);
                act = false;
            }
        }
    }
}

// Grid of a persistent walk kernel: as many blocks as fit on the device at once (with
// their dynamic k-buffer memory), at most blocks_max.
template <class Kernel>
inline long long persistent_grid(Kernel kernel, size_t dyn_smem, long long blocks_max) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPersistentThreads, dyn_smem);
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    return grid < blocks_max ? grid : blocks_max;
}

}  // namespace grt
