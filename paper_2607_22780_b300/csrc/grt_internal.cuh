// grt_internal.cuh -- device-side building blocks of libgrt (sm_103a).
//
// Two kinds of arithmetic live here:
//  * "decision" functions (suffix _d): every operation is an explicitly rounded FP32
//    +,-,*,/ or sqrt (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn), never contracted
//    into FMA, in one fixed order.  They decide integer outcomes -- which surfels a ray
//    admits and in which order (Eq. 7-8), which direction a sample takes (Sec. III-D),
//    which environment texel a direction falls in -- so those outcomes are a pure
//    function of the FP32 inputs.
//  * everything else is ordinary FP32 (FMA allowed, fast exp).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/grt.h"

namespace grt {

// ----------------------------------------------------------------------------- vectors
struct f3 {
    float x, y, z;
};
__host__ __device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }

__device__ __forceinline__ float add_d(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_d(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_d(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_d(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_d(float a) { return __fsqrt_rn(a); }

// ((a.x*b.x + a.y*b.y) + a.z*b.z) with every product and sum rounded
__device__ __forceinline__ float dot_d(f3 a, f3 b) {
    float s = mul_d(a.x, b.x);
    s = add_d(s, mul_d(a.y, b.y));
    s = add_d(s, mul_d(a.z, b.z));
    return s;
}
__device__ __forceinline__ f3 norm_d(f3 a) {
    float l = sqrt_d(dot_d(a, a));
    return mk3(div_d(a.x, l), div_d(a.y, l), div_d(a.z, l));
}

__device__ __forceinline__ float dot3(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// ----------------------------------------------------------------------------- Philox
// Philox4x32-10 of Salmon et al. (SC'11): two 32x32->64 multiplies per round, Weyl key
// increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// top 24 bits times 2^-24: exact
__device__ __forceinline__ float unif24(uint32_t x) { return __uint2float_rn(x >> 8) * 0x1p-24f; }

// ----------------------------------------------------------------------------- trig (decision)
// sin, cos of 2*pi*t, t in [0,1]: exact octant reduction, Taylor polynomials on [0,pi/4].
__device__ __forceinline__ void sincos2pi_d(float t, float* so, float* co) {
    float y = mul_d(t, 8.0f);
    float kf = floorf(y);
    int k = ((int)kf) & 7;
    float f = sub_d(y, kf);
    float g = (k & 1) ? sub_d(1.0f, f) : f;
    float x = mul_d(g, 0.785398163397448309616f);
    float x2 = mul_d(x, x);
    float ps = 2.7557319223985890653e-6f;
    ps = add_d(mul_d(ps, x2), -1.9841269841269841270e-4f);
    ps = add_d(mul_d(ps, x2), 8.3333333333333333333e-3f);
    ps = add_d(mul_d(ps, x2), -1.6666666666666666667e-1f);
    float s0 = add_d(x, mul_d(mul_d(x, x2), ps));
    float pc = -2.7557319223985890653e-7f;
    pc = add_d(mul_d(pc, x2), 2.4801587301587301587e-5f);
    pc = add_d(mul_d(pc, x2), -1.3888888888888888889e-3f);
    pc = add_d(mul_d(pc, x2), 4.1666666666666666667e-2f);
    pc = add_d(mul_d(pc, x2), -0.5f);
    float c0 = add_d(1.0f, mul_d(x2, pc));
    float s, c;
    switch (k) {
        case 0: s = s0; c = c0; break;
        case 1: s = c0; c = s0; break;
        case 2: s = c0; c = -s0; break;
        case 3: s = s0; c = -c0; break;
        case 4: s = -s0; c = -c0; break;
        case 5: s = -c0; c = -s0; break;
        case 6: s = -c0; c = s0; break;
        default: s = -s0; c = c0; break;
    }
    *so = s;
    *co = c;
}

// atan2 in radians: a = min/max, reduce past tan(pi/8) with pi/4 + atan((a-1)/(a+1)),
// Taylor series of atan to t^15.
__device__ __forceinline__ float atan2_d(float y, float x) {
    float ax = fabsf(x), ay = fabsf(y);
    float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float a = div_d(mn, mx);
    float base = 0.0f, t = a;
    if (a > 0.414213562373095f) {
        t = div_d(sub_d(a, 1.0f), add_d(a, 1.0f));
        base = 0.785398163397448309616f;
    }
    float t2 = mul_d(t, t);
    float p = -6.6666666666666666667e-2f;
    p = add_d(mul_d(p, t2), 7.6923076923076923077e-2f);
    p = add_d(mul_d(p, t2), -9.0909090909090909091e-2f);
    p = add_d(mul_d(p, t2), 1.1111111111111111111e-1f);
    p = add_d(mul_d(p, t2), -1.4285714285714285714e-1f);
    p = add_d(mul_d(p, t2), 2.0e-1f);
    p = add_d(mul_d(p, t2), -3.3333333333333333333e-1f);
    float r = add_d(base, add_d(t, mul_d(mul_d(t, t2), p)));
    if (ay > ax) r = sub_d(1.57079632679489661923f, r);
    if (x < 0.0f) r = sub_d(3.14159265358979323846f, r);
    if (y < 0.0f) r = -r;
    return r;
}

// Surfel normal: third column of R(q/|q|), q = (w,x,y,z).
__device__ __forceinline__ f3 normal_from_quat_d(float w, float x, float y, float z) {
    float s2 = mul_d(w, w);
    s2 = add_d(s2, mul_d(x, x));
    s2 = add_d(s2, mul_d(y, y));
    s2 = add_d(s2, mul_d(z, z));
    float s = sqrt_d(s2);
    w = div_d(w, s);
    x = div_d(x, s);
    y = div_d(y, s);
    z = div_d(z, s);
    float nx = mul_d(2.0f, add_d(mul_d(x, z), mul_d(w, y)));
    float ny = mul_d(2.0f, sub_d(mul_d(y, z), mul_d(w, x)));
    float nz = sub_d(1.0f, mul_d(2.0f, add_d(mul_d(x, x), mul_d(y, y))));
    return mk3(nx, ny, nz);
}

// Orthonormal basis of Duff et al., "Building an Orthonormal Basis, Revisited" (2017).
__device__ __forceinline__ void frame_d(f3 n, f3* b1, f3* b2) {
    float sign = n.z >= 0.0f ? 1.0f : -1.0f;
    float a = div_d(-1.0f, add_d(sign, n.z));
    float b = mul_d(mul_d(n.x, n.y), a);
    *b1 = mk3(add_d(1.0f, mul_d(mul_d(mul_d(sign, n.x), n.x), a)), mul_d(sign, b), -mul_d(sign, n.x));
    *b2 = mk3(b, add_d(sign, mul_d(mul_d(n.y, n.y), a)), -n.y);
}

__device__ __forceinline__ f3 to_world_d(f3 b1, f3 b2, f3 n, f3 l) {
    return mk3(add_d(add_d(mul_d(b1.x, l.x), mul_d(b2.x, l.y)), mul_d(n.x, l.z)),
               add_d(add_d(mul_d(b1.y, l.x), mul_d(b2.y, l.y)), mul_d(n.y, l.z)),
               add_d(add_d(mul_d(b1.z, l.x), mul_d(b2.z, l.y)), mul_d(n.z, l.z)));
}

// Cosine-weighted direction (Malley's method).
__device__ __forceinline__ f3 sample_cos_d(f3 n, f3 b1, f3 b2, float u0, float u1) {
    float r = sqrt_d(u0);
    float s, c;
    sincos2pi_d(u1, &s, &c);
    float lz = sub_d(1.0f, u0);
    lz = sqrt_d(lz > 0.0f ? lz : 0.0f);
    return to_world_d(b1, b2, n, mk3(mul_d(r, c), mul_d(r, s), lz));
}

// GGX visible normals (Heitz 2018), reflected about the sampled normal; false when w_o is
// below the hemisphere.
__device__ __forceinline__ bool sample_ggx_d(f3 n, f3 b1, f3 b2, f3 wo, float rough, float u0, float u1,
                                             f3* out) {
    f3 v = mk3(dot_d(wo, b1), dot_d(wo, b2), dot_d(wo, n));
    if (!(v.z > 0.0f)) return false;
    float a = mul_d(rough, rough);
    if (a < 1e-4f) a = 1e-4f;
    f3 vh = norm_d(mk3(mul_d(a, v.x), mul_d(a, v.y), v.z));
    float lensq = add_d(mul_d(vh.x, vh.x), mul_d(vh.y, vh.y));
    f3 T1;
    if (lensq > 0.0f) {
        float l = sqrt_d(lensq);
        T1 = mk3(div_d(-vh.y, l), div_d(vh.x, l), 0.0f);
    } else {
        T1 = mk3(1.0f, 0.0f, 0.0f);
    }
    f3 T2 = mk3(sub_d(mul_d(vh.y, T1.z), mul_d(vh.z, T1.y)), sub_d(mul_d(vh.z, T1.x), mul_d(vh.x, T1.z)),
                sub_d(mul_d(vh.x, T1.y), mul_d(vh.y, T1.x)));
    float r = sqrt_d(u0);
    float s, c;
    sincos2pi_d(u1, &s, &c);
    float t1 = mul_d(r, c), t2 = mul_d(r, s);
    float sh = mul_d(0.5f, add_d(1.0f, vh.z));
    float q1 = sub_d(1.0f, mul_d(t1, t1));
    t2 = add_d(mul_d(sub_d(1.0f, sh), sqrt_d(q1 > 0.0f ? q1 : 0.0f)), mul_d(sh, t2));
    float q2 = sub_d(q1, mul_d(t2, t2));
    float nz = sqrt_d(q2 > 0.0f ? q2 : 0.0f);
    f3 nh = mk3(add_d(add_d(mul_d(t1, T1.x), mul_d(t2, T2.x)), mul_d(nz, vh.x)),
                add_d(add_d(mul_d(t1, T1.y), mul_d(t2, T2.y)), mul_d(nz, vh.y)),
                add_d(add_d(mul_d(t1, T1.z), mul_d(t2, T2.z)), mul_d(nz, vh.z)));
    f3 ne = mk3(mul_d(a, nh.x), mul_d(a, nh.y), nh.z > 0.0f ? nh.z : 0.0f);
    float ll = dot_d(ne, ne);
    ne = ll > 0.0f ? norm_d(ne) : mk3(0.0f, 0.0f, 1.0f);
    float d2 = mul_d(2.0f, dot_d(v, ne));
    f3 wl = mk3(sub_d(mul_d(d2, ne.x), v.x), sub_d(mul_d(d2, ne.y), v.y), sub_d(mul_d(d2, ne.z), v.z));
    *out = to_world_d(b1, b2, n, wl);
    return true;
}

// Largest i in [0, n-1] with cdf[i] <= u.
__device__ __forceinline__ int cdf_search(const float* __restrict__ cdf, int n, float u) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void texel_of_d(f3 d, int W, int H, int* row, int* col) {
    float phi = atan2_d(d.x, d.z);
    if (phi < 0.0f) phi = add_d(phi, 6.28318530717958647692f);
    float cf = mul_d(mul_d(phi, 0.159154943091895335769f), (float)W);
    int c = (int)floorf(cf);
    c = c < 0 ? 0 : (c > W - 1 ? W - 1 : c);
    float sxz = sqrt_d(add_d(mul_d(d.x, d.x), mul_d(d.z, d.z)));
    float th = atan2_d(sxz, d.y);
    float rf = mul_d(mul_d(th, 0.318309886183790671538f), (float)H);
    int r = (int)floorf(rf);
    r = r < 0 ? 0 : (r > H - 1 ? H - 1 : r);
    *row = r;
    *col = c;
}

__device__ __forceinline__ f3 env_dir_d(int row, int col, float u_row, float u_col, int W, int H) {
    float xp = div_d(add_d((float)col, u_col), (float)W);
    float xt = div_d(add_d((float)row, u_row), (float)H);
    float sp, cp, st, ct;
    sincos2pi_d(xp, &sp, &cp);
    sincos2pi_d(mul_d(xt, 0.5f), &st, &ct);
    return mk3(mul_d(st, sp), ct, mul_d(st, cp));
}

// ----------------------------------------------------------------------------- BVH layout
// Traversal runs on a 4-wide BVH collapsed from the binary radix tree.  Wide node b is
// made from binary node b (the root is 0 in both); nodes that no traversal from the root
// reaches are built but unused.
// Wide node: 128 bytes = 8 float4
//   [0..2] lo.x, lo.y, lo.z of the four children, [3..5] hi.x, hi.y, hi.z
//   [6]    child refs (int bits): >= 0 wide node, kRefEmpty unused slot, any other
//          negative value a leaf -(1 + (first record << 3) + (count - 1)), count <= kLeafMax
//   [7]    binary-tree ref of each child (to refit boxes without a rebuild)
// Unused slots have lo = +1e38 > hi = -1e38, so every slab test misses them.
constexpr int kWide = 4;
#ifndef GRT_LEAF_MAX
#define GRT_LEAF_MAX 1
#endif
constexpr int kLeafMax = GRT_LEAF_MAX;  // surfels per wide-tree leaf (at most 8)
__host__ __device__ __forceinline__ int leaf_ref(int first, int count) { return -(1 + (first << 3) + (count - 1)); }
__host__ __device__ __forceinline__ int leaf_first(int ref) { return (-ref - 1) >> 3; }
__host__ __device__ __forceinline__ int leaf_count(int ref) { return ((-ref - 1) & 7) + 1; }
//
// Binary radix tree (built first, kept for refits):
// Internal node: 64 bytes = 4 float4
//   f[0..5]  left child box  (lo.xyz, hi.xyz)
//   f[6..11] right child box (lo.xyz, hi.xyz)
//   f[12], f[13] child refs (int bits): >= 0 internal node index, < 0 leaf ~record_index
// Packed surfel record (sorted by Morton code): 64 bytes = 4 float4
//   r0 = (mu.xyz, opacity)          r1 = (n.xyz, surfel id as int bits)
//   r2 = (t_u/s_u .xyz, r2_cut)     r3 = (t_v/s_v .xyz, unused)
// with n the decision normal and r2_cut = 2 ln(opacity / alpha_min) (a hit needs
// u^2+v^2 <= r2_cut).
constexpr int kRefEmpty = (int)0x80000000;

struct DevBvh {
    const float4* nodes;    // wide nodes [cap * 8]
    const float4* records;  // [n * 4]
    const float4* normals;  // [n] decision normal of each surfel by id (xyz, 0), from the build
    int root;               // wide node 0, a leaf ref when n == 1, kRefEmpty when n == 0
    int n;
    int cap;                // wide node capacity (n - 1)
    int* status;
};

}  // namespace grt

// Host-side definition of the opaque handle.
struct grt_bvh {
    char* base;        // single device allocation holding every array below
    int n;
    int n_int;
    float4* nodes;
    float4* records;
    float4* normals;   // [n] decision normal of surfel i at i (surfel trees only)
    int* parent;       // [n + n_int]: (parent node << 1) | slot, root has -1
    int* refit_flags;  // [n_int]
    float* leaf_box;   // [n * 6] in sorted order
    int* sorted_ids;   // [n]
    float4* wnodes;    // [n_int * 8] 4-wide nodes
    float* bin_box;    // [n_int * 6] box of each binary node
    float4* dp_cost;   // [n_int] collapse costs of each binary node's subtree in 1..4 slots
    unsigned* dp_dec;  // [n_int] the splits those costs take
    int* status;       // device status word
    float* bounds;     // [6] scene bounds (device)
    size_t bytes;
    int device;
};

namespace grt {
// error plumbing (api.cu)
int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);
DevBvh dev_bvh(const grt_bvh* b);
}  // namespace grt

#define GRT_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) return grt::check_cuda(e__, #call); \
    } while (0)
