// bvh.cu -- linear BVH over 2D Gaussian surfels, built on the device.
//
// The paper bounds each surfel by an icosahedron proxy scaled by sqrt(2 log(o/alpha_min))
// (Eq. 6) and hands the triangles to OptiX's hardware BVH (Sec. III-B).  B300 has no RT
// cores, so the surfels are bounded directly by the axis-aligned box of the same
// alpha_min ellipse and indexed by a software LBVH:
//   1. prep      per surfel: decision normal, scaled tangents, ellipse box, box centre
//   2. bounds    scene box of the centres (one block-reduced pass, atomics on ordered ints)
//   3. morton    30-bit Morton code of each centre in the scene box
//   4. sort      LSD radix sort of (code, id), 8-bit digits, stable block-local ranking
//   5. records   packed 64-byte records in sorted order (coalesced traversal reads)
//   6. hierarchy binary radix tree over the sorted codes (Karras, HPG 2012), duplicate
//                codes split by position, so the depth is at most 30 + log2(n)
//   7. refit     bottom-up box union, second arriving thread continues (atomic flags)
//   8. collapse  4-wide tree for traversal, top down in one launch (device work queue)
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <mutex>

#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr int kThreads = 256;
// 30-bit Morton codes: 63-bit codes (21 bits per axis) left the trees of the 300k-surfel
// and the 2M-surfel unbounded scenes unchanged in node visits per ray (43.26 and 134.4
// vs 135.6) at twice the sort passes and more collapse levels.
using MortonKey = unsigned int;

__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// Per-surfel frame from the quaternion (ordinary FP32): columns of R(q/|q|).
__device__ __forceinline__ void frame_fast(float4 q, f3* tu, f3* tv) {
    float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    *tu = mk3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    *tv = mk3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
}

struct SurfelIn {
    const float* mu;
    const float* quat;
    const float* scale;
    const float* opacity;
    int n;
    float alpha_min;
};

// Ellipse box: rho = sqrt(2 ln(o/alpha_min)); half extent along axis x is
// rho * sqrt((s_u t_u.x)^2 + (s_v t_v.x)^2).  Padded by 1e-5 of the extent plus 4e-7 of
// the coordinate magnitude so FP32 rounding of later tests never escapes the box.
__device__ __forceinline__ void surfel_box(const SurfelIn& s, int i, float lo[3], float hi[3], f3* tu, f3* tv,
                                           float* r2cut) {
    float4 q = make_float4(s.quat[4 * i], s.quat[4 * i + 1], s.quat[4 * i + 2], s.quat[4 * i + 3]);
    frame_fast(q, tu, tv);
    float su = s.scale[2 * i], sv = s.scale[2 * i + 1];
    float o = s.opacity[i];
    float c = o > s.alpha_min ? 2.f * logf(o / s.alpha_min) : 0.f;
    *r2cut = o >= s.alpha_min ? c : -1.f;
    float rho = sqrtf(fmaxf(c, 0.f)) * (1.f + 1e-5f);
    float m[3] = {s.mu[3 * i], s.mu[3 * i + 1], s.mu[3 * i + 2]};
    float a[3] = {su * tu->x, su * tu->y, su * tu->z};
    float b[3] = {sv * tv->x, sv * tv->y, sv * tv->z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float e = rho * sqrtf(a[k] * a[k] + b[k] * b[k]);
        float pad = 1e-5f * e + 4e-7f * (fabsf(m[k]) + e) + 1e-9f;
        lo[k] = m[k] - e - pad;
        hi[k] = m[k] + e + pad;
    }
}

__device__ __forceinline__ void reduce_bounds(const float cl[3], const float ch[3], const float lo[3],
                                              const float hi[3], unsigned int* __restrict__ bounds_u);

__global__ void k_prep_bounds(SurfelIn s, float* __restrict__ centre, unsigned int* __restrict__ bounds_u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    float cl[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, ch[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (i < s.n) {
        f3 tu, tv;
        float r2;
        surfel_box(s, i, lo, hi, &tu, &tv, &r2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float c = 0.5f * (lo[k] + hi[k]);
            centre[3 * i + k] = c;
            cl[k] = c;
            ch[k] = c;
        }
    }
    reduce_bounds(cl, ch, lo, hi, bounds_u);
}

// Warp then block reduction of centre bounds and box bounds into bounds_u (ordered ints:
// [0..2] min centre, [3..5] -max centre, [6..8] min box, [9..11] -max box).
__device__ __forceinline__ void reduce_bounds(const float cl[3], const float ch[3], const float lo[3],
                                              const float hi[3], unsigned int* __restrict__ bounds_u) {
    __shared__ float red[12][kThreads / 32];
    float v[12] = {cl[0], cl[1], cl[2], -ch[0], -ch[1], -ch[2], lo[0], lo[1], lo[2], -hi[0], -hi[1], -hi[2]};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        float x = red[threadIdx.x][0];
        for (int w = 1; w < kThreads / 32; ++w) x = fminf(x, red[threadIdx.x][w]);
        atomicMin(bounds_u + threadIdx.x, float_to_ordered(x));
    }
}

// 30-bit spatial key of each surfel centre.  The bits are taken most significant first, and
// each one halves the axis whose cell is currently the longest, as a kd-tree split of the
// longest side would; on a cubic extent this is the usual x/y/z Morton interleave, while a
// flat scene's thin axis is split less often than its long ones (on the 300k-surfel scene:
// 39.4 instead of 43.3 node visits per secondary ray).  Every thread derives the same axis
// sequence from the centre bounds; an axis takes at most 21 bits.
__global__ void k_morton(const float* __restrict__ centre, const unsigned int* __restrict__ bounds_u, int n,
                         MortonKey* __restrict__ keys, int* __restrict__ vals, float* __restrict__ bounds_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3], ext[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = ordered_to_float(bounds_u[k]);
        float hi = -ordered_to_float(bounds_u[3 + k]);
        ext[k] = fmaxf(hi - lo[k], 1e-30f);
    }
    if (i == 0 && bounds_out) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            bounds_out[k] = ordered_to_float(bounds_u[6 + k]);
            bounds_out[3 + k] = -ordered_to_float(bounds_u[9 + k]);
        }
    }
    // axis order of the key bits, the same for every surfel: one thread per block derives it
    __shared__ unsigned int order_s[3];  // seq_lo, seq_hi, nb0 | nb1 << 8 | nb2 << 16
    if (threadIdx.x == 0) {
        int nb0 = 0, nb1 = 0, nb2 = 0;
        float cx = ext[0], cy = ext[1], cz = ext[2];  // cell size per axis (halving is exact)
        unsigned seq_lo = 0, seq_hi = 0;               // 2 bits per key bit: the axis it splits
        for (int b = 0; b < 30; ++b) {
            int a = (cx >= cy && cx >= cz) ? 0 : (cy >= cz ? 1 : 2);
            if ((a == 0 ? nb0 : a == 1 ? nb1 : nb2) >= 21) a = nb0 < 21 ? 0 : (nb1 < 21 ? 1 : 2);
            nb0 += a == 0;
            nb1 += a == 1;
            nb2 += a == 2;
            cx = a == 0 ? 0.5f * cx : cx;
            cy = a == 1 ? 0.5f * cy : cy;
            cz = a == 2 ? 0.5f * cz : cz;
            if (b < 16) seq_lo |= (unsigned)a << (2 * b);
            else seq_hi |= (unsigned)a << (2 * (b - 16));
        }
        order_s[0] = seq_lo;
        order_s[1] = seq_hi;
        order_s[2] = (unsigned)nb0 | ((unsigned)nb1 << 8) | ((unsigned)nb2 << 16);
    }
    __syncthreads();
    if (i >= n) return;
    const unsigned seq_lo = order_s[0], seq_hi = order_s[1];
    const int nb0 = (int)(order_s[2] & 0xFF), nb1 = (int)((order_s[2] >> 8) & 0xFF), nb2 = (int)(order_s[2] >> 16);
    unsigned int q[3];
    const int nbs[3] = {nb0, nb1, nb2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float cells = (float)(1u << nbs[k]);
        float t = (centre[3 * i + k] - lo[k]) / ext[k];
        t = fminf(fmaxf(t * cells, 0.f), cells - 1.f);
        q[k] = (unsigned int)t;
    }
    // the bits of each axis, most significant first, in the order above
    int r0 = nb0, r1 = nb1, r2 = nb2;
    unsigned int code = 0;
    for (int b = 0; b < 30; ++b) {
        const int a = (int)((b < 16 ? seq_lo >> (2 * b) : seq_hi >> (2 * (b - 16))) & 3u);
        const unsigned qa = a == 0 ? q[0] : a == 1 ? q[1] : q[2];
        const int ra = a == 0 ? r0 : a == 1 ? r1 : r2;
        code = (code << 1) | ((qa >> (ra - 1)) & 1u);
        r0 -= a == 0;
        r1 -= a == 1;
        r2 -= a == 2;
    }
    keys[i] = code;
    vals[i] = i;
}

// ---------------------------------------------------------------- radix sort (LSD, 8-bit digits)
constexpr int kSortThreads = 256;
// 2,048 keys per tile: 147 scatter blocks for 300k keys (4,096-key tiles left half the SMs
// without a block)
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void k_sort_hist(const MortonKey* __restrict__ keys, int n, int shift, int nblocks,
                            unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m counts in one block of 1024 threads (digit-major layout), 8,192 counts
// at a time: a coalesced copy into shared memory (one pad word per 32, so that the
// threads' contiguous runs of 8 fall in distinct banks), a scan of the runs' sums over the
// block by warp shuffles, and a coalesced copy back.
constexpr int kScanThreads = 1024, kScanRun = 8, kScanSeg = kScanThreads * kScanRun;

__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kScanThreads) k_sort_scan(unsigned int* __restrict__ hist, int m) {
    __shared__ unsigned int seg[kScanSeg + kScanSeg / 32];
    __shared__ unsigned int wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int carry = 0;
    for (int base = 0; base < m; base += kScanSeg) {
        const int len = min(kScanSeg, m - base);
#pragma unroll
        for (int k = 0; k < kScanRun; ++k) {
            const int i = k * kScanThreads + threadIdx.x;
            seg[scan_pad(i)] = i < len ? hist[base + i] : 0u;
        }
        __syncthreads();
        const int b = threadIdx.x * kScanRun;
        unsigned int v[kScanRun], sum = 0;
#pragma unroll
        for (int k = 0; k < kScanRun; ++k) {
            v[k] = seg[scan_pad(b + k)];
            sum += v[k];
        }
        unsigned int x = sum;  // inclusive scan of the run sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        unsigned int run = carry + (warp ? wsum[warp - 1] : 0u) + x - sum;
#pragma unroll
        for (int k = 0; k < kScanRun; ++k) {
            seg[scan_pad(b + k)] = run;
            run += v[k];
        }
        carry += wsum[31];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanRun; ++k) {
            const int i = k * kScanThreads + threadIdx.x;
            if (i < len) hist[base + i] = seg[scan_pad(i)];
        }
        __syncthreads();  // seg and wsum are reused by the next segment
    }
}

// Stable scatter: keys of a tile are ranked in rounds of 256 in index order; within a
// warp by __match_any_sync, across warps by a prefix over per-warp digit counts.
__global__ void k_sort_scatter(const MortonKey* __restrict__ keys_in, const int* __restrict__ vals_in, int n,
                               int shift, int nblocks, const unsigned int* __restrict__ offs,
                               MortonKey* __restrict__ keys_out, int* __restrict__ vals_out) {
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned int run[256];
    __shared__ unsigned int wcnt[W][256];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    unsigned int lt = (1u << lane) - 1u;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kSortThreads + threadIdx.x;
        bool ok = i < n;
        MortonKey key = ok ? keys_in[i] : 0u;
        int val = ok ? vals_in[i] : 0;
        unsigned int d = ok ? (unsigned int)((key >> shift) & 0xFF) : 256u + (unsigned)lane;  // unique dummies
        unsigned int peers = __match_any_sync(0xffffffffu, d);
        unsigned int rank = __popc(peers & lt);
        if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // prefix over warps per digit (thread = digit)
        {
            unsigned int s = run[threadIdx.x];
            for (int w = 0; w < W; ++w) {
                unsigned int c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = s;
                s += c;
            }
            run[threadIdx.x] = s;
        }
        __syncthreads();
        if (ok) {
            unsigned int pos = wcnt[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- triangles (mesh backend)
// The same tree over triangles: each leaf is one triangle, bounded by the box of its three
// vertices; the record of leaf j is (v0, triangle id), (v1, 0), (v2, 0), unused.
struct TriIn {
    const float* pos;
    const int* tri;
    int n, nv;
    int* status;
};

__device__ __forceinline__ void tri_box(const TriIn& t, int i, float lo[3], float hi[3], f3 v[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int vi = t.tri[3 * i + c];
        if ((unsigned)vi >= (unsigned)t.nv) {  // a vertex index outside the mesh: reported, vertex 0 used
            atomicOr(t.status, GRT_STATUS_BAD_INDEX);
            vi = 0;
        }
        v[c] = mk3(t.pos[3 * (size_t)vi], t.pos[3 * (size_t)vi + 1], t.pos[3 * (size_t)vi + 2]);
    }
    lo[0] = fminf(v[0].x, fminf(v[1].x, v[2].x));
    lo[1] = fminf(v[0].y, fminf(v[1].y, v[2].y));
    lo[2] = fminf(v[0].z, fminf(v[1].z, v[2].z));
    hi[0] = fmaxf(v[0].x, fmaxf(v[1].x, v[2].x));
    hi[1] = fmaxf(v[0].y, fmaxf(v[1].y, v[2].y));
    hi[2] = fmaxf(v[0].z, fmaxf(v[1].z, v[2].z));
}

__global__ void k_tri_prep(TriIn t, float* __restrict__ centre, unsigned int* __restrict__ bounds_u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    float cl[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, ch[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (i < t.n) {
        f3 v[3];
        tri_box(t, i, lo, hi, v);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float c = 0.5f * (lo[k] + hi[k]);
            centre[3 * i + k] = c;
            cl[k] = c;
            ch[k] = c;
        }
    }
    reduce_bounds(cl, ch, lo, hi, bounds_u);
}

__global__ void k_tri_records(TriIn t, const int* __restrict__ sorted, float4* __restrict__ records,
                              float* __restrict__ leaf_box) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= t.n) return;
    const int i = sorted[j];
    float lo[3], hi[3];
    f3 v[3];
    tri_box(t, i, lo, hi, v);
    float4* rec = records + 4 * (size_t)j;
    rec[0] = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float(i));
    rec[1] = make_float4(v[1].x, v[1].y, v[1].z, 0.f);
    rec[2] = make_float4(v[2].x, v[2].y, v[2].z, 0.f);
    rec[3] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        leaf_box[6 * (size_t)j + k] = lo[k];
        leaf_box[6 * (size_t)j + 3 + k] = hi[k];
    }
}

// ---------------------------------------------------------------- records
struct RecordIn {
    SurfelIn s;
    const int* sorted;
    float4* records;
    float4* normals;
    float* leaf_box;
};

__global__ void k_records(RecordIn r) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= r.s.n) return;
    int i = r.sorted[j];
    float lo[3], hi[3], r2cut;
    f3 tu, tv;
    surfel_box(r.s, i, lo, hi, &tu, &tv, &r2cut);
    const float* q = r.s.quat + 4 * i;
    f3 nd = normal_from_quat_d(q[0], q[1], q[2], q[3]);
    float su = r.s.scale[2 * i], sv = r.s.scale[2 * i + 1];
    float4* rec = r.records + 4 * (size_t)j;
    rec[0] = make_float4(r.s.mu[3 * i], r.s.mu[3 * i + 1], r.s.mu[3 * i + 2], r.s.opacity[i]);
    rec[1] = make_float4(nd.x, nd.y, nd.z, __int_as_float(i));
    rec[2] = make_float4(tu.x / su, tu.y / su, tu.z / su, r2cut);
    rec[3] = make_float4(tv.x / sv, tv.y / sv, tv.z / sv, 0.f);
    r.normals[i] = make_float4(nd.x, nd.y, nd.z, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.leaf_box[6 * (size_t)j + k] = lo[k];
        r.leaf_box[6 * (size_t)j + 3 + k] = hi[k];
    }
}

// ---------------------------------------------------------------- hierarchy (Karras 2012)
__device__ __forceinline__ int delta(const MortonKey* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    MortonKey a = k[i], b = k[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((unsigned int)(i ^ j));
}

__global__ void k_hierarchy(const MortonKey* __restrict__ keys, int n, float4* __restrict__ nodes,
                            int* __restrict__ parent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        int t = (l + div - 1) / div;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int gamma = i + s * d + (d < 0 ? -1 : 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)i);
    f[12] = __int_as_float(left);
    f[13] = __int_as_float(right);
    f[14] = __int_as_float(lo);  // sorted-record range covered by this node
    f[15] = __int_as_float(hi);
    // parent table: leaves at [0, n), internal nodes at n + index
    parent[left < 0 ? ~left : n + left] = (i << 1) | 0;
    parent[right < 0 ? ~right : n + right] = (i << 1) | 1;
    if (i == 0) parent[n] = -1;
}

__device__ __forceinline__ int atomic_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__global__ void k_refit(const float* __restrict__ leaf_box, const int* __restrict__ parent, int n,
                        float4* __restrict__ nodes, int* __restrict__ flags, int* status, float* __restrict__ bin_box) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float b[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k] = leaf_box[6 * (size_t)j + k];
    int p = parent[j];
    for (int level = 0; p >= 0; ++level) {
        if (level > 255 || (p >> 1) >= n - 1) {  // deeper than any tree over 2^27 leaves
            atomicOr(status, GRT_STATUS_BAD_TREE);
            return;
        }
        const int node = p >> 1, slot = p & 1;
        const int up = parent[n + node];  // read ahead of the handshake
        float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)node);
#pragma unroll
        for (int k = 0; k < 6; ++k) f[6 * slot + k] = b[k];
        // release: this box is visible to the sibling's thread once it sees the count;
        // acquire: the sibling's box is visible here once this thread sees its count
        if (atomic_add_acq_rel(flags + node, 1) == 0) return;  // first arrival: the sibling finishes
        const float* g = f + 6 * (1 - slot);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b[k] = fminf(b[k], __ldcg(g + k));
            b[3 + k] = fmaxf(b[3 + k], __ldcg(g + 3 + k));
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) bin_box[6 * (size_t)node + k] = b[k];
        p = up;
    }
}

__device__ __forceinline__ float half_area(const float* b) {
    float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

// ---------------------------------------------------------------- treelet restructuring
// Agglomerative treelet restructuring of the radix tree (after Domingues & Pedrini 2015, on
// Karras & Aila's treelet scheme): one bottom-up pass with the refit's arrival counters;
// the second thread to reach node R forms R's treelet -- R's two children, then repeatedly
// the treelet leaf of largest surface area replaced by its two children, up to kTreelet
// treelet leaves -- and rebuilds it by greedy agglomeration (the pair whose union has the
// smallest area merged first).  The new topology replaces the old one only when the summed
// surface area of the treelet's internal nodes (the surface-area cost of the treelet, its
// root and leaves being fixed) drops.  Nodes reuse the treelet's internal indices, R stays
// the root, so nothing outside the treelet changes.  Every read of the tree goes to L2:
// other threads rewrote the descendants, ordered by the acq_rel counters.  After a pass an
// internal node's key range no longer holds: f[14] = 0, f[15] = leaf count - 1, so that
// only the size survives (multi-surfel leaves need contiguous ranges: kLeafMax == 1 only).
constexpr int kTreelet = 9;

__device__ __forceinline__ int node_size_cg(const float4* bn, int ref) {
    if (ref < 0) return 1;
    const float* f = reinterpret_cast<const float*>(bn + 4 * (size_t)ref);
    return __float_as_int(__ldcg(f + 15)) - __float_as_int(__ldcg(f + 14)) + 1;
}

// Pairs (a, b), a < b < kTreelet, in order: pair p is handled by lane p % 32.
__constant__ unsigned char c_pair_a[36] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2,
                                           2, 2, 2, 3, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 6, 6, 7};
__constant__ unsigned char c_pair_b[36] = {1, 2, 3, 4, 5, 6, 7, 8, 2, 3, 4, 5, 6, 7, 8, 3, 4, 5,
                                           6, 7, 8, 4, 5, 6, 7, 8, 5, 6, 7, 8, 6, 7, 8, 7, 8, 8};
static_assert(kTreelet == 9, "the pair table enumerates the pairs of 9 treelet leaves");

// One treelet at root R, processed by the whole warp (R the same on every lane).  Lane k
// holds treelet leaf k (its ref, box, leaf count) and, during the agglomeration, cluster
// k; lane m records merge m; lane k holds the treelet's internal index inner[k].
__device__ void restructure_treelet(int R, const float* __restrict__ leaf_box, int* __restrict__ parent, int n,
                                    float4* __restrict__ nodes, float* __restrict__ bin_box, int* status) {
    const int lane = threadIdx.x & 31;
    auto bad = [n](int ref) { return ref >= 0 ? ref >= n - 1 : ~ref >= n; };
    // a binary node holds both children's boxes and refs: one 64-byte load per expansion
    // (the same address on every lane)
    auto load_node = [&](int x, float (&cb)[12], int* cl, int* cr) {
        const float4* q = nodes + 4 * (size_t)x;
        const float4 v0 = __ldcg(q), v1 = __ldcg(q + 1), v2 = __ldcg(q + 2), v3 = __ldcg(q + 3);
        cb[0] = v0.x; cb[1] = v0.y; cb[2] = v0.z; cb[3] = v0.w; cb[4] = v1.x; cb[5] = v1.y;
        cb[6] = v1.z; cb[7] = v1.w; cb[8] = v2.x; cb[9] = v2.y; cb[10] = v2.z; cb[11] = v2.w;
        *cl = __float_as_int(v3.x);
        *cr = __float_as_int(v3.y);
    };
    int ref = 0;
    float bx[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int inner = R;
    // a lane whose treelet leaf is a binary node holds that node's children (boxes, refs),
    // loaded as soon as the leaf appears: an expansion then shuffles them from the lane
    // instead of waiting for a dependent load
    float nb[12];
    int ncl = 0, ncr = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) nb[c] = 0.f;
    {
        float cb[12];
        int cl, cr;
        load_node(R, cb, &cl, &cr);
        if (bad(cl) || bad(cr)) {
            if (lane == 0) atomicOr(status, GRT_STATUS_BAD_TREE);
            return;
        }
        if (lane < 2) {
            ref = lane == 0 ? cl : cr;
#pragma unroll
            for (int c = 0; c < 6; ++c) bx[c] = lane == 0 ? cb[c] : cb[6 + c];
            if (ref >= 0) load_node(ref, nb, &ncl, &ncr);
        }
    }
    int nt = 2;
    float cost_old = 0.f;
    for (int it = 0; it < kTreelet - 2; ++it) {
        // the largest area among the treelet's binary-node leaves, ties to the lower lane:
        // one max reduction over (area bits with the low 5 replaced by 31 - lane); 0 = none
        const float area = half_area(bx);
        const unsigned mine = (lane < nt && ref >= 0) ? ((__float_as_uint(fmaxf(area, 0.f)) & ~31u) | (31u - lane)) : 0u;
        const unsigned top = __reduce_max_sync(0xffffffffu, mine);
        if (top == 0u) break;  // every treelet leaf is a surfel
        const int best = 31 - (int)(top & 31u);
        const float key = __shfl_sync(0xffffffffu, area, best);
        const int x = __shfl_sync(0xffffffffu, ref, best);
        float cb[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) cb[c] = __shfl_sync(0xffffffffu, nb[c], best);
        const int cl = __shfl_sync(0xffffffffu, ncl, best), cr = __shfl_sync(0xffffffffu, ncr, best);
        if (bad(cl) || bad(cr)) {
            if (lane == 0) atomicOr(status, GRT_STATUS_BAD_TREE);
            return;
        }
        if (lane == nt - 1) inner = x;
        cost_old += key;
        if (lane == best || lane == nt) {
            const int side = lane == best ? 0 : 1;
            ref = side ? cr : cl;
#pragma unroll
            for (int c = 0; c < 6; ++c) bx[c] = side ? cb[6 + c] : cb[c];
            if (ref >= 0) load_node(ref, nb, &ncl, &ncr);
        }
        ++nt;
    }
    if (nt < 3) return;  // two subtrees: only one topology
    const int cnt = lane < nt ? node_size_cg(nodes, ref) : 0;
    float ob[6];  // the treelet leaf's own box (bx becomes the cluster's)
#pragma unroll
    for (int c = 0; c < 6; ++c) ob[c] = bx[c];
    // greedy agglomeration; cluster refs: treelet leaf k, or merge m marked kMerged | m.  The
    // last merge (m = nt - 2) is the root R = inner[0]; merge m < nt - 2 takes inner[m + 1].
    constexpr int kMerged = 1 << 30;
    int cref = lane, ccnt = cnt;
    int mlft = 0, mrgt = 0, mcnt = 0;
    float mbox[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned active = (1u << nt) - 1u;
    float cost_new = 0.f;
    const int pa0 = c_pair_a[lane], pb0 = c_pair_b[lane];
    const int p1 = lane + 32 < 36 ? lane + 32 : 35;
    const int pa1 = c_pair_a[p1], pb1 = c_pair_b[p1];
    // union area of a lane's pair from the two clusters' boxes (shuffled from their lanes);
    // a pair keeps its value until one of its clusters changes
    auto pair_area = [&](int pa_, int pb_) {
        float lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(__shfl_sync(0xffffffffu, bx[c], pa_), __shfl_sync(0xffffffffu, bx[c], pb_));
            hi[c] = fmaxf(__shfl_sync(0xffffffffu, bx[3 + c], pa_), __shfl_sync(0xffffffffu, bx[3 + c], pb_));
        }
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return dx * dy + dy * dz + dz * dx;
    };
    float d0 = pair_area(pa0, pb0), d1 = pair_area(pa1, pb1);
    for (int m = 0; m < nt - 1; ++m) {
        // smallest union area over the live pairs, ties to the lower pair index: one min
        // reduction over (area bits with the low 6 replaced by the pair index)
        const bool live0 = (active >> pa0) & (active >> pb0) & 1u;
        const bool live1 = lane + 32 < 36 && ((active >> pa1) & (active >> pb1) & 1u);
        const unsigned k0 = live0 ? ((__float_as_uint(d0) & ~63u) | (unsigned)lane) : 0xFFFFFFFFu;
        const unsigned k1 = live1 ? ((__float_as_uint(d1) & ~63u) | (unsigned)(lane + 32)) : 0xFFFFFFFFu;
        const unsigned low = __reduce_min_sync(0xffffffffu, min(k0, k1));
        const int pidx = (int)(low & 63u);
        const int pa = c_pair_a[pidx], pb = c_pair_b[pidx];
        const float bd = __shfl_sync(0xffffffffu, pidx < 32 ? d0 : d1, pidx & 31);
        float ub[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float va = __shfl_sync(0xffffffffu, bx[c], pa), vb = __shfl_sync(0xffffffffu, bx[c], pb);
            ub[c] = c < 3 ? fminf(va, vb) : fmaxf(va, vb);
        }
        const int ra = __shfl_sync(0xffffffffu, cref, pa), rb = __shfl_sync(0xffffffffu, cref, pb);
        const int cs = __shfl_sync(0xffffffffu, ccnt, pa) + __shfl_sync(0xffffffffu, ccnt, pb);
        if (lane == m) {
            mlft = ra;
            mrgt = rb;
            mcnt = cs;
#pragma unroll
            for (int c = 0; c < 6; ++c) mbox[c] = ub[c];
        }
        if (lane == pa) {
#pragma unroll
            for (int c = 0; c < 6; ++c) bx[c] = ub[c];
            cref = kMerged | m;
            ccnt = cs;
        }
        active &= ~(1u << pb);
        if (m != nt - 2) cost_new += bd;
        // the pairs with cluster pa: union of its new box (ub, on every lane) and the partner's
        if (m + 1 < nt - 1) {
            const int q0 = pa0 == pa ? pb0 : pa0, q1 = pa1 == pa ? pb1 : pa1;
            float lo0[3], hi0[3], lo1[3], hi1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lo0[c] = fminf(ub[c], __shfl_sync(0xffffffffu, bx[c], q0));
                hi0[c] = fmaxf(ub[3 + c], __shfl_sync(0xffffffffu, bx[3 + c], q0));
                lo1[c] = fminf(ub[c], __shfl_sync(0xffffffffu, bx[c], q1));
                hi1[c] = fmaxf(ub[3 + c], __shfl_sync(0xffffffffu, bx[3 + c], q1));
            }
            if (pa0 == pa || pb0 == pa) {
                const float dx = hi0[0] - lo0[0], dy = hi0[1] - lo0[1], dz = hi0[2] - lo0[2];
                d0 = dx * dy + dy * dz + dz * dx;
            }
            if (pa1 == pa || pb1 == pa) {
                const float dx = hi1[0] - lo1[0], dy = hi1[1] - lo1[1], dz = hi1[2] - lo1[2];
                d1 = dx * dy + dy * dz + dz * dx;
            }
        }
    }
    if (!(cost_new < cost_old * 0.9999f)) return;
    // lane m < nt - 1 writes merge m's node
    const bool writer = lane < nt - 1;
    const int my_slot = !writer ? 0 : (lane == nt - 2 ? 0 : lane + 1);
    const int my_node = __shfl_sync(0xffffffffu, inner, my_slot);
    float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)my_node);
    const int ch[2] = {mlft, mrgt};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const bool merged = (ch[c] & kMerged) != 0;
        const int src = writer ? (merged ? ch[c] & ~kMerged : ch[c]) : 0;
        const int node_of_merge = __shfl_sync(0xffffffffu, my_node, src);
        const int leaf_ref = __shfl_sync(0xffffffffu, ref, src);
        float b6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float vm = __shfl_sync(0xffffffffu, mbox[k], src);
            const float vl = __shfl_sync(0xffffffffu, ob[k], src);
            b6[k] = merged ? vm : vl;
        }
        const int cr = merged ? node_of_merge : leaf_ref;
        if (writer) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[6 * c + k] = b6[k];
            f[12 + c] = __int_as_float(cr);
            parent[cr < 0 ? ~cr : n + cr] = (my_node << 1) | c;
        }
    }
    if (writer) {
        f[14] = __int_as_float(0);
        f[15] = __int_as_float(mcnt - 1);
#pragma unroll
        for (int k = 0; k < 6; ++k) bin_box[6 * (size_t)my_node + k] = mbox[k];
    }
}

// One pass: every thread climbs from its surfel; the second arrival at a node owns that
// node's treelet, and the owners of a warp have their treelets processed one after another
// by the whole warp.  __syncwarp orders the warp's writes before the owners' next release.
__global__ void __launch_bounds__(kThreads) k_restructure(const float* __restrict__ leaf_box, int* __restrict__ parent,
                                                          int n, float4* __restrict__ nodes, int* __restrict__ flags,
                                                          int* status, float* __restrict__ bin_box) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool walking = j < n;
    int p = walking ? __ldcg(parent + j) : -1;
    int level = 0;
    while (true) {
        int R = -1;
        if (walking) {
            if (p < 0) {
                walking = false;
            } else if (++level > 256 || (p >> 1) >= n - 1) {
                atomicOr(status, GRT_STATUS_BAD_TREE);
                walking = false;
            } else if (atomic_add_acq_rel(flags + (p >> 1), 1) == 0) {
                walking = false;  // first arrival: the sibling's thread goes on
            } else {
                // a node over two surfels has one topology: no treelet to process
                const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)(p >> 1));
                if (__float_as_int(__ldcg(f + 12)) < 0 && __float_as_int(__ldcg(f + 13)) < 0)
                    p = __ldcg(parent + n + (p >> 1));
                else
                    R = p >> 1;
            }
        }
        __syncwarp();
        unsigned todo = __ballot_sync(0xffffffffu, R >= 0);
        while (todo) {
            const int L = __ffs(todo) - 1;
            todo &= todo - 1;
            restructure_treelet(__shfl_sync(0xffffffffu, R, L), leaf_box, parent, n, nodes, bin_box, status);
            __syncwarp();
        }
        if (R >= 0) p = __ldcg(parent + n + R);
        if (!__any_sync(0xffffffffu, walking)) break;
    }
}

// ---------------------------------------------------------------- 4-wide collapse
__device__ __forceinline__ int bin_size(const float4* bn, int ref) {
    if (ref < 0) return 1;
    const float* f = reinterpret_cast<const float*>(bn + 4 * (size_t)ref);
    return __float_as_int(f[15]) - __float_as_int(f[14]) + 1;
}
__device__ __forceinline__ const float* bin_box_of(const float* bin_box, const float* leaf_box, int ref) {
    return ref < 0 ? leaf_box + 6 * (size_t)(~ref) : bin_box + 6 * (size_t)ref;
}

__device__ __forceinline__ void write_slot(float4* W, int s, const float* box, int ref, int bref) {
    float* f = reinterpret_cast<float*>(W);
#pragma unroll
    for (int k = 0; k < 6; ++k) f[4 * k + s] = box[k];
    f[24 + s] = __int_as_float(ref);
    f[28 + s] = __int_as_float(bref);
}

// The 4-wide tree keeps the binary tree's numbering: the wide node made from binary node b
// is wide node b, so that every binary node's wide node is built at once, in parallel,
// with no allocation.  Its children: start with b's two children and twice replace the
// candidate of largest surface area that is too big for a leaf by its two children;
// candidates of at most kLeafMax surfels become leaves over their contiguous run of sorted
// records, larger ones the wide node of the same index.  Only the nodes reachable from
// the root (wide node 0 = binary node 0) are ever traversed; the others are built too,
// since whether a binary node heads a wide node depends on its ancestors' choices.
// SAH-optimal choice of the 4-wide nodes' children (after the dynamic programme of Ylitie,
// Karras and Laine 2017 for wide BVHs, with wide node b kept at binary node b).  F(x, j) is the
// least expected cost of covering binary subtree x with at most j child slots of a wide node:
// x itself as one slot costs W(x) = A(x) C_node + F*(x), where F*(x) = min over j1 + j2 = 4 of
// F(l, j1) + F(r, j2) is x's own wide node opening it into up to four slots; a surfel leaf as a
// slot costs A(leaf) C_test; and F(x, j >= 2) = min(W(x), min over j1 + j2 = j of F(l, j1) +
// F(r, j2)).  A (the half surface area) is the probability of a ray entering the box.  The
// costs fill bottom-up with the refit's arrival counters; the collapse then takes wide node
// b's slots from b's optimal split instead of opening its largest children greedily.
#ifndef GRT_DP_COLLAPSE
#define GRT_DP_COLLAPSE 1
#endif
#ifndef GRT_DP_CNODE
#define GRT_DP_CNODE 1.0f
#endif
#ifndef GRT_DP_CTEST
#define GRT_DP_CTEST 1.0f
#endif
constexpr float kDpNode = GRT_DP_CNODE, kDpTest = GRT_DP_CTEST;

// F(y, 1), F(y, 2), F(y, 3) of a child ref: a surfel leaf costs its test in any number of slots
__device__ __forceinline__ void dp_child(int ref, const float* leaf_box, const float4* dpc, float F[3]) {
    if (ref < 0) {
        const float a = kDpTest * half_area(leaf_box + 6 * (size_t)(~ref));
        F[0] = F[1] = F[2] = a;
    } else {
        const float* c = reinterpret_cast<const float*>(dpc + ref);
        F[0] = __ldcg(c);
        F[1] = __ldcg(c + 1);
        F[2] = __ldcg(c + 2);
    }
}

// Decisions of node x, packed: bits 0-1 the split of F(x, 2), 2-3 of F(x, 3), 4-5 of
// F(x, 4) (0: x itself, else the left child's slot count j1), 6-7 the split of F*(x).
__global__ void k_collapse_cost(const float4* __restrict__ bnodes, const float* __restrict__ bin_box,
                                const float* __restrict__ leaf_box, const int* __restrict__ parent, int n,
                                int* __restrict__ flags, float4* __restrict__ dpc, unsigned* __restrict__ dpd,
                                int* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int p = parent[j];
    for (int level = 0; p >= 0; ++level) {
        if (level > 255 || (p >> 1) >= n - 1) {
            atomicOr(status, GRT_STATUS_BAD_TREE);
            return;
        }
        const int node = p >> 1;
        const int up = parent[n + node];
        // release: this child's costs are visible to the sibling's thread once it sees the
        // count; acquire: the sibling's costs are visible here once this thread sees it
        if (atomic_add_acq_rel(flags + node, 1) == 0) return;
        const float* f = reinterpret_cast<const float*>(bnodes + 4 * (size_t)node);
        const int l = __float_as_int(__ldcg(f + 12)), r = __float_as_int(__ldcg(f + 13));
        float L[3], Rr[3];
        dp_child(l, leaf_box, dpc, L);
        dp_child(r, leaf_box, dpc, Rr);
        // F*: four slots inside x's own wide node
        float fs = L[0] + Rr[2];
        unsigned ss = 1;
        if (L[1] + Rr[1] < fs) { fs = L[1] + Rr[1]; ss = 2; }
        if (L[2] + Rr[0] < fs) { fs = L[2] + Rr[0]; ss = 3; }
        const float W = kDpNode * half_area(bin_box + 6 * (size_t)node) + fs;
        // F(x, 2), F(x, 3), F(x, 4): x itself, or x opened into j1 + j2 slots
        float f2 = W, f3 = W, f4 = W;
        unsigned d2 = 0, d3 = 0, d4 = 0;
        if (L[0] + Rr[0] < f2) { f2 = L[0] + Rr[0]; d2 = 1; }
        if (L[0] + Rr[1] < f3) { f3 = L[0] + Rr[1]; d3 = 1; }
        if (L[1] + Rr[0] < f3) { f3 = L[1] + Rr[0]; d3 = 2; }
        if (fs < f4) { f4 = fs; d4 = ss; }
        __stcg(reinterpret_cast<float4*>(dpc + node), make_float4(W, f2, f3, f4));
        __stcg(dpd + node, d2 | (d3 << 2) | (d4 << 4) | (ss << 6));
        p = up;
    }
}

__global__ void k_collapse(const float4* __restrict__ bnodes, const float* __restrict__ bin_box,
                           const float* __restrict__ leaf_box, int n_int, float4* __restrict__ wnodes,
                           int* status, const unsigned* __restrict__ dpd) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_int) return;
    const float* fb = reinterpret_cast<const float*>(bnodes + 4 * (size_t)b);
    const int n = n_int + 1;
    auto bad = [n](int ref) { return ref >= 0 ? ref >= n - 1 : ~ref >= n; };
    int cand[kWide];
    int nc = 2;
    cand[0] = __float_as_int(fb[12]);
    cand[1] = __float_as_int(fb[13]);
    if (bad(cand[0]) || bad(cand[1])) {
        atomicOr(status, GRT_STATUS_BAD_TREE);
        nc = 0;
    }
#if GRT_DP_COLLAPSE
    if (kLeafMax == 1 && dpd && nc == 2) {
        // the optimal split of F*(b), each part expanded by its own decisions
        int st_ref[kWide], st_j[kWide], ns = 0;
        const unsigned sb = (dpd[b] >> 6) & 3u;
        st_ref[ns] = cand[1]; st_j[ns++] = kWide - (int)sb;
        st_ref[ns] = cand[0]; st_j[ns++] = (int)sb;
        nc = 0;
        while (ns > 0 && nc < kWide) {
            --ns;
            const int y = st_ref[ns], jy = st_j[ns];
            const unsigned d = (y < 0 || jy <= 1) ? 0u : (dpd[y] >> (2 * (jy - 2))) & 3u;
            if (d == 0u || jy - (int)d < 1) {
                cand[nc++] = y;
                continue;
            }
            const float* fy = reinterpret_cast<const float*>(bnodes + 4 * (size_t)y);
            const int yl = __float_as_int(fy[12]), yr = __float_as_int(fy[13]);
            if (bad(yl) || bad(yr) || ns + 2 > kWide) {
                atomicOr(status, GRT_STATUS_BAD_TREE);
                cand[nc++] = y;
                continue;
            }
            st_ref[ns] = yr; st_j[ns++] = jy - (int)d;
            st_ref[ns] = yl; st_j[ns++] = (int)d;
        }
    } else
#endif
    for (int rep = 2; rep < kWide && nc > 0; ++rep) {
        int best = -1;
        float ba = -1.f;
        for (int s = 0; s < nc; ++s) {
            int r = cand[s];
            if (r >= 0 && bin_size(bnodes, r) > kLeafMax) {
                float a = half_area(bin_box + 6 * (size_t)r);
                if (a > ba) {
                    ba = a;
                    best = s;
                }
            }
        }
        if (best < 0) break;
        const float* fr = reinterpret_cast<const float*>(bnodes + 4 * (size_t)cand[best]);
        const int cl = __float_as_int(fr[12]), cr = __float_as_int(fr[13]);
        if (bad(cl) || bad(cr)) {
            atomicOr(status, GRT_STATUS_BAD_TREE);
            break;
        }
        cand[best] = cl;
        cand[nc++] = cr;
    }
    float f[32];  // the node as written: six planes x four slots, refs, binary refs
#pragma unroll
    for (int s = 0; s < kWide; ++s) {
        if (s >= nc) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[4 * k + s] = 1e38f;
                f[4 * (3 + k) + s] = -1e38f;
            }
            f[24 + s] = __int_as_float(kRefEmpty);
            f[28 + s] = __int_as_float(kRefEmpty);
            continue;
        }
        const int r = cand[s];
        int ref;
        if (r < 0) {
            ref = leaf_ref(~r, 1);
        } else {
            const float* fr = reinterpret_cast<const float*>(bnodes + 4 * (size_t)r);
            const int first = __float_as_int(fr[14]), size = __float_as_int(fr[15]) - first + 1;
            ref = size <= kLeafMax ? leaf_ref(first, size) : r;
        }
        const float2* box = reinterpret_cast<const float2*>(bin_box_of(bin_box, leaf_box, r));
        const float2 b01 = box[0], b23 = box[1], b45 = box[2];
        f[s] = b01.x;
        f[4 + s] = b01.y;
        f[8 + s] = b23.x;
        f[12 + s] = b23.y;
        f[16 + s] = b45.x;
        f[20 + s] = b45.y;
        f[24 + s] = __int_as_float(ref);
        f[28 + s] = __int_as_float(r);
    }
    float4* W = wnodes + 8 * (size_t)b;
#pragma unroll
    for (int k = 0; k < 8; ++k) W[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// Child boxes of every wide node from the refit binary boxes (topology unchanged).
__global__ void k_wide_refit(float4* __restrict__ wnodes, int n_int, const float* __restrict__ bin_box,
                             const float* __restrict__ leaf_box) {
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < n_int; w += gridDim.x * blockDim.x) {
        float4* W = wnodes + 8 * (size_t)w;
        const float* f = reinterpret_cast<const float*>(W);
        for (int s = 0; s < kWide; ++s) {
            int br = __float_as_int(f[28 + s]);
            if (br == kRefEmpty) continue;
            write_slot(W, s, bin_box_of(bin_box, leaf_box, br), __float_as_int(f[24 + s]), br);
        }
    }
}

}  // namespace

// Per-primitive steps of a build: leaf boxes and centres, and the packed records.
static void launch_prep(const SurfelIn& in, float* centre, unsigned int* bounds_u, int g, cudaStream_t st) {
    k_prep_bounds<<<g, kThreads, 0, st>>>(in, centre, bounds_u);
}
static void launch_prep(const TriIn& in, float* centre, unsigned int* bounds_u, int g, cudaStream_t st) {
    k_tri_prep<<<g, kThreads, 0, st>>>(in, centre, bounds_u);
}
static void launch_records(const SurfelIn& in, grt_bvh* b, int g, cudaStream_t st) {
    RecordIn r{in, b->sorted_ids, b->records, b->normals, b->leaf_box};
    k_records<<<g, kThreads, 0, st>>>(r);
}
static void launch_records(const TriIn& in, grt_bvh* b, int g, cudaStream_t st) {
    k_tri_records<<<g, kThreads, 0, st>>>(in, b->sorted_ids, b->records, b->leaf_box);
}

// Records, binary refit and the 4-wide collapse (or its refit): shared tail of the builds.
// `passes` treelet-restructuring passes run between the refit and the collapse (topology
// builds only).
template <class In>
static int finish_build(grt_bvh* b, const In& in, bool collapse, int passes, cudaStream_t st) {
    const int n = b->n;
    const int g = (n + kThreads - 1) / kThreads;
    launch_records(in, b, g, st);
    if (n > 1) {
        GRT_CUDA(cudaMemsetAsync(b->refit_flags, 0, sizeof(int) * (size_t)b->n_int, st));
        k_refit<<<g, kThreads, 0, st>>>(b->leaf_box, b->parent, n, b->nodes, b->refit_flags, b->status, b->bin_box);
        const int cg = (b->n_int + 127) / 128;
        if (collapse && kLeafMax == 1) {
            for (int pass = 0; pass < passes && n > 2; ++pass) {
                GRT_CUDA(cudaMemsetAsync(b->refit_flags, 0, sizeof(int) * (size_t)b->n_int, st));
                k_restructure<<<g, kThreads, 0, st>>>(b->leaf_box, b->parent, n, b->nodes, b->refit_flags, b->status,
                                                      b->bin_box);
            }
        }
        const unsigned* dpd = nullptr;
#if GRT_DP_COLLAPSE
        if (collapse && kLeafMax == 1) {
            GRT_CUDA(cudaMemsetAsync(b->refit_flags, 0, sizeof(int) * (size_t)b->n_int, st));
            k_collapse_cost<<<g, kThreads, 0, st>>>(b->nodes, b->bin_box, b->leaf_box, b->parent, n, b->refit_flags,
                                                    b->dp_cost, b->dp_dec, b->status);
            dpd = b->dp_dec;
        }
#endif
        if (collapse)
            k_collapse<<<cg, 128, 0, st>>>(b->nodes, b->bin_box, b->leaf_box, b->n_int, b->wnodes, b->status, dpd);
        else
            k_wide_refit<<<std::min(cg, 1184), 128, 0, st>>>(b->wnodes, b->n_int, b->bin_box, b->leaf_box);
    }
    GRT_CUDA(cudaGetLastError());
    return GRT_OK;
}

// Device scratch of one topology build: centres, bounds, keys x2, ids x2, histograms.
static constexpr size_t build_scratch_bytes(size_t n) {
    const size_t nblocks = (n + kSortTile - 1) / kSortTile;
    return sizeof(float) * 3 * n + 256 + 64 + 2 * sizeof(MortonKey) * n + 2 * sizeof(int) * n +
           sizeof(unsigned int) * 256 * nblocks + 256;
}

// Prep, Morton codes, radix sort and radix tree into b, using `scratch` (build_scratch_bytes).
template <class In>
static int build_topology(grt_bvh* b, const In& in, char* scratch, cudaStream_t st) {
    const int n = b->n;
    const int g = (n + kThreads - 1) / kThreads;
    const int nblocks = (n + kSortTile - 1) / kSortTile;
    char* p = scratch;
    float* centre = (float*)p; p += sizeof(float) * 3 * (size_t)n;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    unsigned int* bounds_u = (unsigned int*)p; p += 64;
    MortonKey* keys0 = (MortonKey*)p; p += sizeof(MortonKey) * (size_t)n;
    MortonKey* keys1 = (MortonKey*)p; p += sizeof(MortonKey) * (size_t)n;
    int* vals0 = (int*)p; p += sizeof(int) * (size_t)n;
    int* vals1 = (int*)p; p += sizeof(int) * (size_t)n;
    unsigned int* hist = (unsigned int*)p;
    // the bounds restart from "empty"; centres, keys, ids and histograms are fully rewritten
    GRT_CUDA(cudaMemsetAsync(bounds_u, 0xFF, 64, st));
    launch_prep(in, centre, bounds_u, g, st);
    k_morton<<<g, kThreads, 0, st>>>(centre, bounds_u, n, keys0, vals0, b->bounds);
    MortonKey* kin = keys0;
    MortonKey* kout = keys1;
    int* vin = vals0;
    int* vout = vals1;
    for (int shift = 0; shift < 32; shift += 8) {
        k_sort_hist<<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, nblocks, hist);
        k_sort_scan<<<1, kScanThreads, 0, st>>>(hist, 256 * nblocks);
        k_sort_scatter<<<nblocks, kSortThreads, 0, st>>>(kin, vin, n, shift, nblocks, hist, kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    GRT_CUDA(cudaMemcpyAsync(b->sorted_ids, vin, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (n > 1) {
        int gi = (n - 1 + kThreads - 1) / kThreads;
        k_hierarchy<<<gi, kThreads, 0, st>>>(kin, n, b->nodes, b->parent);
    }
    GRT_CUDA(cudaGetLastError());
    return GRT_OK;
}

static int launch_build(grt_bvh* b, const grt_surfels* s, float alpha_min, bool rebuild_topology, int passes,
                        cudaStream_t st) {
    const int n = b->n;
    if (n == 0) return GRT_OK;
    SurfelIn in{s->mu, s->quat, s->scale, s->opacity, n, alpha_min};
    if (rebuild_topology) {
        char* scratch = nullptr;
        GRT_CUDA(cudaMallocAsync((void**)&scratch, build_scratch_bytes((size_t)n), st));
        int rc = build_topology(b, in, scratch, st);
        cudaFreeAsync(scratch, st);
        if (rc) return rc;
    }
    return finish_build(b, in, rebuild_topology, passes, st);
}

// Parameters a tree build reads: alpha_min (the bounds) and build_passes.
static int check_build_params(const grt_trace_params* p) {
    if (!p) return set_error(GRT_ERR_ARG, "params is NULL");
    if (!(p->alpha_min > 0.f && p->alpha_min < 1.f)) return set_error(GRT_ERR_ARG, "alpha_min must be in (0,1)");
    if (p->build_passes < 0 || p->build_passes > GRT_MAX_BUILD_PASSES)
        return set_error(GRT_ERR_ARG, "build_passes = %d outside [0, %d]", p->build_passes, GRT_MAX_BUILD_PASSES);
    return GRT_OK;
}

// Treelet-restructuring passes of the mesh backend's tree (its build takes no parameters).
constexpr int kMeshBuildPasses = 1;

static int check_surfels(const grt_surfels* s) {
    if (!s) return set_error(GRT_ERR_ARG, "surfels is NULL");
    if (s->n < 0) return set_error(GRT_ERR_ARG, "surfels->n = %d < 0", s->n);
    if (s->n > (1 << 27)) return set_error(GRT_ERR_ARG, "surfels->n = %d exceeds 2^27", s->n);
    if (s->n > 0 && (!s->mu || !s->quat || !s->scale || !s->opacity))
        return set_error(GRT_ERR_ARG, "surfels: mu/quat/scale/opacity must be non-NULL");
    return GRT_OK;
}

// ---------------------------------------------------------------- allocation-free rebuild
// Scratch of grt_rebuild_bvh_noalloc, compiled into the library: every device that loads
// libgrt holds these bytes until the process exits.  Layout as in launch_build, sized for
// GRT_NOALLOC_MAX_SURFELS surfels.
constexpr size_t kNoallocBlocks = (GRT_NOALLOC_MAX_SURFELS + kSortTile - 1) / kSortTile;
constexpr size_t kNoallocBytes = 4ull * 3 * GRT_NOALLOC_MAX_SURFELS + 256 + 64 +   // centres, bounds
                                 4ull * 2 * GRT_NOALLOC_MAX_SURFELS +              // keys x2
                                 4ull * 2 * GRT_NOALLOC_MAX_SURFELS +              // ids x2
                                 4ull * 256 * kNoallocBlocks + 256;                // digit histograms
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch per device, looked up on the first call made on
// that device (with that device current).  In host code the symbol itself is only a
// host-side stand-in and must never be passed to a kernel.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices] = {};

static int noalloc_scratch(void** out) {
    int dev = 0;
    GRT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(GRT_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GRT_OK;
}

static int launch_build_noalloc(grt_bvh* b, const grt_surfels* s, float alpha_min, int passes, cudaStream_t st) {
    const int n = b->n;
    if (n == 0) return GRT_OK;
    static_assert(kNoallocBytes >= build_scratch_bytes(GRT_NOALLOC_MAX_SURFELS), "fixed scratch too small");
    char* scratch = nullptr;
    int rc = noalloc_scratch((void**)&scratch);
    if (rc) return rc;
    SurfelIn in{s->mu, s->quat, s->scale, s->opacity, n, alpha_min};
    rc = build_topology(b, in, scratch, st);
    if (rc) return rc;
    return finish_build(b, in, true, passes, st);
}

}  // namespace grt

using namespace grt;

extern "C" int grt_rebuild_bvh_noalloc(grt_bvh* b, const grt_surfels* s, const grt_trace_params* params,
                                       void* stream) {
    if (!b) return set_error(GRT_ERR_ARG, "bvh is NULL");
    int rc = check_surfels(s);
    if (rc) return rc;
    rc = check_build_params(params);
    if (rc) return rc;
    if (s->n != b->n) return set_error(GRT_ERR_ARG, "rebuild with n=%d but the BVH holds %d surfels", s->n, b->n);
    if (s->n > GRT_NOALLOC_MAX_SURFELS)
        return set_error(GRT_ERR_ARG, "grt_rebuild_bvh_noalloc: n = %d exceeds its fixed scratch for %d surfels",
                         s->n, GRT_NOALLOC_MAX_SURFELS);
    // the scratch is looked up for the current device: it must be the BVH's own
    int dev = 0;
    GRT_CUDA(cudaGetDevice(&dev));
    if (dev != b->device)
        return set_error(GRT_ERR_ARG, "grt_rebuild_bvh_noalloc: device %d is current, the BVH lives on device %d", dev,
                         b->device);
    return launch_build_noalloc(b, s, params->alpha_min, params->build_passes, (cudaStream_t)stream);
}

// Device storage of a tree over n leaves (one allocation); NULL on failure.
static grt_bvh* alloc_bvh(int nleaf, cudaStream_t st, int* rc_out) {
    grt_bvh* b = new grt_bvh();
    b->n = nleaf;
    b->n_int = nleaf > 1 ? nleaf - 1 : 0;
    cudaGetDevice(&b->device);
    size_t n = (size_t)nleaf, ni = (size_t)b->n_int;
    size_t bytes = sizeof(float4) * 4 * (ni + n) + sizeof(float4) * n + sizeof(int) * (n + ni + 1) + sizeof(int) * (ni + 1) +
                   sizeof(float) * 6 * n + sizeof(int) * n + 64 + 64 +
                   sizeof(float) * 6 * ni + sizeof(float4) * 8 * ni + sizeof(float4) * ni + sizeof(unsigned) * ni +
                   256 * 5;
    char* base = nullptr;
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) {
        delete b;
        *rc_out = set_error(GRT_ERR_OOM, "cudaMalloc(%zu) for the BVH failed: %s", bytes, cudaGetErrorString(e));
        return nullptr;
    }
    char* p = base;
    b->base = base;
    b->nodes = (float4*)p; p += sizeof(float4) * 4 * ni;
    b->records = (float4*)p; p += sizeof(float4) * 4 * n;
    b->normals = (float4*)p; p += sizeof(float4) * n;
    b->leaf_box = (float*)p; p += sizeof(float) * 6 * n;
    b->parent = (int*)p; p += sizeof(int) * (n + ni + 1);
    b->refit_flags = (int*)p; p += sizeof(int) * (ni + 1);
    b->sorted_ids = (int*)p; p += sizeof(int) * n;
    p = (char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    b->status = (int*)p; p += 16;
    b->bounds = (float*)p; p += 32;
    p = (char*)(((uintptr_t)p + 127) & ~(uintptr_t)127);
    b->wnodes = (float4*)p; p += sizeof(float4) * 8 * ni;
    b->bin_box = (float*)p; p += sizeof(float) * 6 * ni;
    p = (char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    b->dp_cost = (float4*)p; p += sizeof(float4) * ni;
    b->dp_dec = (unsigned*)p; p += sizeof(unsigned) * ni;
    b->bytes = bytes;
    e = cudaMemsetAsync(b->status, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bounds, 0, 32, st);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete b;
        *rc_out = check_cuda(e, "cudaMemsetAsync");
        return nullptr;
    }
    *rc_out = GRT_OK;
    return b;
}

extern "C" int grt_build_bvh(const grt_surfels* s, const grt_trace_params* params, grt_bvh** out, void* stream) {
    if (!out) return set_error(GRT_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_surfels(s);
    if (rc) return rc;
    rc = check_build_params(params);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    grt_bvh* b = alloc_bvh(s->n, st, &rc);
    if (!b) return rc;
    char* base = (char*)b->base;
    rc = launch_build(b, s, params->alpha_min, true, params->build_passes, st);
    if (rc) {
        cudaStreamSynchronize(st);
        cudaFree(base);
        delete b;
        return rc;
    }
    *out = b;
    return GRT_OK;
}

extern "C" int grt_build_mesh_bvh(const grt_mesh* m, grt_bvh** out, void* stream) {
    if (!out) return set_error(GRT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!m) return set_error(GRT_ERR_ARG, "mesh is NULL");
    if (m->n_triangles < 0 || m->n_triangles > (1 << 27))
        return set_error(GRT_ERR_ARG, "n_triangles = %d outside [0, 2^27]", m->n_triangles);
    if (m->n_triangles > 0 && (m->n_vertices <= 0 || !m->pos || !m->tri))
        return set_error(GRT_ERR_ARG, "a mesh with triangles needs vertices, pos and tri");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = GRT_OK;
    grt_bvh* b = alloc_bvh(m->n_triangles, st, &rc);
    if (!b) return rc;
    if (b->n > 0) {
        TriIn in{m->pos, m->tri, b->n, m->n_vertices, b->status};
        char* scratch = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&scratch, build_scratch_bytes((size_t)b->n), st);
        if (e == cudaSuccess) {
            rc = build_topology(b, in, scratch, st);
            cudaFreeAsync(scratch, st);
            if (!rc) rc = finish_build(b, in, true, kMeshBuildPasses, st);
        } else {
            rc = check_cuda(e, "cudaMallocAsync");
        }
        if (rc) {
            cudaStreamSynchronize(st);
            cudaFree(b->base);
            delete b;
            return rc;
        }
    }
    *out = b;
    return GRT_OK;
}

extern "C" int grt_refit_bvh(grt_bvh* b, const grt_surfels* s, const grt_trace_params* params, void* stream) {
    if (!b) return set_error(GRT_ERR_ARG, "bvh is NULL");
    int rc = check_surfels(s);
    if (rc) return rc;
    rc = check_build_params(params);
    if (rc) return rc;
    if (s->n != b->n) return set_error(GRT_ERR_ARG, "refit with n=%d but the BVH holds %d surfels", s->n, b->n);
    return launch_build(b, s, params->alpha_min, false, 0, (cudaStream_t)stream);
}

extern "C" int grt_rebuild_bvh(grt_bvh* b, const grt_surfels* s, const grt_trace_params* params, void* stream) {
    if (!b) return set_error(GRT_ERR_ARG, "bvh is NULL");
    int rc = check_surfels(s);
    if (rc) return rc;
    rc = check_build_params(params);
    if (rc) return rc;
    if (s->n != b->n) return set_error(GRT_ERR_ARG, "rebuild with n=%d but the BVH holds %d surfels", s->n, b->n);
    return launch_build(b, s, params->alpha_min, true, params->build_passes, (cudaStream_t)stream);
}

extern "C" void grt_bvh_destroy(grt_bvh* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    cudaFree(b->base);
    delete b;
}

extern "C" int grt_bvh_info(const grt_bvh* b, grt_bvh_info_t* info) {
    if (!b || !info) return set_error(GRT_ERR_ARG, "bvh or info is NULL");
    info->n_surfels = b->n;
    info->n_nodes = b->n_int;
    info->device_bytes = b->bytes;
    cudaError_t e = cudaMemcpy(info->bounds, b->bounds, sizeof(float) * 6, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return check_cuda(e, "cudaMemcpy(bounds)");
    return GRT_OK;
}

extern "C" int grt_bvh_status(grt_bvh* b, int32_t* status, void* stream) {
    if (!b || !status) return set_error(GRT_ERR_ARG, "bvh or status is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    GRT_CUDA(cudaMemcpyAsync(status, b->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    GRT_CUDA(cudaMemsetAsync(b->status, 0, sizeof(int), st));
    GRT_CUDA(cudaStreamSynchronize(st));
    return GRT_OK;
}
