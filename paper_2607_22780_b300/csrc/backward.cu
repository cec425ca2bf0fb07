// backward.cu -- grt_trace_backward / grt_shade_backward: adjoint of the Trace operator
// (Eq. 8) and of the MIS estimate (Eq. 13) with respect to the surfels.
//
// Per ray, with adjoints Gc = dL/dc_rt and Go = dL/do_rt, composited hits k = 1..K,
// T_k the transmittance before hit k, T_f after the last one:
//   dL/dc_k     = Gc T_k a_k
//   dL/da_k     = Gc . (T_k c_k - S_k / (1 - a_k)) + Go T_f / (1 - a_k),
//                 S_k = sum_{j>k} T_j a_j c_j = c_rt - sum_{j<=k} T_j a_j c_j
// then a = o G (zero when clamped at alpha_max), G = exp(-(u^2+v^2)/2),
// u = (p - mu).t_u / s_u, v = (p - mu).t_v / s_v, p = o_ray + tau d,
// tau = n.(mu - o_ray)/(n.d), into mu, the quaternion through R(q/|q|), s_u, s_v, o and
// the colour (RGB or SH coefficients, zero where max(0, .) clamps).
//
// Shading rays get their (tau, id, alpha) sequences from a per-ray hit record: the
// caller's forward record (grt_shade_backward_saved) or a transient one that the backward
// traces itself (grt_shade_backward, chunked to bound memory).  Recorded rays are replayed
// by one thread each; rays with more hits than the record holds, and the rays of
// grt_trace_backward, are traversed again in compositing order.
#include <algorithm>

#include "wavefront.cuh"

namespace grt {
namespace {

struct GradPtrs {
    float *mu, *quat, *scale, *opacity, *color;
};

struct AdjointVisitor {
    const float *mu, *quat, *scale, *opacity, *color;
    int cdim;
    f3 o, d;
    float Gc[3], Go, Tf;
    float crt[3];    // total c_rt from the first pass
    float Cacc[3];   // running sum_{j<=k} T_j a_j c_j
    float alpha_max;
    GradPtrs g;

    // one call site in the replay loop and in the walks' in-order compositing loop
#ifndef GRT_ADJ_INLINE
#define GRT_ADJ_INLINE 1
#endif
#if GRT_ADJ_INLINE
    __device__ __forceinline__ void composite(int, int id, float tau, float alpha, float Tb) {
#else
    __device__ __noinline__ void composite(int, int id, float tau, float alpha, float Tb) {
#endif
        // geometry of the hit, loaded first so that its latency overlaps the colour's
        // (vector loads where the caller's arrays are aligned for them: fewer memory
        // instructions per hit for the load/store unit, which throttles this kernel)
        const float op = __ldg(opacity + id);
        const float4 q = (reinterpret_cast<uintptr_t>(quat) & 15) == 0
                             ? __ldg(reinterpret_cast<const float4*>(quat) + id)
                             : make_float4(__ldg(quat + 4 * (size_t)id), __ldg(quat + 4 * (size_t)id + 1),
                                           __ldg(quat + 4 * (size_t)id + 2), __ldg(quat + 4 * (size_t)id + 3));
        const float2 sc = (reinterpret_cast<uintptr_t>(scale) & 7) == 0
                              ? __ldg(reinterpret_cast<const float2*>(scale) + id)
                              : make_float2(__ldg(scale + 2 * (size_t)id), __ldg(scale + 2 * (size_t)id + 1));
        const float su = sc.x, sv = sc.y;
        const f3 m = mk3(__ldg(mu + 3 * (size_t)id), __ldg(mu + 3 * (size_t)id + 1), __ldg(mu + 3 * (size_t)id + 2));
        // colour of the hit and, for SH, which channels are live
        float Y[16];
        float c[3];
        bool live[3] = {true, true, true};
        if (cdim == 3) {
            c[0] = __ldg(color + 3 * (size_t)id);
            c[1] = __ldg(color + 3 * (size_t)id + 1);
            c[2] = __ldg(color + 3 * (size_t)id + 2);
        } else {
            sh_basis(d.x, d.y, d.z, Y);
            const float4* s = reinterpret_cast<const float4*>(color + 48 * (size_t)id);
            float4 sv4[12];
            if ((reinterpret_cast<uintptr_t>(color) & 31) == 0) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const F8 v = ld_v8(s + 2 * q);
                    sv4[2 * q] = v.a;
                    sv4[2 * q + 1] = v.b;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 12; ++q) sv4[q] = __ldg(s + q);
            }
            float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const float4 v = sv4[q];
                float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[(4 * q + t) % 3] = fmaf(e[t], Y[(4 * q + t) / 3], acc[(4 * q + t) % 3]);
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                live[ch] = acc[ch] > 0.f;
                c[ch] = fmaxf(acc[ch], 0.f);
            }
        }
        float w = Tb * alpha;
        float inv1a = 1.f / (1.f - alpha);
        float dLda = Go * Tf * inv1a;
        float dLdc[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            Cacc[ch] = fmaf(w, c[ch], Cacc[ch]);
            float S = crt[ch] - Cacc[ch];
            dLda = fmaf(Gc[ch], fmaf(Tb, c[ch], -S * inv1a), dLda);
            dLdc[ch] = Gc[ch] * w;
        }
        if (g.color) {
            if (cdim == 3) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) atomicAdd(g.color + 3 * (size_t)id + ch, dLdc[ch]);
            } else {
                float4* gs = reinterpret_cast<float4*>(g.color + 48 * (size_t)id);
                float m0 = live[0] ? dLdc[0] : 0.f, m1 = live[1] ? dLdc[1] : 0.f, m2 = live[2] ? dLdc[2] : 0.f;
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    float e[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        int idx = 4 * q + t, ch = idx % 3;
                        e[t] = (ch == 0 ? m0 : (ch == 1 ? m1 : m2)) * Y[idx / 3];
                    }
                    atomicAdd(gs + q, make_float4(e[0], e[1], e[2], e[3]));
                }
            }
        }
        float ql = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        float iql = 1.f / ql;
        float qw = q.x * iql, qx = q.y * iql, qy = q.z * iql, qz = q.w * iql;
        f3 tu = mk3(1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy + qw * qz), 2.f * (qx * qz - qw * qy));
        f3 tv = mk3(2.f * (qx * qy - qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz + qw * qx));
        f3 n = mk3(2.f * (qx * qz + qw * qy), 2.f * (qy * qz - qw * qx), 1.f - 2.f * (qx * qx + qy * qy));
        f3 dp = mk3(fmaf(tau, d.x, o.x) - m.x, fmaf(tau, d.y, o.y) - m.y, fmaf(tau, d.z, o.z) - m.z);
        float u = dot3(dp, tu) / su, v = dot3(dp, tv) / sv;
        float G = __expf(-0.5f * fmaf(u, u, v * v));
        if (op * G > alpha_max) return;  // clamped: alpha does not depend on the geometry
        if (g.opacity) atomicAdd(g.opacity + id, dLda * G);
        float dLdu = -dLda * alpha * u, dLdv = -dLda * alpha * v;
        if (g.scale)
            atomicAdd(reinterpret_cast<float2*>(g.scale + 2 * (size_t)id), make_float2(-dLdu * u / su, -dLdv * v / sv));
        float nd = dot3(n, d), tud = dot3(tu, d), tvd = dot3(tv, d);
        float au = dLdu / su, av = dLdv / sv;
        float kn = (au * tud + av * tvd) / nd;
        if (g.mu) {
            atomicAdd(g.mu + 3 * (size_t)id, kn * n.x - au * tu.x - av * tv.x);
            atomicAdd(g.mu + 3 * (size_t)id + 1, kn * n.y - au * tu.y - av * tv.y);
            atomicAdd(g.mu + 3 * (size_t)id + 2, kn * n.z - au * tu.z - av * tv.z);
        }
        if (g.quat) {
            // dL/dR columns: t_u -> dp au, t_v -> dp av, n -> -dp kn
            float G00 = dp.x * au, G10 = dp.y * au, G20 = dp.z * au;
            float G01 = dp.x * av, G11 = dp.y * av, G21 = dp.z * av;
            float G02 = -dp.x * kn, G12 = -dp.y * kn, G22 = -dp.z * kn;
            float gw = 2.f * (-qz * G01 + qy * G02 + qz * G10 - qx * G12 - qy * G20 + qx * G21);
            float gx = 2.f * (qy * G01 + qz * G02 + qy * G10 - 2.f * qx * G11 - qw * G12 + qz * G20 + qw * G21 -
                              2.f * qx * G22);
            float gy = 2.f * (-2.f * qy * G00 + qx * G01 + qw * G02 + qx * G10 + qz * G12 - qw * G20 + qz * G21 -
                              2.f * qy * G22);
            float gz = 2.f * (-2.f * qz * G00 - qw * G01 + qx * G02 + qw * G10 - 2.f * qz * G11 + qy * G12 + qx * G20 +
                              qy * G21);
            float qd = qw * gw + qx * gx + qy * gy + qz * gz;
            atomicAdd(reinterpret_cast<float4*>(g.quat + 4 * (size_t)id),
                      make_float4((gw - qw * qd) * iql, (gx - qx * qd) * iql, (gy - qy * qd) * iql, (gz - qz * qd) * iql));
        }
    }
    __device__ __forceinline__ void finish(float) {}
};

template <int K>
__device__ __forceinline__ void ray_adjoint(const DevBvh& bvh, const TraceParams& P, const grt_surfels& s, f3 o, f3 d,
                                            const float Gc[3], float Go, const GradPtrs& g) {
    if (Gc[0] == 0.f && Gc[1] == 0.f && Gc[2] == 0.f && Go == 0.f) return;
    RayState r = make_ray(o, d);
    Counters cnt{0, 0, 0};
    ColourVisitor fwd(s.color, s.color_dim, d, nullptr, 0);
    trace_ray<K, false>(bvh, r, P, fwd, cnt);
    if (fwd.nh == 0) return;
    AdjointVisitor adj;
    adj.mu = s.mu;
    adj.quat = s.quat;
    adj.scale = s.scale;
    adj.opacity = s.opacity;
    adj.color = s.color;
    adj.cdim = s.color_dim;
    adj.o = o;
    adj.d = d;
    adj.Go = Go;
    adj.Tf = fwd.T;
    adj.alpha_max = P.alpha_max;
    adj.g = g;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        adj.Gc[c] = Gc[c];
        adj.crt[c] = fwd.c[c];
        adj.Cacc[c] = 0.f;
    }
    trace_ray<K, false>(bvh, r, P, adj, cnt);
}

template <int K>
__global__ void __launch_bounds__(128) k_trace_backward(DevBvh bvh, TraceParams P, grt_surfels s,
                                                        const float* __restrict__ ro, const float* __restrict__ rd, int R,
                                                        const float* __restrict__ dc, const float* __restrict__ dop,
                                                        GradPtrs g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    f3 o = mk3(ro[3 * (size_t)i], ro[3 * (size_t)i + 1], ro[3 * (size_t)i + 2]);
    f3 d = mk3(rd[3 * (size_t)i], rd[3 * (size_t)i + 1], rd[3 * (size_t)i + 2]);
    float Gc[3] = {dc[3 * (size_t)i], dc[3 * (size_t)i + 1], dc[3 * (size_t)i + 2]};
    float Go = dop ? dop[i] : 0.f;
    ray_adjoint<K>(bvh, P, s, o, d, Gc, Go, g);
}

// Per-ray adjoint of the shaded outputs (Eq. 13): for a traced sample with weight
// g = f cos / q and environment radiance L,
//   dL/dc_rt = (dL/dcolor * g + dL/dind) / N_r,  dL/do_rt = -(sum_c dL/dcolor_c g_c L_c + dL/dvis) / N_r.
// (0, 0, 0, 0) marks a ray without hits or without a sample.
struct AdjIn {
    const float *dcol, *dvis, *dind;
};

__global__ void __launch_bounds__(kShadeThreads) k_adjoint_weights(const __grid_constant__ JobTable<1> T,
                                                                   const float4* __restrict__ dirs,
                                                                   const float4* __restrict__ res, AdjIn in,
                                                                   float4* __restrict__ adj) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T.total_rays) return;
    float4 rr = __ldg(res + r);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rr.w >= 0.f && !(rr.w == 1.f && rr.x == 0.f && rr.y == 0.f && rr.z == 0.f)) {
        const ShadeJob& J = T.job[0];
        int li = (int)(r / J.Nr);
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        PixelState ps = load_pixel(J.gb, pix);
        float4 dw = __ldg(dirs + r);
        SampleWeight sw = sample_weight(J.S, J.env, ps, mk3(dw.x, dw.y, dw.z));
        const float inv = 1.f / (float)J.Nr;
        float Gc[3], Go = in.dvis ? -__ldg(in.dvis + li) * inv : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float dc = __ldg(in.dcol + 3 * (size_t)li + c) * inv;
            float di = in.dind ? __ldg(in.dind + 3 * (size_t)li + c) * inv : 0.f;
            Gc[c] = fmaf(dc, sw.g[c], di);
            Go = fmaf(-dc * sw.g[c], sw.L[c], Go);
        }
        out = make_float4(Gc[0], Gc[1], Gc[2], Go);
    }
    adj[r] = out;
}

// Adjoint rays: same origin/direction as the forward shading rays, totals (c_rt, T_f)
// from the forward pass, adjoints (dL/dc_rt, dL/do_rt) from k_adjoint_weights; one
// traversal per ray in the persistent two-phase walk.
// Adjoint state of shading ray r: origin from the G-buffer, direction and forward totals
// (c_rt, T_f) from the forward pass, adjoints (dL/dc_rt, dL/do_rt) from k_adjoint_weights.
__device__ __forceinline__ void adjoint_init(AdjointVisitor& av, const ShadeJob& J, const TraceParams& P, GradPtrs g,
                                             float4 a, float4 rr, f3 o, f3 d) {
    av.mu = J.mu;
    av.quat = J.quat;
    av.scale = J.scale;
    av.opacity = J.opacity;
    av.color = J.color;
    av.cdim = J.cdim;
    av.alpha_max = P.alpha_max;
    av.g = g;
    av.o = o;
    av.d = d;
    av.Gc[0] = a.x;
    av.Gc[1] = a.y;
    av.Gc[2] = a.z;
    av.Go = a.w;
    av.Tf = rr.w;
    av.crt[0] = rr.x;
    av.crt[1] = rr.y;
    av.crt[2] = rr.z;
    av.Cacc[0] = av.Cacc[1] = av.Cacc[2] = 0.f;
}

__device__ __forceinline__ f3 ray_origin(const ShadeJob& J, long long r) {
    int li = (int)(r / J.Nr);
    int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
    return mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
               __ldg(J.gb.pos + 3 * (size_t)pix + 2));
}

// Adjoint rays in the persistent two-phase walk: the (tau, id) sequence is recomputed by
// tracing the ray again.  With a hit record, only the rays k_adjoint_replay listed (more
// hits than the record holds) are walked here: their L recorded hits are replayed, and
// the traversal resumes after the last of them.
template <int K>
struct AdjointTask {
    using Visitor = AdjointVisitor;
    const JobTable<1>* T;
    const float4 *dirs, *res, *adj;
    GradPtrs g;
    const long long* list;  // record rows to walk (rays the replay could not take), or NULL: all rays
    const SavedHits* sv;    // with a list: their records, replayed before the walk resumes
    __device__ __forceinline__ bool begin(long long i, WalkState<K>& ts, Visitor& av, const DevBvh*& bvh) {
        const long long row = list ? __ldg(list + i) : i;
        const long long r = (list && sv->order) ? (long long)__ldg(sv->order + row) : row;
        float4 a = __ldg(adj + r);
        if (a.x == 0.f && a.y == 0.f && a.z == 0.f && a.w == 0.f) return false;
        const ShadeJob& J = T->job[0];
        float4 rr = __ldg(res + r), dw = __ldg(dirs + r);
        f3 o = ray_origin(J, r);
        f3 d = mk3(dw.x, dw.y, dw.z);
        bvh = &J.bvh;
        adjoint_init(av, J, T->P, g, a, rr, o, d);
        if (!list) {
            trace_begin(J.bvh, ts, o, d, T->P);
            return true;
        }
        // the recorded first L hits, then the traversal from the last recorded key on
        float Tb = 1.f, tau = 0.f;
        int id = 0;
        for (int k = 0; k < sv->L; ++k) {
            const size_t j = (size_t)k * sv->R + row;
            id = __ldg(sv->ids + j);
            tau = __ldg(sv->tau + j);
            const float alpha = __ldg(sv->alpha + j);
            if ((unsigned)id >= (unsigned)J.bvh.n) {
                atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
                return false;
            }
            av.composite(k, id, tau, alpha, Tb);
            Tb = mul_d(Tb, sub_d(1.0f, alpha));
        }
        trace_resume(J.bvh, ts, o, d, T->P, make_key(tau, id), Tb, sv->L);
        return true;
    }
    __device__ __forceinline__ void end(long long, const WalkState<K>&, Visitor&) {}
};

// Replay of the saved hit records: one thread per ray walks its (id, tau, alpha) list in
// compositing order, rebuilding T_k exactly as the forward compositor did.  The first
// ov_cap threads take the rays that hold an overflow slot (more than L hits), so that the
// longest lists start first and do not trail the launch; the other threads take the record
// rows in order, i.e. the rays in the forward walk's coherent order, so that a warp reads
// neighbouring words of the record and meets the same surfels.  Rays longer than the
// record and its overflow slot, and rays that found no slot free, are listed (by row) for
// the traced adjoint walk.
__device__ __forceinline__ void replay_hit(const SavedHits& sv, long long row, int slot, int k, int* id, float* tau,
                                           float* alpha) {
    if (k < sv.L) {
        const size_t i = (size_t)k * sv.R + row;
        *id = __ldg(sv.ids + i);
        *tau = __ldg(sv.tau + i);
        *alpha = __ldg(sv.alpha + i);
    } else {
        const size_t i = (size_t)(k - sv.L) * sv.ov_cap + slot;
        *id = __ldg(sv.ov_ids + i);
        *tau = __ldg(sv.ov_tau + i);
        *alpha = __ldg(sv.ov_alpha + i);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of a surfel's parameters and gradient lines (the replay's next hit): on a
// scene whose parameters exceed L2 each hit otherwise waits on DRAM for both in turn.
__device__ __forceinline__ void prefetch_surfel(const AdjointVisitor& av, const GradPtrs& g, int id) {
    prefetch_l2(av.mu + 3 * (size_t)id);
    prefetch_l2(av.quat + 4 * (size_t)id);
    prefetch_l2(av.scale + 2 * (size_t)id);
    prefetch_l2(av.opacity + id);
    const float* c = av.color + (size_t)av.cdim * id;
    prefetch_l2(c);
    if (av.cdim == 48) prefetch_l2(c + 47);  // a 192-byte row spans two 128-byte lines
    if (g.mu) prefetch_l2(g.mu + 3 * (size_t)id);
    if (g.quat) prefetch_l2(g.quat + 4 * (size_t)id);
    if (g.scale) prefetch_l2(g.scale + 2 * (size_t)id);
    if (g.opacity) prefetch_l2(g.opacity + id);
    if (g.color) {
        const float* gc = g.color + (size_t)av.cdim * id;
        prefetch_l2(gc);
        if (av.cdim == 48) prefetch_l2(gc + 47);
    }
}

// Scenes from this many surfels on take the replay that prefetches: their parameters and
// gradients (464 bytes per surfel) are several times L2.  Below it the prefetches only cost:
// the 300k-surfel replay is bound by L2 atomics and ran 0.98 -> 1.20 ms with them (96
// registers against 80), while the 2M-surfel 1080p forward + backward ran 193.0 -> 189.5 ms.
constexpr int kReplayPrefetchSurfels = 1 << 20;

template <bool PF>
__global__ void __launch_bounds__(kShadeThreads) k_adjoint_replay(const __grid_constant__ JobTable<1> T,
                                                                  const float4* __restrict__ dirs,
                                                                  const float4* __restrict__ res,
                                                                  const float4* __restrict__ adj,
                                                                  const __grid_constant__ SavedHits sv, GradPtrs g,
                                                                  unsigned long long* __restrict__ over_count,
                                                                  long long* __restrict__ over_list) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long row;  // record row = walk position
    int slot = -1;
    if (t < sv.ov_cap) {
        const unsigned used = *sv.ov_count;
        if (t >= (long long)(used < (unsigned)sv.ov_cap ? used : (unsigned)sv.ov_cap)) return;
        slot = (int)t;
        row = __ldg(sv.ov_ray + slot);
        if ((unsigned long long)row >= (unsigned long long)T.total_rays) {
            atomicOr(T.job[0].bvh.status, GRT_STATUS_BAD_INDEX);
            return;
        }
    } else {
        row = t - sv.ov_cap;
        if (row >= T.total_rays) return;
    }
    const long long r = sv.order ? (long long)__ldg(sv.order + row) : row;  // the ray's slot
    const int raw = __ldg(sv.nh + r);
    const int n = raw & (kNoSlot - 1);
    if (n == 0) return;
    float4 a = __ldg(adj + r);
    if (a.x == 0.f && a.y == 0.f && a.z == 0.f && a.w == 0.f) return;
    if (n > sv.L) {
        if (slot < 0) {  // a long ray: its slot thread takes it, or, without a slot, the walk
            if (raw & kNoSlot) over_list[atomicAdd(over_count, 1ull)] = row;
            return;
        }
        if (n > sv.L + kOverflowHits) {  // longer than record and slot: left to the walk
            over_list[atomicAdd(over_count, 1ull)] = row;
            return;
        }
    }
    const ShadeJob& J = T.job[0];
    float4 rr = __ldg(res + r), dw = __ldg(dirs + r);
    AdjointVisitor av;
    adjoint_init(av, J, T.P, g, a, rr, ray_origin(J, r), mk3(dw.x, dw.y, dw.z));
    const int ns = J.bvh.n;
    float Tb = 1.f;
    if constexpr (PF) {
        // the record two hits ahead is loaded, and the next hit's surfel lines prefetched into
        // L2, while the current hit is composited
        int id, id1 = 0;
        float tau, alpha, tau1 = 0.f, alpha1 = 0.f;
        replay_hit(sv, row, slot, 0, &id, &tau, &alpha);
        if (n > 1) replay_hit(sv, row, slot, 1, &id1, &tau1, &alpha1);
        for (int k = 0; k < n; ++k) {
            int id2 = 0;
            float tau2 = 0.f, alpha2 = 0.f;
            if (k + 2 < n) replay_hit(sv, row, slot, k + 2, &id2, &tau2, &alpha2);
            if (k + 1 < n && (unsigned)id1 < (unsigned)ns) prefetch_surfel(av, g, id1);
            if ((unsigned)id >= (unsigned)ns) {
                atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
                return;
            }
            av.composite(k, id, tau, alpha, Tb);
            Tb = mul_d(Tb, sub_d(1.0f, alpha));
            id = id1;
            tau = tau1;
            alpha = alpha1;
            id1 = id2;
            tau1 = tau2;
            alpha1 = alpha2;
        }
    } else {
        // the next hit's record is loaded while the current one is composited
        int id;
        float tau, alpha;
        replay_hit(sv, row, slot, 0, &id, &tau, &alpha);
        for (int k = 0; k < n; ++k) {
            int idn = 0;
            float taun = 0.f, alphan = 0.f;
            if (k + 1 < n) replay_hit(sv, row, slot, k + 1, &idn, &taun, &alphan);
            if ((unsigned)id >= (unsigned)ns) {
                atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
                return;
            }
            av.composite(k, id, tau, alpha, Tb);
            Tb = mul_d(Tb, sub_d(1.0f, alpha));
            id = idn;
            tau = taun;
            alpha = alphan;
        }
    }
}

template <int K>
__global__ void __launch_bounds__(kShadeThreads, K >= 32 ? 3 : 4) k_adjoint_ww(const __grid_constant__ JobTable<1> T,
                                                                               const float4* __restrict__ dirs,
                                                                               const float4* __restrict__ res,
                                                                               const float4* __restrict__ adj, GradPtrs g,
                                                                               const unsigned long long* __restrict__ n_list,
                                                                               const long long* __restrict__ list,
                                                                               const __grid_constant__ SavedHits sv,
                                                                               unsigned long long* __restrict__ next_ray) {
    __shared__ int q[kQueue * kShadeThreads];
    AdjointTask<K> task{&T, dirs, res, adj, g, list, &sv};
    const long long total = n_list ? (long long)*n_list : T.total_rays;
    persistent_trace<K>(task, T.P, next_ray, total, q + threadIdx.x, kShadeThreads);
}

}  // namespace
}  // namespace grt

using namespace grt;

static int check_grads(const grt_grads* g, const grt_surfels* s) {
    if (!g) return set_error(GRT_ERR_ARG, "grads is NULL");
    if (g->quat && ((uintptr_t)g->quat & 15)) return set_error(GRT_ERR_ARG, "grads->quat must be 16-byte aligned");
    if (g->scale && ((uintptr_t)g->scale & 7)) return set_error(GRT_ERR_ARG, "grads->scale must be 8-byte aligned");
    if (g->color && s->color_dim == 48 && ((uintptr_t)g->color & 15))
        return set_error(GRT_ERR_ARG, "grads->color must be 16-byte aligned for SH");
    if (s->n > 0 && (!s->mu || !s->quat || !s->scale || !s->opacity))
        return set_error(GRT_ERR_ARG, "surfels need mu, quat, scale and opacity for gradients");
    return GRT_OK;
}

extern "C" int grt_trace_backward(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const float* ray_o,
                                  const float* ray_d, int32_t R, const float* dL_drgb, const float* dL_dopacity,
                                  const grt_grads* grads, void* stream) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    rc = check_grads(grads, s);
    if (rc) return rc;
    if (R < 0 || (R > 0 && (!ray_o || !ray_d || !dL_drgb))) return set_error(GRT_ERR_ARG, "bad rays or dL_drgb");
    if (R == 0) return GRT_OK;
    DevBvh bvh = dev_bvh(b);
    TraceParams P = to_params(*p);
    GradPtrs g{grads->mu, grads->quat, grads->scale, grads->opacity, grads->color};
    grt_surfels sc = *s;
    cudaStream_t st = (cudaStream_t)stream;
    int grid = (R + 127) / 128;
    dispatch_k(p->k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        k_trace_backward<K><<<grid, 128, 0, st>>>(bvh, P, sc, ray_o, ray_d, R, dL_drgb, dL_dopacity, g);
    });
    return launch_error("k_trace_backward");
}

// Recomputing adjoint (no forward record): the backward draws the samples again and
// traces them once, keeping a transient hit record that it then replays.  Rays are taken
// in chunks so that the transient record (directions, totals, adjoints, hit count and
// kRecomputeHits hits, overflow list: 828 bytes per ray; two chunks in flight) stays
// within ~14 GB whatever the frame size.  On the 2M-surfel 1080p frame (33M ray slots)
// forward + backward takes 442 ms in 8M-ray chunks, 432 ms unchunked, 512 ms in 2M-ray
// chunks: each chunk's persistent kernels end in a tail of long rays.
// 64 slots hold every hit of all but ~0.2% of the rays of the object and unbounded scenes
// (at most 96 hits seen); the few longer rays are traversed again.
#ifndef GRT_RECOMPUTE_CHUNK_RAYS
#define GRT_RECOMPUTE_CHUNK_RAYS (8ll << 20)
#endif
constexpr long long kRecomputeChunkRays = GRT_RECOMPUTE_CHUNK_RAYS;
constexpr int kRecomputeHits = 64;

// Optional timing (grt_adjoint_timing): events on the call's stream around the three
// kernels of the most recent adjoint pass of this thread.
struct AdjointTiming {
    bool on = false;
    bool have = false;
    bool ok = false;  // every mark of the current pass was recorded
    int device = -1;  // device the events belong to
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // Events are made on the current device and made again when a pass runs on another
    // one; a failed record leaves the pass without timings (`have` stays false).
    void mark(int i, cudaStream_t st) {
        if (!on) return;
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (dev != device) {
            for (auto& e : ev) {
                if (e) cudaEventDestroy(e);  // an event of another device: released, not reused
                e = nullptr;
            }
            device = dev;
        }
        if (i == 0) ok = true;
        if (!ev[i] && cudaEventCreate(&ev[i]) != cudaSuccess) ev[i] = nullptr;
        if (!ev[i] || cudaEventRecord(ev[i], st) != cudaSuccess) ok = false;
    }
};
thread_local AdjointTiming g_adj_timing;

// Adjoint weights, replay of the recorded rays, and a traced adjoint walk for the rays
// the record does not hold (all rays when hits.L == 0).  `work` holds two counters and,
// with a record, room for a list of every ray.
template <int K>
static void run_adjoint(const JobTable<1>& T, const float4* dirs, const float4* res, const SavedHits& hits,
                        float4* adj, unsigned long long* work, const AdjIn& in, const GradPtrs& g, cudaStream_t st) {
    const long long gr = (T.total_rays + kShadeThreads - 1) / kShadeThreads;
    unsigned long long* next_ray = work;
    unsigned long long* n_over = work + 1;
    long long* over = reinterpret_cast<long long*>(work + 2);
    cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), st);
    g_adj_timing.mark(0, st);
    k_adjoint_weights<<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, res, in, adj);
    g_adj_timing.mark(1, st);
    if (hits.L > 0) {
        const long long gp = (T.total_rays + hits.ov_cap + kShadeThreads - 1) / kShadeThreads;
        if (T.job[0].bvh.n >= kReplayPrefetchSurfels)
            k_adjoint_replay<true><<<(unsigned)gp, kShadeThreads, 0, st>>>(T, dirs, res, adj, hits, g, n_over, over);
        else
            k_adjoint_replay<false><<<(unsigned)gp, kShadeThreads, 0, st>>>(T, dirs, res, adj, hits, g, n_over, over);
    }
    g_adj_timing.mark(2, st);
    constexpr size_t smem = walk_smem_bytes<K>();
    const long long grid = persistent_grid(k_adjoint_ww<K>, smem, gr);
    k_adjoint_ww<K><<<(unsigned)grid, kShadeThreads, smem, st>>>(T, dirs, res, adj, g, hits.L > 0 ? n_over : nullptr,
                                                              hits.L > 0 ? over : nullptr, hits, next_ray);
    g_adj_timing.mark(3, st);
    g_adj_timing.have = g_adj_timing.on && g_adj_timing.ok;
}

// Two library streams per host thread and device: consecutive chunks of the recomputing
// adjoint alternate between them, so that one chunk's rays fill the SMs that the long rays
// at the end of the previous chunk leave idle.
struct AuxStreams {
    bool ready = false;
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
};

static int aux_streams(AuxStreams** out) {
    constexpr int kMaxDev = 64;
    static thread_local AuxStreams tab[kMaxDev];
    int dev = 0;
    GRT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return set_error(GRT_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDev);
    AuxStreams& a = tab[dev];
    if (!a.ready) {
        for (int i = 0; i < 2; ++i) {
            GRT_CUDA(cudaStreamCreateWithFlags(&a.s[i], cudaStreamNonBlocking));
            GRT_CUDA(cudaEventCreateWithFlags(&a.join[i], cudaEventDisableTiming));
        }
        GRT_CUDA(cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming));
        a.ready = true;
    }
    *out = &a;
    return GRT_OK;
}

// Device workspace of a shading adjoint over `rays` ray slots (n_pixels x N_r): with a
// forward record, the adjoint per ray and the overflow list; recomputing, one or two chunk
// buffers (directions, totals, transient hit record, adjoints, ray order).
struct BackwardLayout {
    long long chunk_px, n_chunks, Rc;
    SavedLayout lay;
    size_t ord_off, per, total;
    int nbuf;
};

static BackwardLayout backward_layout(long long n_pixels, int Nr, bool saved) {
    BackwardLayout b{};
    const long long rays = n_pixels * Nr;
    if (saved) {
        b.total = (sizeof(float4) + sizeof(long long)) * (size_t)rays + 16;
        return b;
    }
    b.chunk_px = std::min<long long>(n_pixels, std::max<long long>(1, kRecomputeChunkRays / Nr));
    b.n_chunks = (n_pixels + b.chunk_px - 1) / b.chunk_px;
    b.Rc = b.chunk_px * Nr;
    b.lay = saved_layout(b.Rc, kRecomputeHits);
    b.ord_off = (b.lay.total + (sizeof(float4) + sizeof(long long)) * (size_t)b.Rc + 16 + 255) & ~(size_t)255;
    b.per = (b.ord_off + (use_ray_order(b.Rc) ? order_scratch_bytes(b.Rc) : 0) + 255) & ~(size_t)255;
    b.nbuf = b.n_chunks > 1 ? 2 : 1;
    b.total = b.per * b.nbuf;
    return b;
}

// Shading adjoint, from a caller's forward record (save) or recomputing (save == NULL).
static int shade_backward_impl(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                               const grt_gbuffer* gb, const grt_envmap* e, const grt_sampling* smp,
                               const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                               const float* dL_dvis, const float* dL_dind, const grt_grads* grads,
                               const SaveBufs* save, const Workspace& ws, cudaStream_t st) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    rc = check_grads(grads, s);
    if (rc) return rc;
    if (n_pixels < 0 || (n_pixels > 0 && !dL_dcolor)) return set_error(GRT_ERR_ARG, "bad n_pixels or dL_dcolor");
    JobTable<1> T;
    T.P = to_params(*p);
    T.n_jobs = 1;
    rc = make_job(b, s, gb, e, smp, pixel_list, n_pixels, nullptr, nullptr, nullptr, &T.job[0]);
    if (rc) return rc;
    const ShadeJob& J = T.job[0];
    if (J.n_pixels == 0) return GRT_OK;
    const long long rays = (long long)J.n_pixels * J.Nr;
    T.total_rays = rays;
    T.total_units = 0;
    GradPtrs g{grads->mu, grads->quat, grads->scale, grads->opacity, grads->color};
    const BackwardLayout BL = backward_layout(J.n_pixels, J.Nr, save != nullptr);
    char* mem = nullptr;  // pool memory of this call (no caller workspace)
    char* buf = nullptr;
    if (ws.ptr) {
        if (ws.bytes < BL.total) return set_error(GRT_ERR_ARG, "workspace holds %zu bytes, %zu needed", ws.bytes, BL.total);
        buf = static_cast<char*>(ws.ptr);
    } else {
        keep_pool_memory();
        GRT_CUDA(cudaMallocAsync((void**)&mem, BL.total, st));
        buf = mem;
    }
    if (save) {
        float4* adj = reinterpret_cast<float4*>(buf);
        unsigned long long* work = reinterpret_cast<unsigned long long*>(adj + rays);
        dispatch_k(p->k, [&](auto kc) {
            run_adjoint<decltype(kc)::value>(T, save->dirs, save->res, save->hits, adj, work,
                                             AdjIn{dL_dcolor, dL_dvis, dL_dind}, g, st);
        });
    } else {
        const long long chunk_px = BL.chunk_px, n_chunks = BL.n_chunks, Rc = BL.Rc;
        const SavedLayout lay = BL.lay;
        const size_t ord_off = BL.ord_off, per = BL.per;
        AuxStreams* aux = nullptr;
        if (BL.nbuf > 1) {
            rc = aux_streams(&aux);
            if (rc) {
                if (mem) cudaFreeAsync(mem, st);
                return rc;
            }
        }
        if (aux) {
            GRT_CUDA(cudaEventRecord(aux->fork, st));
            for (int i = 0; i < 2; ++i) GRT_CUDA(cudaStreamWaitEvent(aux->s[i], aux->fork, 0));
        }
        for (long long c = 0; c < n_chunks; ++c) {
            const long long p0 = c * chunk_px;
            cudaStream_t cs = aux ? aux->s[c & 1] : st;
            char* cb = buf + per * (size_t)(c & 1);
            float4* dirs = reinterpret_cast<float4*>(cb + lay.dirs);
            float4* res = reinterpret_cast<float4*>(cb + lay.res);
            unsigned long long* next_ray = reinterpret_cast<unsigned long long*>(cb + lay.next);
            float4* adj = reinterpret_cast<float4*>(cb + lay.total);
            unsigned long long* work = reinterpret_cast<unsigned long long*>(adj + Rc);
            JobTable<1> Tc = T;
            ShadeJob& Jc = Tc.job[0];
            Jc.n_pixels = (int)std::min<long long>(chunk_px, J.n_pixels - p0);
            if (Jc.pixel_list)
                Jc.pixel_list += p0;
            else
                Jc.pixel_offset += (int)p0;
            Tc.total_rays = (long long)Jc.n_pixels * Jc.Nr;
            SavedHits hits = saved_hits(cb, lay, Tc.total_rays, kRecomputeHits);
            const AdjIn in{dL_dcolor + 3 * p0, dL_dvis ? dL_dvis + p0 : nullptr, dL_dind ? dL_dind + 3 * p0 : nullptr};
            const long long gr = (Tc.total_rays + kShadeThreads - 1) / kShadeThreads;
            // the chunk's rays go to the walk in bucket order, as in the forward
            RayOrder ro{nullptr, nullptr, nullptr, nullptr};
            const bool ord = use_ray_order(Tc.total_rays);
            if (!ord) hits.order = nullptr;  // a short last chunk is walked in slot order
            if (ord) {
                ro = ray_order_bufs(cb + ord_off, Tc.total_rays, hits.order);
                cudaMemsetAsync(ro.hist, 0, 4 * (size_t)kAllBuckets, cs);
            }
            k_sample_rays<1><<<(unsigned)gr, kShadeThreads, 0, cs>>>(Tc, dirs, ro);
            if (ord) launch_ray_order(ro, Tc.total_rays, cs);
            const unsigned* oorder = ro.order;
            dispatch_k(p->k, [&](auto kc) {
                constexpr int K = decltype(kc)::value;
                launch_trace_save<K, 1>(Tc, dirs, res, hits, next_ray, gr, cs, oorder);
                run_adjoint<K>(Tc, dirs, res, hits, adj, work, in, g, cs);
            });
        }
        if (aux) {
            for (int i = 0; i < 2; ++i) {
                GRT_CUDA(cudaEventRecord(aux->join[i], aux->s[i]));
                GRT_CUDA(cudaStreamWaitEvent(st, aux->join[i], 0));
            }
        }
    }
    cudaError_t err = cudaGetLastError();
    if (mem) cudaFreeAsync(mem, st);
    if (err != cudaSuccess) return check_cuda(err, "shade backward kernels");
    return GRT_OK;
}

extern "C" int grt_shade_backward(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                  const grt_gbuffer* gb, const grt_envmap* e, const grt_sampling* smp,
                                  const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                                  const float* dL_dvis, const float* dL_dind, const grt_grads* grads,
                                  void* workspace, size_t workspace_bytes, void* stream) {
    Workspace ws;
    int rc = workspace_arg(workspace, workspace_bytes, &ws);
    if (rc) return rc;
    return shade_backward_impl(b, s, p, gb, e, smp, pixel_list, n_pixels, dL_dcolor, dL_dvis, dL_dind, grads, nullptr,
                               ws, (cudaStream_t)stream);
}

extern "C" size_t grt_shade_backward_workspace_size(int32_t n_pixels, const grt_sampling* smp, int32_t saved) {
    if (n_pixels < 0 || !smp || smp->n_cos < 0 || smp->n_ggx < 0 || smp->n_env < 0) {
        set_error(GRT_ERR_ARG, "bad n_pixels or sampling");
        return 0;
    }
    const int Nr = smp->n_cos + smp->n_ggx + smp->n_env;
    if (Nr <= 0 || n_pixels == 0) return 256;
    return backward_layout(n_pixels, Nr, saved != 0).total;
}

extern "C" int grt_shade_backward_saved(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                        const grt_gbuffer* gb, const grt_envmap* e, const grt_sampling* smp,
                                        const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                                        const float* dL_dvis, const float* dL_dind, int32_t max_hits,
                                        const void* saved, size_t saved_bytes, const grt_grads* grads,
                                        void* workspace, size_t workspace_bytes, void* stream) {
    SaveBufs sb;
    int rc = saved_buffers(saved, saved_bytes, n_pixels, smp, max_hits, &sb);
    if (rc) return rc;
    Workspace ws;
    rc = workspace_arg(workspace, workspace_bytes, &ws);
    if (rc) return rc;
    return shade_backward_impl(b, s, p, gb, e, smp, pixel_list, n_pixels, dL_dcolor, dL_dvis, dL_dind, grads, &sb,
                               ws, (cudaStream_t)stream);
}

extern "C" int grt_adjoint_timing(int32_t enable, float* ms_out) {
    if (enable >= 0) {
        g_adj_timing.on = enable != 0;
        g_adj_timing.have = false;
    }
    if (!ms_out) return GRT_OK;
    if (!g_adj_timing.have) return set_error(GRT_ERR_ARG, "no timed adjoint pass on this thread");
    GRT_CUDA(cudaEventSynchronize(g_adj_timing.ev[3]));
    for (int i = 0; i < 3; ++i)
        GRT_CUDA(cudaEventElapsedTime(ms_out + i, g_adj_timing.ev[i], g_adj_timing.ev[i + 1]));
    return GRT_OK;
}
