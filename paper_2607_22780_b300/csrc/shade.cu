// shade.cu -- grt_shade_pixels / grt_shade_batch / grt_shade_count: MIS sampling, secondary
// trace and rendering-equation accumulation (Eq. 10-13), as three wavefront kernels:
//
//   k_sample_rays  one thread per (pixel, sample j): Philox numbers, proposal of sample j
//                  (Sec. III-D allocation order), direction -> ray buffer (or "no ray")
//   k_trace_rays   one thread per ray: LBVH walk, k-buffer, compositing -> (c_rt, T)
//   k_accumulate   G lanes per pixel: g/q (V L_env + L_ind), V, L_ind per sample, summed
//                  lane-wise in sample order then by a fixed butterfly
//
// Keeping the three phases apart keeps each kernel's code small and its warps on one
// code path; the ray buffers cost 32 bytes per ray of HBM traffic.  A pixel's result is
// a fixed function of its own samples, so it is the same alone and in any batch.
#include "wavefront.cuh"

namespace grt {
namespace {

// Eq. 13: a warp unit shades 32/G pixels; lane sub of a pixel group takes samples
// j = sub + m G in order, the group sums with a butterfly, so the result is fixed.
// 8 blocks per SM (64 registers, a 24-byte spill): the kernel waits on its ray, G-buffer
// and texel loads, and 72 registers had left it at 7 blocks (0.552 -> 0.515 ms for 10 M
// rays on the 300k-surfel 800x800 frame)
#ifndef GRT_ACC_MIN_BLOCKS
#define GRT_ACC_MIN_BLOCKS 8
#endif
template <int CAP>
__global__ void __launch_bounds__(kShadeThreads, GRT_ACC_MIN_BLOCKS) k_accumulate(const __grid_constant__ JobTable<CAP> T,
                                                              const float4* __restrict__ dirs,
                                                              const float4* __restrict__ res) {
    long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= T.total_units) return;  // whole warps leave together
    const ShadeJob& J = T.job[T.find_unit(u)];
    const int lane = threadIdx.x & 31;
    const int G = J.G;
    const int slot = lane / G, sub = lane - slot * G;
    const int li = (int)(u - J.unit_begin) * (32 / G) + slot;
    const bool active = li < J.n_pixels;
    float col[3] = {0.f, 0.f, 0.f}, ind[3] = {0.f, 0.f, 0.f}, light[3] = {0.f, 0.f, 0.f}, vis = 0.f;
    const bool want_light = J.out_light != nullptr;  // the same for the whole warp (one job)
    if (active) {
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        if ((unsigned)pix < (unsigned)(J.gb.W * J.gb.H) && __ldg(J.gb.valid + pix)) {
            PixelState ps = load_pixel(J.gb, pix);
            const long long r0 = J.ray_begin + (long long)li * J.Nr;
            for (int m = 0; m < J.spl; ++m) {
                int j = sub + m * G;
                if (j >= J.Nr) break;
                float4 rr = __ldg(res + r0 + j);
                if (rr.w < 0.f) continue;
                float4 dw = __ldg(dirs + r0 + j);
                SampleWeight sw = sample_weight(J.S, J.env, ps, mk3(dw.x, dw.y, dw.z));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float Lind = c == 0 ? rr.x : (c == 1 ? rr.y : rr.z);
                    const float Li = fmaf(rr.w, sw.L[c], Lind);
                    col[c] = fmaf(sw.g[c], Li, col[c]);
                    ind[c] += Lind;
                    light[c] += Li;
                }
                vis += rr.w;
            }
        }
    }
    for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            col[c] += __shfl_xor_sync(0xffffffffu, col[c], off);
            ind[c] += __shfl_xor_sync(0xffffffffu, ind[c], off);
        }
        vis += __shfl_xor_sync(0xffffffffu, vis, off);
        if (want_light) {
#pragma unroll
            for (int c = 0; c < 3; ++c) light[c] += __shfl_xor_sync(0xffffffffu, light[c], off);
        }
    }
    if (active && sub == 0 && want_light) {
        const float inv = 1.f / (float)J.Nr;
#pragma unroll
        for (int c = 0; c < 3; ++c) J.out_light[3 * (size_t)li + c] = light[c] * inv;
    }
    if (active && sub == 0 && J.out_color) {
        const float inv = 1.f / (float)J.Nr;
        J.out_color[3 * (size_t)li] = col[0] * inv;
        J.out_color[3 * (size_t)li + 1] = col[1] * inv;
        J.out_color[3 * (size_t)li + 2] = col[2] * inv;
        if (J.out_vis) J.out_vis[li] = vis * inv;
        if (J.out_ind) {
            J.out_ind[3 * (size_t)li] = ind[0] * inv;
            J.out_ind[3 * (size_t)li + 1] = ind[1] * inv;
            J.out_ind[3 * (size_t)li + 2] = ind[2] * inv;
        }
    }
}

// Adjoint of the estimate (Eq. 13) and of the mean incident radiance (Eq. 16) into the
// environment map and the per-pixel materials, directions and proposal held fixed: the
// lane layout of k_accumulate; material gradients summed in the same fixed order and added
// to the list entry's outputs, map gradients added to the sample's texel by atomics.
struct MaterialAdj {
    const float *dcol, *dlight;
    float *g_env, *g_albedo, *g_rough, *g_metal;
};

__global__ void __launch_bounds__(kShadeThreads) k_material_adjoint(const __grid_constant__ JobTable<1> T,
                                                                    const float4* __restrict__ dirs,
                                                                    const float4* __restrict__ res, MaterialAdj A) {
    long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= T.total_units) return;
    const ShadeJob& J = T.job[0];
    const int lane = threadIdx.x & 31;
    const int G = J.G;
    const int slot = lane / G, sub = lane - slot * G;
    const int li = (int)(u - J.unit_begin) * (32 / G) + slot;
    const bool active = li < J.n_pixels;
    float ga[3] = {0.f, 0.f, 0.f}, gr = 0.f, gm = 0.f;
    if (active) {
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        if ((unsigned)pix < (unsigned)(J.gb.W * J.gb.H) && __ldg(J.gb.valid + pix)) {
            PixelState ps = load_pixel(J.gb, pix);
            float dc[3], dl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dc[c] = __ldg(A.dcol + 3 * (size_t)li + c);
                dl[c] = A.dlight ? __ldg(A.dlight + 3 * (size_t)li + c) : 0.f;
            }
            const float inv = 1.f / (float)J.Nr;
            const long long r0 = J.ray_begin + (long long)li * J.Nr;
            for (int m = 0; m < J.spl; ++m) {
                int j = sub + m * G;
                if (j >= J.Nr) break;
                float4 rr = __ldg(res + r0 + j);
                if (rr.w < 0.f) continue;
                float4 dw = __ldg(dirs + r0 + j);
                const f3 w = mk3(dw.x, dw.y, dw.z);
                SampleWeight sw = sample_weight(J.S, J.env, ps, w);
                float dfa[3], dfm[3], dfr[3];
                brdf_partials(J.S.brdf, ps.wo, w, ps.n, ps.alb, ps.rough, ps.metal, dfa, dfm, dfr);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float Lind = c == 0 ? rr.x : (c == 1 ? rr.y : rr.z);
                    const float Li = fmaf(rr.w, sw.L[c], Lind);
                    const float k = dc[c] * sw.cq * Li;
                    ga[c] = fmaf(k, dfa[c], ga[c]);
                    gm = fmaf(k, dfm[c], gm);
                    gr = fmaf(k, dfr[c], gr);
                    if (A.g_env) atomicAdd(A.g_env + 3 * (size_t)sw.texel + c, fmaf(dc[c], sw.g[c], dl[c]) * rr.w * inv);
                }
            }
        }
    }
    for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ga[c] += __shfl_xor_sync(0xffffffffu, ga[c], off);
        gr += __shfl_xor_sync(0xffffffffu, gr, off);
        gm += __shfl_xor_sync(0xffffffffu, gm, off);
    }
    if (active && sub == 0) {
        const float inv = 1.f / (float)J.Nr;
        if (A.g_albedo)
#pragma unroll
            for (int c = 0; c < 3; ++c) A.g_albedo[3 * (size_t)li + c] += ga[c] * inv;
        if (A.g_rough) A.g_rough[li] += gr * inv;
        if (A.g_metal) A.g_metal[li] += gm * inv;
    }
}

// Lays out the jobs' rays and accumulation units, then runs the three kernels.
// Optional phase timing (grt_phase_timing): events on the call's stream around the
// sample, trace and accumulate kernels of the most recent shading call of this thread.
struct PhaseTiming {
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
thread_local PhaseTiming g_timing;

template <bool COUNT, int CAP>
int run_jobs(JobTable<CAP>& T, int k, long long* counters, cudaStream_t st, const SaveBufs* save = nullptr,
             const RelightDev* rel = nullptr, const MeshDev* mesh = nullptr, const Workspace& ws = Workspace{}) {
    long long rays = 0, units = 0;
    for (int i = 0; i < T.n_jobs; ++i) {
        ShadeJob& J = T.job[i];
        J.ray_begin = rays;
        J.unit_begin = units;
        rays += (long long)J.n_pixels * J.Nr;
        units += (J.n_pixels + (32 / J.G) - 1) / (32 / J.G);
    }
    T.total_rays = rays;
    T.total_units = units;
    if (rays == 0) return GRT_OK;
    float4* buf = nullptr;
    char* order_buf = nullptr;
    float4 *dirs, *res;
    unsigned long long* next_ray;
    // every walk but the counting pass takes its rays in bucket order (32-bit slot indices)
    const bool ord = !COUNT && use_ray_order(rays);
    const size_t extra = ord ? order_scratch_bytes(rays) : 0;
    const size_t need = save ? extra : shade_ws_bytes(rays, ord);
    char* mem = nullptr;    // from the pool, freed at the end of the call
    char* base = nullptr;   // the call's ray buffers: caller workspace or `mem`
    if (ws.ptr) {
        if (ws.bytes < need) return set_error(GRT_ERR_ARG, "workspace holds %zu bytes, %zu needed", ws.bytes, need);
        base = static_cast<char*>(ws.ptr);
    } else if (need > 0) {
        keep_pool_memory();
        GRT_CUDA(cudaMallocAsync((void**)&mem, need, st));
        base = mem;
    }
    if (save) {
        dirs = save->dirs;
        res = save->res;
        next_ray = save->next;
        if (ord) order_buf = base;
    } else {
        buf = reinterpret_cast<float4*>(base);
        dirs = buf;
        res = buf + rays;
        next_ray = reinterpret_cast<unsigned long long*>(buf + 2 * rays);
        if (ord) order_buf = reinterpret_cast<char*>(buf + 2 * rays + 1);
    }
    const long long gr = (rays + kShadeThreads - 1) / kShadeThreads;
    g_timing.mark(0, st);
    RayOrder ro{nullptr, nullptr, nullptr, nullptr};
    if (order_buf) {
        // a saving pass keeps its order in the record, for the replay
        ro = ray_order_bufs(order_buf, rays, save ? save->hits.order : nullptr);
        cudaMemsetAsync(ro.hist, 0, 4 * (size_t)kAllBuckets, st);
    }
    k_sample_rays<CAP><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, ro);
    if (order_buf) launch_ray_order(ro, rays, st);
    const unsigned* oorder = ro.order;
    g_timing.mark(1, st);
    dispatch_k(k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (COUNT) {  // counting pass: one ray per thread, same traversal
            k_trace_rays<K, COUNT, CAP><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, res, counters);
        } else if (save) {
            if constexpr (CAP == 1) launch_trace_save<K, CAP>(T, dirs, res, save->hits, next_ray, gr, st, oorder);
        } else if (rel && mesh) {
            if constexpr (CAP == 1)
                k_trace_rays_mesh<CAP><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, res, *rel, *mesh, oorder);
        } else if (rel) {
            if constexpr (CAP == 1) launch_trace_relight<K, CAP>(T, dirs, res, *rel, next_ray, gr, st, oorder);
        } else {
            launch_trace_dyn<K, CAP>(T, dirs, res, next_ray, gr, st, oorder);
        }
    });
    if (!COUNT) {
        const long long ga = (units * 32 + kShadeThreads - 1) / kShadeThreads;
        g_timing.mark(2, st);
        k_accumulate<CAP><<<(unsigned)ga, kShadeThreads, 0, st>>>(T, dirs, res);
        g_timing.mark(3, st);
        g_timing.have = g_timing.on && g_timing.ok;
    }
    cudaError_t e = cudaGetLastError();
    if (mem) cudaFreeAsync(mem, st);
    if (e != cudaSuccess) return check_cuda(e, "shade kernels");
    return GRT_OK;
}

template <bool COUNT>
int launch_single(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                  const grt_envmap* e, const grt_sampling* smp, const int* pl, int n, float* oc, float* ov, float* oi,
                  long long* counters, cudaStream_t st, const SaveBufs* save = nullptr,
                  const RelightDev* rel = nullptr, const Workspace& ws = Workspace{}) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    JobTable<1> T;
    T.P = to_params(*p);
    T.n_jobs = 1;
    rc = make_job(b, s, g, e, smp, pl, n, oc, ov, oi, &T.job[0]);
    if (rc) return rc;
    if (n == 0) return GRT_OK;
    if (T.job[0].n_pixels == 0) {  // N_r = 0: every output is zero
        if (oc) k_zero_outputs<<<(n + 255) / 256, 256, 0, st>>>(oc, ov, oi, n);
        return launch_error("k_zero_outputs");
    }
    return run_jobs<COUNT>(T, p->k, counters, st, save, rel, nullptr, ws);
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_shade_pixels(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                                const grt_envmap* e, const grt_sampling* smp, const int32_t* pixel_list,
                                int32_t n_pixels, float* out_color, float* out_vis, float* out_ind, void* workspace,
                                size_t workspace_bytes, void* stream) {
    if (n_pixels > 0 && !out_color) return set_error(GRT_ERR_ARG, "out_color is NULL");
    Workspace ws;
    int rc = workspace_arg(workspace, workspace_bytes, &ws);
    if (rc) return rc;
    return launch_single<false>(b, s, p, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, nullptr,
                                (cudaStream_t)stream, nullptr, nullptr, ws);
}

extern "C" size_t grt_shade_workspace_size(int64_t n_rays) {
    if (n_rays < 0) {
        set_error(GRT_ERR_ARG, "n_rays < 0");
        return 0;
    }
    return shade_ws_bytes(n_rays, use_ray_order(n_rays));
}

extern "C" int grt_shade_count(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                               const grt_envmap* e, const grt_sampling* smp, const int32_t* pixel_list,
                               int32_t n_pixels, long long* counters, void* stream) {
    if (!counters) return set_error(GRT_ERR_ARG, "counters is NULL");
    return launch_single<true>(b, s, p, g, e, smp, pixel_list, n_pixels, nullptr, nullptr, nullptr, counters,
                               (cudaStream_t)stream);
}

extern "C" size_t grt_shade_saved_bytes(int32_t n_pixels, const grt_sampling* smp, int32_t max_hits) {
    if (n_pixels < 0 || !smp || smp->n_cos < 0 || smp->n_ggx < 0 || smp->n_env < 0) {
        set_error(GRT_ERR_ARG, "bad n_pixels or sampling");
        return 0;
    }
    if (max_hits < 0 || max_hits > GRT_MAX_SAVED_HITS) {
        set_error(GRT_ERR_ARG, "max_hits = %d outside [0, %d]", max_hits, GRT_MAX_SAVED_HITS);
        return 0;
    }
    const long long R = (long long)n_pixels * (smp->n_cos + smp->n_ggx + smp->n_env);
    return saved_layout(R, max_hits).total;
}

extern "C" int grt_shade_pixels_save(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                     const grt_gbuffer* g, const grt_envmap* e, const grt_sampling* smp,
                                     const int32_t* pixel_list, int32_t n_pixels, float* out_color, float* out_vis,
                                     float* out_ind, int32_t max_hits, void* saved, size_t saved_bytes,
                                     void* workspace, size_t workspace_bytes, void* stream) {
    if (n_pixels > 0 && !out_color) return set_error(GRT_ERR_ARG, "out_color is NULL");
    SaveBufs sb;
    int rc = saved_buffers(saved, saved_bytes, n_pixels, smp, max_hits, &sb);
    if (rc) return rc;
    Workspace ws;
    rc = workspace_arg(workspace, workspace_bytes, &ws);
    if (rc) return rc;
    return launch_single<false>(b, s, p, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, nullptr,
                                (cudaStream_t)stream, &sb, nullptr, ws);
}

extern "C" int grt_shade_relight(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                 const grt_gbuffer* g, const grt_envmap* e, const void* prefiltered,
                                 const grt_sampling* smp, const int32_t* pixel_list, int32_t n_pixels,
                                 float* out_color, float* out_vis, float* out_ind, void* stream) {
    if (n_pixels > 0 && !out_color) return set_error(GRT_ERR_ARG, "out_color is NULL");
    if (!prefiltered || ((uintptr_t)prefiltered & 15))
        return set_error(GRT_ERR_ARG, "prefiltered must be a 16-byte aligned device pointer");
    if (s && s->n > 0 && (!s->albedo || !s->rough || !s->metal || !s->quat))
        return set_error(GRT_ERR_ARG, "surfels need quat, albedo, rough and metal for relighting");
    const PrefLayout L = pref_layout();
    const float* f = static_cast<const float*>(prefiltered);
    const RelightDev E{f + L.diff, f + L.spec, f + L.lut, f + L.poles};
    return launch_single<false>(b, s, p, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, nullptr,
                                (cudaStream_t)stream, nullptr, &E);
}

extern "C" int grt_shade_pixels_light(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                      const grt_gbuffer* g, const grt_envmap* e, const grt_sampling* smp,
                                      const int32_t* pixel_list, int32_t n_pixels, float* out_color, float* out_vis,
                                      float* out_ind, float* out_light, void* stream) {
    if (n_pixels > 0 && (!out_color || !out_light)) return set_error(GRT_ERR_ARG, "out_color or out_light is NULL");
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    JobTable<1> T;
    T.P = to_params(*p);
    T.n_jobs = 1;
    rc = make_job(b, s, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, &T.job[0]);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_pixels == 0) return GRT_OK;
    if (T.job[0].n_pixels == 0) {  // N_r = 0: every output is zero
        k_zero_outputs<<<(n_pixels + 255) / 256, 256, 0, st>>>(out_color, out_vis, out_ind, n_pixels);
        GRT_CUDA(cudaMemsetAsync(out_light, 0, sizeof(float) * 3 * (size_t)n_pixels, st));
        return launch_error("k_zero_outputs");
    }
    T.job[0].out_light = out_light;
    return run_jobs<false>(T, p->k, nullptr, st);
}

extern "C" int grt_shade_backward_material(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                           const grt_gbuffer* g, const grt_envmap* e, const grt_sampling* smp,
                                           const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                                           const float* dL_dlight, float* grad_env, float* grad_albedo,
                                           float* grad_rough, float* grad_metal, void* stream) {
    if (n_pixels > 0 && !dL_dcolor) return set_error(GRT_ERR_ARG, "dL_dcolor is NULL");
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    JobTable<1> T;
    T.P = to_params(*p);
    T.n_jobs = 1;
    rc = make_job(b, s, g, e, smp, pixel_list, n_pixels, nullptr, nullptr, nullptr, &T.job[0]);
    if (rc) return rc;
    ShadeJob& J = T.job[0];
    if (J.n_pixels == 0) return GRT_OK;
    const long long rays = (long long)J.n_pixels * J.Nr;
    const long long units = (J.n_pixels + (32 / J.G) - 1) / (32 / J.G);
    T.total_rays = rays;
    T.total_units = units;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_memory();
    float4* buf = nullptr;
    const bool ord = use_ray_order(rays);
    const size_t extra = ord ? order_scratch_bytes(rays) : 0;
    GRT_CUDA(cudaMallocAsync((void**)&buf, sizeof(float4) * (2 * (size_t)rays + 1) + extra, st));
    float4* dirs = buf;
    float4* res = buf + rays;
    unsigned long long* next_ray = reinterpret_cast<unsigned long long*>(buf + 2 * rays);
    RayOrder ro{nullptr, nullptr, nullptr, nullptr};
    if (ord) {
        ro = ray_order_bufs(buf + 2 * rays + 1, rays);
        cudaMemsetAsync(ro.hist, 0, 4 * (size_t)kAllBuckets, st);
    }
    const long long gr = (rays + kShadeThreads - 1) / kShadeThreads;
    k_sample_rays<1><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, ro);
    if (ord) launch_ray_order(ro, rays, st);
    const unsigned* oorder = ro.order;
    dispatch_k(p->k, [&](auto kc) {
        launch_trace_dyn<decltype(kc)::value, 1>(T, dirs, res, next_ray, gr, st, oorder);
    });
    const long long ga = (units * 32 + kShadeThreads - 1) / kShadeThreads;
    k_material_adjoint<<<(unsigned)ga, kShadeThreads, 0, st>>>(
        T, dirs, res, MaterialAdj{dL_dcolor, dL_dlight, grad_env, grad_albedo, grad_rough, grad_metal});
    cudaError_t err = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (err != cudaSuccess) return check_cuda(err, "material adjoint kernels");
    return GRT_OK;
}

extern "C" int grt_shade_relight_mesh(const grt_bvh* b, const grt_mesh* m, const grt_trace_params* p,
                                      const grt_gbuffer* g, const grt_envmap* e, const void* prefiltered,
                                      const grt_sampling* smp, const int32_t* pixel_list, int32_t n_pixels,
                                      float* out_color, float* out_vis, float* out_ind, void* stream) {
    if (!b || !m) return set_error(GRT_ERR_ARG, "mesh bvh or mesh is NULL");
    if (m->n_triangles != b->n) return set_error(GRT_ERR_ARG, "mesh has %d triangles, the tree %d", m->n_triangles, b->n);
    if (m->n_triangles > 0 && (!m->tri || !m->normal || !m->albedo || !m->rough || !m->metal))
        return set_error(GRT_ERR_ARG, "mesh attributes must be non-NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (n_pixels > 0 && !out_color) return set_error(GRT_ERR_ARG, "out_color is NULL");
    if (!prefiltered || ((uintptr_t)prefiltered & 15))
        return set_error(GRT_ERR_ARG, "prefiltered must be a 16-byte aligned device pointer");
    grt_surfels none{};
    none.n = b->n;
    none.color_dim = 3;
    JobTable<1> T;
    T.P = to_params(*p);
    T.n_jobs = 1;
    rc = make_job(b, &none, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, &T.job[0]);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_pixels == 0) return GRT_OK;
    if (T.job[0].n_pixels == 0) {
        k_zero_outputs<<<(n_pixels + 255) / 256, 256, 0, st>>>(out_color, out_vis, out_ind, n_pixels);
        return launch_error("k_zero_outputs");
    }
    const PrefLayout L = pref_layout();
    const float* f = static_cast<const float*>(prefiltered);
    const RelightDev E{f + L.diff, f + L.spec, f + L.lut, f + L.poles};
    const MeshDev M{m->tri, m->normal, m->albedo, m->rough, m->metal, m->n_vertices};
    return run_jobs<false>(T, p->k, nullptr, st, nullptr, &E, &M);
}

extern "C" int grt_shade_batch(const grt_shade_request* req, int32_t n_req, const grt_trace_params* p,
                               void* workspace, size_t workspace_bytes, void* stream) {
    if (!req || n_req <= 0 || n_req > GRT_MAX_BATCH)
        return set_error(GRT_ERR_ARG, "need 1 <= n_requests <= %d", GRT_MAX_BATCH);
    int rc = check_params(p);
    if (rc) return rc;
    Workspace ws;
    rc = workspace_arg(workspace, workspace_bytes, &ws);
    if (rc) return rc;
    static thread_local JobTable<GRT_MAX_BATCH> T;
    T.P = to_params(*p);
    T.n_jobs = 0;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n_req; ++i) {
        rc = check_trace_inputs(req[i].bvh, req[i].surfels, p);
        if (rc) return rc;
        if (req[i].n_pixels > 0 && !req[i].out_color) return set_error(GRT_ERR_ARG, "request %d: out_color is NULL", i);
        ShadeJob J;
        rc = make_job(req[i].bvh, req[i].surfels, &req[i].gbuffer, &req[i].env, &req[i].sampling, req[i].pixel_list,
                      req[i].n_pixels, req[i].out_color, req[i].out_vis, req[i].out_ind, &J);
        if (rc) return rc;
        if (!req[i].pixel_list) {
            if (req[i].pixel_offset < 0 ||
                (long long)req[i].pixel_offset + req[i].n_pixels > (long long)req[i].gbuffer.W * req[i].gbuffer.H)
                return set_error(GRT_ERR_ARG, "request %d: pixel slice outside the G-buffer", i);
            J.pixel_offset = req[i].pixel_offset;
        }
        if (J.n_pixels == 0) {
            if (req[i].n_pixels > 0)
                k_zero_outputs<<<(req[i].n_pixels + 255) / 256, 256, 0, st>>>(req[i].out_color, req[i].out_vis,
                                                                              req[i].out_ind, req[i].n_pixels);
            continue;
        }
        T.job[T.n_jobs++] = J;
    }
    if (T.n_jobs == 0) return launch_error("k_zero_outputs");
    return run_jobs<false>(T, p->k, nullptr, st, nullptr, nullptr, nullptr, ws);
}

extern "C" int grt_phase_timing(int32_t enable, float* ms_out) {
    if (enable >= 0) {
        g_timing.on = enable != 0;
        g_timing.have = false;
    }
    if (!ms_out) return GRT_OK;
    if (!g_timing.have) return set_error(GRT_ERR_ARG, "no timed shading call on this thread");
    GRT_CUDA(cudaEventSynchronize(g_timing.ev[3]));
    for (int i = 0; i < 3; ++i) GRT_CUDA(cudaEventElapsedTime(ms_out + i, g_timing.ev[i], g_timing.ev[i + 1]));
    return GRT_OK;
}
