// shade.cu -- grt_shade_pixels / grt_shade_batch / grt_shade_count: fused MIS sampling,
// secondary trace and rendering-equation accumulation (Eq. 10-13).
//
// A warp shades 32/G pixels at once: the G lanes of a pixel group take samples
// j = lane + m G (Sec. III-D allocation order), trace them (Eq. 11) and accumulate
// g/q (V L_env + L_ind); the group then sums its lanes with a fixed butterfly, so a
// pixel's result depends only on its own samples, never on what else is in the launch.
#include "common_args.cuh"
#include "shade.cuh"

namespace grt {

struct ShadeJob {
    DevBvh bvh;
    const float* color;
    int cdim;
    GbufDev gb;
    EnvDev env;
    Sampling S;
    const int* pixel_list;
    int n_pixels;
    float *out_color, *out_vis, *out_ind;
    int G, spl;        // lanes per pixel, samples per lane
    int unit_begin;    // first warp unit of this job
};

struct JobTable {
    TraceParams P;
    int n_jobs;
    int total_units;
    ShadeJob job[GRT_MAX_BATCH];
};

namespace {

constexpr int kShadeThreads = 128;

template <int K, bool COUNT>
__device__ __forceinline__ void shade_unit(const ShadeJob& J, const TraceParams& P, int u, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    const int G = J.G;
    const int slot = lane / G, sub = lane - slot * G;
    const int li = u * (32 / G) + slot;
    const bool active = li < J.n_pixels;
    int pix = active ? (J.pixel_list ? __ldg(J.pixel_list + li) : li) : 0;
    if ((unsigned)pix >= (unsigned)(J.gb.W * J.gb.H)) {
        if (active) atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
        pix = 0;
    }
    const bool valid = active && pix == (J.pixel_list ? __ldg(J.pixel_list + li) : li) && __ldg(J.gb.valid + pix) != 0;
    const int Nr = J.S.n_cos + J.S.n_ggx + J.S.n_env;
    float col[3] = {0.f, 0.f, 0.f}, ind[3] = {0.f, 0.f, 0.f}, vis = 0.f;
    if (valid) {
        PixelState ps = load_pixel(J.gb, pix);
        for (int m = 0; m < J.spl; ++m) {
            int j = sub + m * G;
            if (j >= Nr) break;
            f3 w;
            if (!draw_direction(J.S, J.env, ps, pix, j, &w)) continue;
            RayState r = make_ray(ps.x, w);
            ColourVisitor v(J.color, J.cdim, w, nullptr, 0);
            trace_ray<K, COUNT>(J.bvh, r, P, v, cnt);
            SampleWeight sw = sample_weight(J.S, J.env, ps, w);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                col[c] = fmaf(sw.g[c], fmaf(v.T, sw.L[c], v.c[c]), col[c]);
                ind[c] += v.c[c];
            }
            vis += v.T;
        }
    }
    // butterfly over the G lanes of the group (same tree for every lane)
    for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            col[c] += __shfl_xor_sync(0xffffffffu, col[c], off);
            ind[c] += __shfl_xor_sync(0xffffffffu, ind[c], off);
        }
        vis += __shfl_xor_sync(0xffffffffu, vis, off);
    }
    if (active && sub == 0 && J.out_color) {
        float inv = Nr > 0 ? 1.f / (float)Nr : 0.f;
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

__device__ __forceinline__ void flush_counters(Counters c, long long* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c.nodes += __shfl_xor_sync(0xffffffffu, c.nodes, o);
        c.tests += __shfl_xor_sync(0xffffffffu, c.tests, o);
        c.comp += __shfl_xor_sync(0xffffffffu, c.comp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long*)out, (unsigned long long)c.nodes);
        atomicAdd((unsigned long long*)out + 1, (unsigned long long)c.tests);
        atomicAdd((unsigned long long*)out + 2, (unsigned long long)c.comp);
    }
}

// One job, one warp unit per warp of the grid.
template <int K, bool COUNT>
__global__ void __launch_bounds__(kShadeThreads) k_shade(const __grid_constant__ ShadeJob J, TraceParams P,
                                                         long long* counters) {
    int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Counters cnt{0, 0, 0};
    int units = (J.n_pixels + (32 / J.G) - 1) / (32 / J.G);
    if (u < units) shade_unit<K, COUNT>(J, P, u, cnt);
    if (COUNT) flush_counters(cnt, counters);
}

// Many jobs, persistent warps pulling units from a shared counter.
template <int K>
__global__ void __launch_bounds__(kShadeThreads) k_shade_batch(const __grid_constant__ JobTable T, int* counter) {
    const int lane = threadIdx.x & 31;
    Counters cnt{0, 0, 0};
    while (true) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= T.total_units) break;
        int j = 0;
        while (j + 1 < T.n_jobs && unit >= T.job[j + 1].unit_begin) ++j;
        shade_unit<K, false>(T.job[j], T.P, unit - T.job[j].unit_begin, cnt);
    }
}

int make_job(const grt_bvh* b, const grt_surfels* s, const grt_gbuffer* g, const grt_envmap* e,
             const grt_sampling* smp, const int* pixel_list, int n_pixels, float* oc, float* ov, float* oi,
             ShadeJob* J) {
    if (!g || !e || !smp) return set_error(GRT_ERR_ARG, "gbuffer, env or sampling is NULL");
    if (!g->pos || !g->normal || !g->albedo || !g->rough || !g->metal || !g->valid)
        return set_error(GRT_ERR_ARG, "gbuffer arrays must be non-NULL");
    if (g->W <= 0 || g->H <= 0) return set_error(GRT_ERR_ARG, "gbuffer size %dx%d", g->W, g->H);
    if (n_pixels < 0) return set_error(GRT_ERR_ARG, "n_pixels < 0");
    if (!pixel_list && n_pixels > g->W * g->H) return set_error(GRT_ERR_ARG, "n_pixels exceeds W*H");
    if (!e->tables || e->W <= 0 || e->H <= 0) return set_error(GRT_ERR_ARG, "environment tables missing");
    if (smp->n_cos < 0 || smp->n_ggx < 0 || smp->n_env < 0) return set_error(GRT_ERR_ARG, "negative sample count");
    int Nr = smp->n_cos + smp->n_ggx + smp->n_env;
    if (Nr > 1024) return set_error(GRT_ERR_ARG, "N_r = %d exceeds 1024", Nr);
    if (smp->brdf != 0 && smp->brdf != 1) return set_error(GRT_ERR_ARG, "brdf must be 0 or 1");
    J->bvh = dev_bvh(b);
    J->color = s->color;
    J->cdim = s->color_dim;
    J->gb = GbufDev{g->pos, g->normal, g->albedo, g->rough, g->metal, g->valid, g->eye[0], g->eye[1], g->eye[2], g->W, g->H};
    EnvLayout l = env_layout(e->W, e->H);
    const char* tb = (const char*)e->tables;
    J->env = EnvDev{(const float4*)(tb + l.texel), (const float*)(tb + l.marg), (const float*)(tb + l.cond), e->W, e->H,
                    (float)e->W * (float)e->H / (2.f * kPi * kPi)};
    J->S = Sampling{smp->n_cos, smp->n_ggx, smp->n_env, smp->brdf, (uint32_t)(smp->seed & 0xFFFFFFFFu),
                    (uint32_t)(smp->seed >> 32)};
    J->pixel_list = pixel_list;
    J->n_pixels = n_pixels;
    J->out_color = oc;
    J->out_vis = ov;
    J->out_ind = oi;
    J->G = group_lanes(Nr > 0 ? Nr : 1);
    J->spl = Nr > 0 ? (Nr + J->G - 1) / J->G : 0;
    J->unit_begin = 0;
    return GRT_OK;
}

template <bool COUNT>
int launch_single(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                  const grt_envmap* e, const grt_sampling* smp, const int* pl, int n, float* oc, float* ov, float* oi,
                  long long* counters, cudaStream_t st) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    ShadeJob J;
    rc = make_job(b, s, g, e, smp, pl, n, oc, ov, oi, &J);
    if (rc) return rc;
    if (n == 0) return GRT_OK;
    int units = (n + (32 / J.G) - 1) / (32 / J.G);
    long long threads = (long long)units * 32;
    int grid = (int)((threads + kShadeThreads - 1) / kShadeThreads);
    TraceParams P = to_params(*p);
    dispatch_k(p->k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        k_shade<K, COUNT><<<grid, kShadeThreads, 0, st>>>(J, P, counters);
    });
    return launch_error("k_shade");
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_shade_pixels(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                                const grt_envmap* e, const grt_sampling* smp, const int32_t* pixel_list,
                                int32_t n_pixels, float* out_color, float* out_vis, float* out_ind, void* stream) {
    if (n_pixels > 0 && !out_color) return set_error(GRT_ERR_ARG, "out_color is NULL");
    return launch_single<false>(b, s, p, g, e, smp, pixel_list, n_pixels, out_color, out_vis, out_ind, nullptr,
                                (cudaStream_t)stream);
}

extern "C" int grt_shade_count(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                               const grt_envmap* e, const grt_sampling* smp, const int32_t* pixel_list,
                               int32_t n_pixels, long long* counters, void* stream) {
    if (!counters) return set_error(GRT_ERR_ARG, "counters is NULL");
    return launch_single<true>(b, s, p, g, e, smp, pixel_list, n_pixels, nullptr, nullptr, nullptr, counters,
                               (cudaStream_t)stream);
}

extern "C" int grt_shade_batch(const grt_shade_request* req, int32_t n_req, const grt_trace_params* p,
                               int32_t* work_counter, void* stream) {
    if (!req || n_req <= 0 || n_req > GRT_MAX_BATCH)
        return set_error(GRT_ERR_ARG, "need 1 <= n_requests <= %d", GRT_MAX_BATCH);
    if (!work_counter) return set_error(GRT_ERR_ARG, "work_counter is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    static thread_local JobTable T;
    T.P = to_params(*p);
    T.n_jobs = n_req;
    int units = 0;
    for (int i = 0; i < n_req; ++i) {
        rc = check_trace_inputs(req[i].bvh, req[i].surfels, p);
        if (rc) return rc;
        rc = make_job(req[i].bvh, req[i].surfels, &req[i].gbuffer, &req[i].env, &req[i].sampling, req[i].pixel_list,
                      req[i].n_pixels, req[i].out_color, req[i].out_vis, req[i].out_ind, &T.job[i]);
        if (rc) return rc;
        T.job[i].unit_begin = units;
        units += (req[i].n_pixels + (32 / T.job[i].G) - 1) / (32 / T.job[i].G);
    }
    T.total_units = units;
    if (units == 0) return GRT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    GRT_CUDA(cudaMemsetAsync(work_counter, 0, sizeof(int32_t), st));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    dispatch_k(p->k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shade_batch<K>, kShadeThreads, 0);
        int grid = sms * (per_sm > 0 ? per_sm : 1);
        int max_grid = (units * 32 + kShadeThreads - 1) / kShadeThreads;
        if (grid > max_grid) grid = max_grid;
        k_shade_batch<K><<<grid, kShadeThreads, 0, st>>>(T, work_counter);
    });
    return launch_error("k_shade_batch");
}
