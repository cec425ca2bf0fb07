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
#include <mutex>

#include "common_args.cuh"
#include "shade.cuh"

namespace grt {

constexpr int kShadeThreads = 128;

struct ShadeJob {
    DevBvh bvh;
    const float* color;
    int cdim;
    GbufDev gb;
    EnvDev env;
    Sampling S;
    const int* pixel_list;
    int n_pixels;
    int Nr;
    float *out_color, *out_vis, *out_ind;
    int G, spl;              // accumulation: lanes per pixel, samples per lane
    long long ray_begin;     // first ray of this job in the launch's ray buffers
    long long unit_begin;    // first accumulation warp unit of this job
};

template <int CAP>
struct JobTable {
    TraceParams P;
    int n_jobs;
    long long total_rays;
    long long total_units;
    ShadeJob job[CAP];

    __device__ __forceinline__ int find_ray(long long r) const {
        int j = 0;
        while (j + 1 < n_jobs && r >= job[j + 1].ray_begin) ++j;
        return j;
    }
    __device__ __forceinline__ int find_unit(long long u) const {
        int j = 0;
        while (j + 1 < n_jobs && u >= job[j + 1].unit_begin) ++j;
        return j;
    }
};

namespace {

__device__ __forceinline__ int pixel_of(const ShadeJob& J, int li) {
    int pix = J.pixel_list ? __ldg(J.pixel_list + li) : li;
    if ((unsigned)pix >= (unsigned)(J.gb.W * J.gb.H)) {
        atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
        return -1;
    }
    return pix;
}

// ray buffer entry: (direction, 1) for a traced sample, (0, 0, 0, 0) for none
template <int CAP>
__global__ void __launch_bounds__(kShadeThreads) k_sample_rays(const __grid_constant__ JobTable<CAP> T,
                                                               float4* __restrict__ dirs) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T.total_rays) return;
    const ShadeJob& J = T.job[T.find_ray(r)];
    long long lr = r - J.ray_begin;
    int li = (int)(lr / J.Nr), j = (int)(lr - (long long)li * J.Nr);
    int pix = pixel_of(J, li);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pix >= 0 && __ldg(J.gb.valid + pix)) {
        PixelState ps = load_pixel(J.gb, pix);
        f3 w;
        if (draw_direction(J.S, J.env, ps, pix, j, &w)) out = make_float4(w.x, w.y, w.z, 1.f);
    }
    dirs[r] = out;
}

// (c_rt, T) per ray; T = -1 marks "no ray"
template <int K, bool COUNT, int CAP>
__global__ void __launch_bounds__(kShadeThreads) k_trace_rays(const __grid_constant__ JobTable<CAP> T,
                                                              const float4* __restrict__ dirs, float4* __restrict__ res,
                                                              long long* counters) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Counters cnt{0, 0, 0};
    if (r < T.total_rays) {
        float4 dw = __ldg(dirs + r);
        float4 out = make_float4(0.f, 0.f, 0.f, -1.f);
        if (dw.w != 0.f) {
            const ShadeJob& J = T.job[T.find_ray(r)];
            int li = (int)((r - J.ray_begin) / J.Nr);
            int pix = J.pixel_list ? __ldg(J.pixel_list + li) : li;
            f3 o = mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
                       __ldg(J.gb.pos + 3 * (size_t)pix + 2));
            f3 d = mk3(dw.x, dw.y, dw.z);
            RayState rs = make_ray(o, d);
            ColourVisitor v(J.color, J.cdim, d, nullptr, 0);
            trace_ray<K, COUNT>(J.bvh, rs, T.P, v, cnt);
            out = make_float4(v.c[0], v.c[1], v.c[2], v.T);
        }
        if (!COUNT) res[r] = out;
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt.nodes += __shfl_xor_sync(0xffffffffu, cnt.nodes, o);
            cnt.tests += __shfl_xor_sync(0xffffffffu, cnt.tests, o);
            cnt.comp += __shfl_xor_sync(0xffffffffu, cnt.comp, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd((unsigned long long*)counters, (unsigned long long)cnt.nodes);
            atomicAdd((unsigned long long*)counters + 1, (unsigned long long)cnt.tests);
            atomicAdd((unsigned long long*)counters + 2, (unsigned long long)cnt.comp);
        }
    }
}

// Persistent variant of k_trace_rays: warps stay resident and walk their rays one wide
// node per step; once kRefillLanes lanes have finished, the warp claims that many new
// rays from a global counter, so a long ray holds one lane instead of a whole warp.
constexpr int kRefillLanes = 8;
#ifndef GRT_TRACE_MIN_BLOCKS
#define GRT_TRACE_MIN_BLOCKS 4  // 128 threads x 4 blocks: at most 128 registers per thread
#endif

template <int K, int CAP>
__global__ void __launch_bounds__(kShadeThreads, GRT_TRACE_MIN_BLOCKS) k_trace_rays_dyn(const __grid_constant__ JobTable<CAP> T,
                                                                  const float4* __restrict__ dirs,
                                                                  float4* __restrict__ res,
                                                                  unsigned long long* __restrict__ next_ray) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int2 stack[kStackDepth];
    TraceState<K> ts;
    ColourVisitor cv(nullptr, 3, mk3(0.f, 0.f, 0.f), nullptr, 0);
    const ShadeJob* J = &T.job[0];
    long long ray = -1;
    bool act = false, drained = false;
    Counters cnt{0, 0, 0};
    while (true) {
        unsigned idle = __ballot_sync(0xffffffffu, !act);
        int nidle = __popc(idle);
        if (!drained && (nidle >= kRefillLanes || nidle == 32)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(next_ray, (unsigned long long)nidle);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + nidle >= (unsigned long long)T.total_rays) drained = true;
            if (!act) {
                long long r = (long long)base + __popc(idle & lt);
                if (r < T.total_rays) {
                    ray = r;
                    float4 dw = __ldg(dirs + r);
                    if (dw.w == 0.f) {
                        res[r] = make_float4(0.f, 0.f, 0.f, -1.f);
                    } else {
                        J = &T.job[T.find_ray(r)];
                        int li = (int)((r - J->ray_begin) / J->Nr);
                        int pix = J->pixel_list ? __ldg(J->pixel_list + li) : li;
                        f3 o = mk3(__ldg(J->gb.pos + 3 * (size_t)pix), __ldg(J->gb.pos + 3 * (size_t)pix + 1),
                                   __ldg(J->gb.pos + 3 * (size_t)pix + 2));
                        f3 d = mk3(dw.x, dw.y, dw.z);
                        trace_begin(J->bvh, ts, o, d, T.P);
                        cv.color = J->color;
                        cv.cdim = J->cdim;
                        cv.d = d;
                        cv.c[0] = cv.c[1] = cv.c[2] = 0.f;
                        cv.nh = 0;
                        act = true;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, act)) {
            if (drained) break;
            continue;
        }
        if (act && !trav_step<K, false>(J->bvh, ts, stack, T.P, cnt)) {
            if (round_end<K, false>(J->bvh, ts, T.P, cv, cnt)) {
                res[ray] = make_float4(cv.c[0], cv.c[1], cv.c[2], ts.T);
                act = false;
            }
        }
    }
}

// Eq. 13: a warp unit shades 32/G pixels; lane sub of a pixel group takes samples
// j = sub + m G in order, the group sums with a butterfly, so the result is fixed.
template <int CAP>
__global__ void __launch_bounds__(kShadeThreads) k_accumulate(const __grid_constant__ JobTable<CAP> T,
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
    float col[3] = {0.f, 0.f, 0.f}, ind[3] = {0.f, 0.f, 0.f}, vis = 0.f;
    if (active) {
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : li;
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
                    col[c] = fmaf(sw.g[c], fmaf(rr.w, sw.L[c], Lind), col[c]);
                    ind[c] += Lind;
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

__global__ void k_zero_outputs(float* c, float* v, float* i, int n) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    c[3 * (size_t)t] = c[3 * (size_t)t + 1] = c[3 * (size_t)t + 2] = 0.f;
    if (v) v[t] = 0.f;
    if (i) i[3 * (size_t)t] = i[3 * (size_t)t + 1] = i[3 * (size_t)t + 2] = 0.f;
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
    J->n_pixels = Nr > 0 ? n_pixels : 0;
    J->Nr = Nr > 0 ? Nr : 1;
    J->out_color = oc;
    J->out_vis = ov;
    J->out_ind = oi;
    J->G = group_lanes(J->Nr);
    J->spl = (J->Nr + J->G - 1) / J->G;
    J->ray_begin = 0;
    J->unit_begin = 0;
    return GRT_OK;
}

// Keeps freed ray buffers in the device's stream-ordered pool between calls.
void keep_pool_memory() {
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// Lays out the jobs' rays and accumulation units, then runs the three kernels.
template <bool COUNT, int CAP>
int run_jobs(JobTable<CAP>& T, int k, long long* counters, cudaStream_t st) {
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
    keep_pool_memory();
    float4* buf = nullptr;
    GRT_CUDA(cudaMallocAsync((void**)&buf, sizeof(float4) * (2 * (size_t)rays + 1), st));
    float4* dirs = buf;
    float4* res = buf + rays;
    unsigned long long* next_ray = reinterpret_cast<unsigned long long*>(buf + 2 * rays);
    const long long gr = (rays + kShadeThreads - 1) / kShadeThreads;
    k_sample_rays<CAP><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs);
    dispatch_k(k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if (COUNT) {  // counting pass: one ray per thread, same traversal
            k_trace_rays<K, COUNT, CAP><<<(unsigned)gr, kShadeThreads, 0, st>>>(T, dirs, res, counters);
        } else {
            cudaMemsetAsync(next_ray, 0, sizeof(unsigned long long), st);
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_rays_dyn<K, CAP>, kShadeThreads, 0);
            long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
            if (grid > gr) grid = gr;
            k_trace_rays_dyn<K, CAP><<<(unsigned)grid, kShadeThreads, 0, st>>>(T, dirs, res, next_ray);
        }
    });
    if (!COUNT) {
        const long long ga = (units * 32 + kShadeThreads - 1) / kShadeThreads;
        k_accumulate<CAP><<<(unsigned)ga, kShadeThreads, 0, st>>>(T, dirs, res);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return check_cuda(e, "shade kernels");
    return GRT_OK;
}

template <bool COUNT>
int launch_single(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const grt_gbuffer* g,
                  const grt_envmap* e, const grt_sampling* smp, const int* pl, int n, float* oc, float* ov, float* oi,
                  long long* counters, cudaStream_t st) {
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
    return run_jobs<COUNT>(T, p->k, counters, st);
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
    (void)work_counter;
    int rc = check_params(p);
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
        if (J.n_pixels == 0) {
            if (req[i].n_pixels > 0)
                k_zero_outputs<<<(req[i].n_pixels + 255) / 256, 256, 0, st>>>(req[i].out_color, req[i].out_vis,
                                                                              req[i].out_ind, req[i].n_pixels);
            continue;
        }
        T.job[T.n_jobs++] = J;
    }
    if (T.n_jobs == 0) return launch_error("k_zero_outputs");
    return run_jobs<false>(T, p->k, nullptr, st);
}
