// trace.cu -- grt_trace_forward / grt_trace_count: the Trace operator of Eq. 8 on rays.
#include "common_args.cuh"

namespace grt {
namespace {

constexpr int kTraceThreads = 128;

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

template <int K, bool COUNT>
__global__ void __launch_bounds__(kTraceThreads) k_trace_forward(DevBvh bvh, TraceParams P, const float* __restrict__ color,
                                                                 int cdim, const float* __restrict__ ro,
                                                                 const float* __restrict__ rd, int R, float* out_rgb,
                                                                 float* out_op, int* hits, int max_hits, int* nhits,
                                                                 long long* counters) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    Counters cnt{0, 0, 0};
    if (i < R) {
        f3 o = mk3(ro[3 * (size_t)i], ro[3 * (size_t)i + 1], ro[3 * (size_t)i + 2]);
        f3 d = mk3(rd[3 * (size_t)i], rd[3 * (size_t)i + 1], rd[3 * (size_t)i + 2]);
        RayState r = make_ray(o, d);
        int* h = hits ? hits + (size_t)i * max_hits : nullptr;
        ColourVisitor v(color, cdim, d, h, max_hits);
        trace_ray<K, COUNT>(bvh, r, P, v, cnt);
        if (out_rgb) {
            out_rgb[3 * (size_t)i] = v.c[0];
            out_rgb[3 * (size_t)i + 1] = v.c[1];
            out_rgb[3 * (size_t)i + 2] = v.c[2];
        }
        if (out_op) out_op[i] = 1.f - v.T;
        if (h)
            for (int k = v.nh; k < max_hits; ++k) h[k] = -1;
        if (nhits) nhits[i] = v.nh;
    }
    if (COUNT) flush_counters(cnt, counters);
}

template <bool COUNT>
int launch_trace(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const float* ro, const float* rd,
                 int R, float* out_rgb, float* out_op, int* hits, int max_hits, int* nhits, long long* counters,
                 cudaStream_t st) {
    if (R == 0) return GRT_OK;
    DevBvh bvh = dev_bvh(b);
    TraceParams P = to_params(*p);
    int grid = (R + kTraceThreads - 1) / kTraceThreads;
    dispatch_k(p->k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        k_trace_forward<K, COUNT><<<grid, kTraceThreads, 0, st>>>(bvh, P, s->color, s->color_dim, ro, rd, R, out_rgb,
                                                                  out_op, hits, max_hits, nhits, counters);
    });
    return launch_error("k_trace_forward");
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_trace_forward(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const float* ray_o,
                                 const float* ray_d, int32_t R, float* out_rgb, float* out_opacity, int32_t* out_hits,
                                 int32_t max_hits, int32_t* out_nhits, void* stream) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    if (R < 0) return set_error(GRT_ERR_ARG, "R = %d < 0", R);
    if (R > 0 && (!ray_o || !ray_d || !out_rgb || !out_opacity))
        return set_error(GRT_ERR_ARG, "ray_o, ray_d, out_rgb and out_opacity must be non-NULL");
    if (out_hits && max_hits <= 0) return set_error(GRT_ERR_ARG, "out_hits needs max_hits > 0");
    return launch_trace<false>(b, s, p, ray_o, ray_d, R, out_rgb, out_opacity, out_hits, out_hits ? max_hits : 0,
                               out_nhits, nullptr, (cudaStream_t)stream);
}

extern "C" int grt_trace_count(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const float* ray_o,
                               const float* ray_d, int32_t R, long long* counters, void* stream) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    if (R < 0 || (R > 0 && (!ray_o || !ray_d)) || !counters) return set_error(GRT_ERR_ARG, "bad rays or counters");
    return launch_trace<true>(b, s, p, ray_o, ray_d, R, nullptr, nullptr, nullptr, 0, nullptr, counters,
                              (cudaStream_t)stream);
}
