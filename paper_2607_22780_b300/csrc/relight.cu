// relight.cu -- grt_env_prefilter (the prefiltered novel map E of Eq. 15) and grt_trace_attr
// (Trace_attr of Eq. 14 for a flat list of rays).  Definitions in relight.cuh.
//
// Prefiltering is a set of exact texel quadratures: one block per output cell, its threads
// striding over the map's texels (centre direction and solid angle precomputed once), a
// block reduction at the end.  The split-sum BRDF table does not depend on the map; it is
// computed per call (1024 cells x 65,536 half-vector samples, well under a millisecond).
#include "common_args.cuh"
#include "relight.cuh"
#include "trace.cuh"

namespace grt {
namespace {

constexpr int kPrefThreads = 256;

// Sum of v over the block (result valid in thread 0).
template <int N>
__device__ __forceinline__ void block_sum(float (&v)[N], float (*sh)[kPrefThreads / 32]) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            float x = 0.f;
            for (int w = 0; w < kPrefThreads / 32; ++w) x += sh[k][w];
            v[k] = x;
        }
    }
}

// Texel centre direction (xyz) and solid angle (w) of the novel map.
__global__ void k_texel_dirs(int W, int H, float4* __restrict__ td) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * H) return;
    const int row = t / W, col = t % W;
    const f3 d = grid_dir(row, col, W, H);
    const float dw = (2.f * kPi / (float)W) * (cospif((float)row / (float)H) - cospif((float)(row + 1) / (float)H));
    td[t] = make_float4(d.x, d.y, d.z, dw);
}

__global__ void __launch_bounds__(kPrefThreads) k_pref_diff(const float* __restrict__ rgb, const float4* __restrict__ td,
                                                            int n, float* __restrict__ diff) {
    __shared__ float sh[3][kPrefThreads / 32];
    const int g = blockIdx.x;
    const f3 nn = grid_dir(g / kDiffW, g % kDiffW, kDiffW, kDiffH);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < n; t += kPrefThreads) {
        const float4 d = __ldg(td + t);
        const float c = nn.x * d.x + nn.y * d.y + nn.z * d.z;
        if (c <= 0.f) continue;
        const float w = c * d.w;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(__ldg(rgb + 3 * (size_t)t + ch), w, acc[ch]);
    }
    block_sum(acc, sh);
    if (threadIdx.x == 0)
        for (int ch = 0; ch < 3; ++ch) diff[3 * g + ch] = acc[ch] * kInvPi;
}

__global__ void __launch_bounds__(kPrefThreads) k_pref_spec(const float* __restrict__ rgb, const float4* __restrict__ td,
                                                            int n, float* __restrict__ spec) {
    __shared__ float sh[4][kPrefThreads / 32];
    const int g = blockIdx.x;
    const int lev = 1 + g / (kSpecW * kSpecH), cell = g % (kSpecW * kSpecH);
    const float a2 = ggx_alpha2((float)lev / (float)(kSpecLevels - 1));
    const f3 R = grid_dir(cell / kSpecW, cell % kSpecW, kSpecW, kSpecH);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < n; t += kPrefThreads) {
        const float4 d = __ldg(td + t);
        const float c = R.x * d.x + R.y * d.y + R.z * d.z;
        if (c <= 0.f) continue;
        f3 h = mk3(d.x + R.x, d.y + R.y, d.z + R.z);
        const float il = rsqrtf(dot3(h, h));
        h = mk3(h.x * il, h.y * il, h.z * il);
        const float w = ggx_D(h, R, dot3(h, R), a2) * c * d.w;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(__ldg(rgb + 3 * (size_t)t + ch), w, acc[ch]);
        acc[3] += w;
    }
    block_sum(acc, sh);
    if (threadIdx.x == 0)
        for (int ch = 0; ch < 3; ++ch) spec[3 * (size_t)g + ch] = acc[3] > 0.f ? acc[ch] / acc[3] : 0.f;
}

// Split-sum BRDF table: A, B = E over GGX half vectors of G1(v) G1(l) (v.h)/(n.v n.h) times
// (1 - (1-v.h)^5) and (1-v.h)^5, midpoint rule on a kLutM x kLutM grid of (u1, u2).
__global__ void __launch_bounds__(kPrefThreads) k_brdf_lut(float* __restrict__ lut) {
    __shared__ float sh[2][kPrefThreads / 32];
    const int i = blockIdx.x / kLutN, j = blockIdx.x % kLutN;
    const float nv = ((float)i + 0.5f) / (float)kLutN;
    const float a = fmaxf(((float)j + 0.5f) / (float)kLutN * (((float)j + 0.5f) / (float)kLutN), 1e-4f);
    const float a2 = a * a;
    const f3 v = mk3(sqrtf(1.f - nv * nv), 0.f, nv);
    const float g1v = ggx_G1(nv, a2);
    float acc[2] = {0.f, 0.f};
    for (int s = threadIdx.x; s < kLutM * kLutM; s += kPrefThreads) {
        const float u1 = ((float)(s / kLutM) + 0.5f) / (float)kLutM, u2 = ((float)(s % kLutM) + 0.5f) / (float)kLutM;
        const float th = atanf(a * sqrtf(u1 / (1.f - u1)));
        float st, ct, sp, cp;
        sincosf(th, &st, &ct);
        sincospif(2.f * u2, &sp, &cp);
        const f3 h = mk3(st * cp, st * sp, ct);
        const float vh = dot3(v, h);
        if (vh <= 0.f) continue;
        const float lz = 2.f * vh * h.z - v.z;
        if (lz <= 0.f) continue;
        const float Gv = g1v * ggx_G1(lz, a2) * vh / (nv * h.z);
        const float x = 1.f - vh, x5 = x * x * x * x * x;
        acc[0] = fmaf(Gv, 1.f - x5, acc[0]);
        acc[1] = fmaf(Gv, x5, acc[1]);
    }
    block_sum(acc, sh);
    if (threadIdx.x == 0) {
        const float inv = 1.f / (float)(kLutM * kLutM);
        lut[2 * blockIdx.x] = acc[0] * inv;
        lut[2 * blockIdx.x + 1] = acc[1] * inv;
    }
}

// Means of the top (block 0) and bottom (block 1) rows of an rgb grid [H][W][3].
__global__ void __launch_bounds__(kPrefThreads) k_row_means(const float* __restrict__ g, int W, int H,
                                                            float* __restrict__ out) {
    __shared__ float sh[3][kPrefThreads / 32];
    const float* row = g + 3 * (size_t)(blockIdx.x == 0 ? 0 : H - 1) * W;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int i = threadIdx.x; i < W; i += kPrefThreads)
        for (int ch = 0; ch < 3; ++ch) acc[ch] += __ldg(row + 3 * i + ch);
    block_sum(acc, sh);
    if (threadIdx.x == 0)
        for (int ch = 0; ch < 3; ++ch) out[3 * blockIdx.x + ch] = acc[ch] / (float)W;
}

// Trace_attr over a flat ray list (ray mode), in the persistent two-phase walk.
struct AttrOut {
    float *vis, *albedo, *rough, *metal, *normal;
};

template <int K>
struct RayAttrTask {
    using Visitor = AttrVisitor;
    const DevBvh* bvh;
    const TraceParams* P;
    const AttrSrc* src;
    const float *ro, *rd;
    AttrOut out;
    __device__ __forceinline__ bool begin(long long r, WalkState<K>& ts, Visitor& v, const DevBvh*& b) {
        const f3 o = mk3(__ldg(ro + 3 * r), __ldg(ro + 3 * r + 1), __ldg(ro + 3 * r + 2));
        const f3 d = mk3(__ldg(rd + 3 * r), __ldg(rd + 3 * r + 1), __ldg(rd + 3 * r + 2));
        trace_begin(*bvh, ts, o, d, *P);
        v = AttrVisitor(src, d);
        b = bvh;
        return true;
    }
    __device__ __forceinline__ void end(long long r, const WalkState<K>& ts, Visitor& v) {
        v.resolve();
        out.vis[r] = ts.T;
        out.rough[r] = v.r;
        out.metal[r] = v.m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out.albedo[3 * r + k] = v.a[k];
            out.normal[3 * r + k] = v.n[k];
        }
    }
};

template <int K>
__global__ void __launch_bounds__(128, K >= 32 ? 3 : GRT_TRACE_MIN_BLOCKS) k_trace_attr(DevBvh bvh, TraceParams P, AttrSrc src,
                                                                     const float* __restrict__ ro,
                                                                     const float* __restrict__ rd, long long R,
                                                                     AttrOut out, unsigned long long* next) {
    __shared__ int q[kQueue * 128];
    RayAttrTask<K> task{&bvh, &P, &src, ro, rd, out};
    persistent_trace<K>(task, P, next, R, q + threadIdx.x, 128);
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" size_t grt_env_prefilter_bytes(void) { return sizeof(float) * pref_layout().total; }

extern "C" int grt_env_prefilter(const float* rgb, int32_t W, int32_t H, void* out, size_t out_bytes, void* stream) {
    if (!rgb || !out) return set_error(GRT_ERR_ARG, "rgb and out must be non-NULL");
    if (W <= 0 || H <= 0 || (long long)W * H > (1LL << 28)) return set_error(GRT_ERR_ARG, "bad map size %dx%d", W, H);
    if ((uintptr_t)out & 15) return set_error(GRT_ERR_ARG, "out must be 16-byte aligned");
    if (out_bytes < grt_env_prefilter_bytes())
        return set_error(GRT_ERR_ARG, "out holds %zu bytes, %zu needed", out_bytes, grt_env_prefilter_bytes());
    cudaStream_t st = (cudaStream_t)stream;
    const int n = W * H;
    float4* td = nullptr;
    GRT_CUDA(cudaMallocAsync((void**)&td, sizeof(float4) * (size_t)n, st));
    const PrefLayout L = pref_layout();
    float* f = static_cast<float*>(out);
    k_texel_dirs<<<(n + 255) / 256, 256, 0, st>>>(W, H, td);
    k_pref_diff<<<kDiffW * kDiffH, kPrefThreads, 0, st>>>(rgb, td, n, f + L.diff);
    k_pref_spec<<<(kSpecLevels - 1) * kSpecW * kSpecH, kPrefThreads, 0, st>>>(rgb, td, n, f + L.spec);
    k_brdf_lut<<<kLutN * kLutN, kPrefThreads, 0, st>>>(f + L.lut);
    k_row_means<<<2, kPrefThreads, 0, st>>>(f + L.diff, kDiffW, kDiffH, f + L.poles);
    for (int l = 1; l < kSpecLevels; ++l)
        k_row_means<<<2, kPrefThreads, 0, st>>>(f + L.spec + 3 * (size_t)(l - 1) * kSpecW * kSpecH, kSpecW, kSpecH,
                                                f + L.poles + 6 * l);
    k_row_means<<<2, kPrefThreads, 0, st>>>(rgb, W, H, f + L.poles + 6 * kSpecLevels);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(td, st);
    if (e != cudaSuccess) return check_cuda(e, "prefilter kernels");
    return GRT_OK;
}

extern "C" int grt_trace_attr(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p, const float* ray_o,
                              const float* ray_d, int32_t R, float* out_vis, float* out_albedo, float* out_rough,
                              float* out_metal, float* out_normal, void* stream) {
    int rc = check_trace_inputs(b, s, p);
    if (rc) return rc;
    if (R < 0) return set_error(GRT_ERR_ARG, "R < 0");
    if (R == 0) return GRT_OK;
    if (!ray_o || !ray_d || !out_vis || !out_albedo || !out_rough || !out_metal || !out_normal)
        return set_error(GRT_ERR_ARG, "rays and every output must be non-NULL");
    if (s->n > 0 && (!s->albedo || !s->rough || !s->metal))
        return set_error(GRT_ERR_ARG, "surfels need albedo, rough and metal for Trace_attr");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* next = nullptr;
    GRT_CUDA(cudaMallocAsync((void**)&next, sizeof(unsigned long long), st));
    GRT_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned long long), st));
    DevBvh bvh = dev_bvh(b);
    TraceParams P = to_params(*p);
    AttrSrc src{b->normals, s->albedo, s->rough, s->metal};
    AttrOut out{out_vis, out_albedo, out_rough, out_metal, out_normal};
    const long long gmax = (R + 127) / 128;
    dispatch_k(p->k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr size_t smem = walk_smem_bytes<K>();
        const long long grid = persistent_grid(k_trace_attr<K>, smem, gmax);
        k_trace_attr<K><<<(unsigned)grid, 128, smem, st>>>(bvh, P, src, ray_o, ray_d, R, out, next);
    });
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(next, st);
    if (e != cudaSuccess) return check_cuda(e, "k_trace_attr");
    return GRT_OK;
}
