// gbuffer.cu -- primary G-buffer (Eq. 9) traced along pinhole camera rays.
//
// The paper rasterises {C, D, N, A, R, M} with normalised blending weights
// w_i = T_i a_i / sum_j T_j a_j (Sec. III-C).  Here the same weights come from the traced
// front-to-back sequence of the camera ray, which keeps the G-buffer consistent with the
// secondary trace (the paper notes the small raster/trace mismatch of tile sorting).
#include "common_args.cuh"

namespace grt {
namespace {

struct Camera {
    float v[10];  // eye xyz, target xyz, up xyz, tan(fovy/2)
};

// Decision computation of the primary ray through the centre of pixel (px, py).
__device__ __forceinline__ void camera_ray_d(const Camera& c, int W, int H, int px, int py, f3* o, f3* d) {
    f3 eye = mk3(c.v[0], c.v[1], c.v[2]);
    f3 fwd = norm_d(mk3(sub_d(c.v[3], c.v[0]), sub_d(c.v[4], c.v[1]), sub_d(c.v[5], c.v[2])));
    f3 up = mk3(c.v[6], c.v[7], c.v[8]);
    f3 right = norm_d(mk3(sub_d(mul_d(fwd.y, up.z), mul_d(fwd.z, up.y)), sub_d(mul_d(fwd.z, up.x), mul_d(fwd.x, up.z)),
                          sub_d(mul_d(fwd.x, up.y), mul_d(fwd.y, up.x))));
    f3 up2 = mk3(sub_d(mul_d(right.y, fwd.z), mul_d(right.z, fwd.y)),
                 sub_d(mul_d(right.z, fwd.x), mul_d(right.x, fwd.z)),
                 sub_d(mul_d(right.x, fwd.y), mul_d(right.y, fwd.x)));
    float th = c.v[9];
    float aspect = div_d((float)W, (float)H);
    float sx = mul_d(mul_d(sub_d(div_d(mul_d(2.0f, add_d((float)px, 0.5f)), (float)W), 1.0f), th), aspect);
    float sy = mul_d(sub_d(1.0f, div_d(mul_d(2.0f, add_d((float)py, 0.5f)), (float)H)), th);
    f3 dd = mk3(add_d(add_d(fwd.x, mul_d(sx, right.x)), mul_d(sy, up2.x)),
                add_d(add_d(fwd.y, mul_d(sx, right.y)), mul_d(sy, up2.y)),
                add_d(add_d(fwd.z, mul_d(sx, right.z)), mul_d(sy, up2.z)));
    *o = eye;
    *d = norm_d(dd);
}

struct GbufVisitor {
    const float4* nrm;  // the tree's decision normals (R(q/|q|) third column, by surfel id)
    const float *albedo, *rough, *metal;
    f3 d;
    float D, wsum, nx, ny, nz, ar, ag, ab, ro, me, T;
    __device__ __forceinline__ GbufVisitor() {}
    __device__ __forceinline__ GbufVisitor(const grt_surfels& s, const float4* normals, f3 dir)
        : nrm(normals), albedo(s.albedo), rough(s.rough), metal(s.metal), d(dir), D(0), wsum(0), nx(0), ny(0), nz(0),
          ar(0), ag(0), ab(0), ro(0), me(0), T(1) {}
    __device__ __forceinline__ void composite(int, int id, float tau, float alpha, float Tb) {
        float w = Tb * alpha;
        const float4 nv = __ldg(nrm + id);
        const f3 n = mk3(nv.x, nv.y, nv.z);
        float sgn = dot_d(n, d) > 0.f ? -1.f : 1.f;  // face the camera
        D = fmaf(w, tau, D);
        nx = fmaf(w * sgn, n.x, nx);
        ny = fmaf(w * sgn, n.y, ny);
        nz = fmaf(w * sgn, n.z, nz);
        ar = fmaf(w, __ldg(albedo + 3 * (size_t)id), ar);
        ag = fmaf(w, __ldg(albedo + 3 * (size_t)id + 1), ag);
        ab = fmaf(w, __ldg(albedo + 3 * (size_t)id + 2), ab);
        ro = fmaf(w, __ldg(rough + id), ro);
        me = fmaf(w, __ldg(metal + id), me);
        wsum += w;
    }
    __device__ __forceinline__ void finish(float Tf) { T = Tf; }
};

struct GbufOut {
    float *pos, *normal, *albedo, *rough, *metal, *alpha, *depth;
    int* valid;
};

// Primary rays in the persistent two-phase walk: ray index = pixel y*W + x.
template <int K>
struct GbufTask {
    using Visitor = GbufVisitor;
    const DevBvh* bvh;
    const grt_surfels* s;
    const Camera* cam;
    const TraceParams* P;
    int W, H;
    GbufOut out;
    __device__ __forceinline__ bool begin(long long r, WalkState<K>& ts, Visitor& v, const DevBvh*& b) {
        f3 o, d;
        camera_ray_d(*cam, W, H, (int)(r % W), (int)(r / W), &o, &d);
        trace_begin(*bvh, ts, o, d, *P);
        v = GbufVisitor(*s, bvh->normals, d);
        b = bvh;
        return true;
    }
    __device__ __forceinline__ void end(long long r, const WalkState<K>& ts, Visitor& v) {
        const size_t p = (size_t)r;
        const f3 o = ts.r.o, d = ts.r.d;
        float a = 1.f - v.T;
        float nl = sqrtf(v.nx * v.nx + v.ny * v.ny + v.nz * v.nz);
        bool ok = a >= 0.5f && nl > 1e-12f;
        out.valid[p] = ok;
        if (out.alpha) out.alpha[p] = a;
        float iw = ok ? 1.f / v.wsum : 0.f;
        float D = v.D * iw;
        if (out.depth) out.depth[p] = D;
        out.pos[3 * p] = ok ? fmaf(D, d.x, o.x) : 0.f;
        out.pos[3 * p + 1] = ok ? fmaf(D, d.y, o.y) : 0.f;
        out.pos[3 * p + 2] = ok ? fmaf(D, d.z, o.z) : 0.f;
        float in = ok ? 1.f / nl : 0.f;
        out.normal[3 * p] = v.nx * in;
        out.normal[3 * p + 1] = v.ny * in;
        out.normal[3 * p + 2] = v.nz * in;
        out.albedo[3 * p] = v.ar * iw;
        out.albedo[3 * p + 1] = v.ag * iw;
        out.albedo[3 * p + 2] = v.ab * iw;
        out.rough[p] = v.ro * iw;
        out.metal[p] = v.me * iw;
    }
};

template <int K>
__global__ void __launch_bounds__(128, K >= 32 ? 3 : GRT_TRACE_MIN_BLOCKS) k_gbuffer(DevBvh bvh, TraceParams P, grt_surfels s, Camera cam,
                                                                  int W, int H, GbufOut out,
                                                                  unsigned long long* next) {
    __shared__ int q[kQueue * 128];
    GbufTask<K> task{&bvh, &s, &cam, &P, W, H, out};
    persistent_trace<K>(task, P, next, (long long)W * H, q + threadIdx.x, 128);
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_gbuffer_primary(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p,
                                   const float camera[10], int32_t W, int32_t H, float* pos, float* normal,
                                   float* albedo, float* rough, float* metal, float* alpha, float* depth,
                                   int32_t* valid, void* stream) {
    if (!b || !s) return set_error(GRT_ERR_ARG, "bvh or surfels is NULL");
    if (s->n != b->n) return set_error(GRT_ERR_ARG, "surfels->n = %d but the BVH holds %d", s->n, b->n);
    int rc = check_params(p);
    if (rc) return rc;
    if (!camera) return set_error(GRT_ERR_ARG, "camera is NULL");
    if (W <= 0 || H <= 0 || (long long)W * H > (1LL << 30)) return set_error(GRT_ERR_ARG, "bad image size %dx%d", W, H);
    if (!pos || !normal || !albedo || !rough || !metal || !valid)
        return set_error(GRT_ERR_ARG, "pos, normal, albedo, rough, metal and valid must be non-NULL");
    if (s->n > 0 && (!s->albedo || !s->rough || !s->metal))
        return set_error(GRT_ERR_ARG, "surfels need albedo, rough and metal for the G-buffer");
    Camera cam;
    for (int i = 0; i < 10; ++i) cam.v[i] = camera[i];
    DevBvh bvh = dev_bvh(b);
    TraceParams P = to_params(*p);
    GbufOut out{pos, normal, albedo, rough, metal, alpha, depth, valid};
    int n = W * H, gmax = (n + 127) / 128;
    cudaStream_t st = (cudaStream_t)stream;
    grt_surfels sc = *s;
    unsigned long long* next = nullptr;
    GRT_CUDA(cudaMallocAsync((void**)&next, sizeof(unsigned long long), st));
    GRT_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned long long), st));
    // a frame too small to fill the device is bound by its slowest warps: fewer rounds
    const int k = p->gbuffer_k ? p->gbuffer_k : ((long long)W * H <= GRT_GBUFFER_SMALL_FRAME ? 32 : p->k);
    dispatch_k(k, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr size_t smem = walk_smem_bytes<K>();
        const long long grid = persistent_grid(k_gbuffer<K>, smem, gmax);
        k_gbuffer<K><<<(unsigned)grid, 128, smem, st>>>(bvh, P, sc, cam, W, H, out, next);
    });
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(next, st);
    if (e != cudaSuccess) return check_cuda(e, "k_gbuffer");
    return GRT_OK;
}
