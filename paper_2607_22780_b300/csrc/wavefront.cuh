// wavefront.cuh -- pieces shared by the wavefront shading and shading-adjoint passes:
// the job table (one or many shading requests laid out as one flat list of rays), the
// ray-sampling kernel and the persistent per-ray trace kernel.
#pragma once

#include <mutex>

#include "common_args.cuh"
#include "mesh.cuh"
#include "relight.cuh"
#include "shade.cuh"

namespace grt {

constexpr int kShadeThreads = 128;
static_assert(kShadeThreads == kPersistentThreads, "persistent kernels index shared memory by 128 lanes");

struct ShadeJob {
    DevBvh bvh;
    const float* color;
    const float *mu, *quat, *scale, *opacity;  // surfel parameters (adjoint pass)
    AttrSrc attr;                              // surfel materials (relighting pass)
    int cdim;
    GbufDev gb;
    EnvDev env;
    Sampling S;
    const int* pixel_list;
    int n_pixels;
    int pixel_offset;        // with no pixel list: pixel = pixel_offset + list index
    int Nr;
    float *out_color, *out_vis, *out_ind;
    float* out_light;        // optional mean incident radiance (Eq. 16)
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
    int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
    if ((unsigned)pix >= (unsigned)(J.gb.W * J.gb.H)) {
        atomicOr(J.bvh.status, GRT_STATUS_BAD_INDEX);
        return -1;
    }
    return pix;
}

// ---- coherent ray order for the persistent walk
// Rays are handed to the walk bucket by bucket: a bucket holds the rays leaving one screen
// tile (Morton order of 2^kTileBits x 2^kTileBits tiles) in one direction cell (octahedral
// map of d, 2^kDirBits x 2^kDirBits cells), so the 32 lanes of a warp start from nearby
// points in similar directions and visit the same nodes.  The order only schedules the
// walk: every ray computes the same result.  The sampler writes each slot's bucket and
// its rank in the bucket (one warp-aggregated atomic per distinct bucket in a warp); a scan
// of the bucket counts and an atomic-free scatter give the order; 12 bytes of pool scratch
// per ray slot.  Measured on the 300k-surfel 800x800 workload (M rays/s, whole step): slot
// order 395; buckets of 32x32 tiles x 8x8 direction cells 416.6, 64x64 x 4x4 416.1,
// 16x16 x 16x16 415.8, 32x32 x 16x16 416.5, 64x64 x 8x8 416.0; direction-major keys
// 401 (the same buckets in another order); the walk itself 20.8 -> 18.85 ms.  On the current
// walk, with the tiled bucket scan: 32x32 tiles x 8x8 / 16x16 / 32x32 direction cells: walk
// 11.31 / 11.18 / 11.06 ms, sampling phase 0.52 / 0.53 / 0.55 ms, step 14.27 / 14.14 / 14.07
// ms; 16x16 tiles x 32x32 cells: 14.17 ms (2^20 buckets: 4 MB of counters per call).
#ifndef GRT_RAY_ORDER
#define GRT_RAY_ORDER 1
#endif
#ifndef GRT_ORDER_TILE_BITS
#define GRT_ORDER_TILE_BITS 5
#endif
#ifndef GRT_ORDER_DIR_BITS
#define GRT_ORDER_DIR_BITS 5
#endif
constexpr int kTileBits = GRT_ORDER_TILE_BITS, kDirBits = GRT_ORDER_DIR_BITS;
// Launches with fewer ray slots keep the slot order: their walk is bound by the latency of
// their longest ray, and sorting them cost more than it saved (the 64x64 frame of 7,400
// rays: bucket scan 54 us against a 265 us walk).
constexpr long long kOrderMinRays = 1ll << 16;
inline bool use_ray_order(long long rays) { return GRT_RAY_ORDER && rays >= kOrderMinRays && rays <= 0xFFFFFFFFLL; }
constexpr unsigned kRayBuckets = 1u << (2 * (kTileBits + kDirBits));
// slots without a ray go last, spread over kEmptyBuckets buckets by slot group so that
// their counting does not serialise on one address
constexpr unsigned kEmptyBuckets = 1024;
constexpr unsigned kAllBuckets = kRayBuckets + kEmptyBuckets;

__device__ __forceinline__ unsigned spread2(unsigned x) {
    x &= 0xFF;
    x = (x | (x << 4)) & 0x0F0F;
    x = (x | (x << 2)) & 0x3333;
    x = (x | (x << 1)) & 0x5555;
    return x;
}

// Bucket of a ray: 2^tb x 2^tb screen tiles (Morton order) x 2^db x 2^db octahedral
// direction cells, offset by `base`.
__device__ __forceinline__ unsigned ray_bucket(const GbufDev& g, int pix, float4 dw, long long r, int tb, int db,
                                               unsigned base) {
    if (dw.w == 0.f) return kRayBuckets + (unsigned)((r >> 5) & (kEmptyBuckets - 1));
    const int px = pix % g.W, py = pix / g.W;
    const int m = (g.W > g.H ? g.W : g.H) - 1;
    int sh = 0;
    while ((m >> sh) >= (1 << tb)) ++sh;
    const unsigned tile = spread2((unsigned)(px >> sh)) | (spread2((unsigned)(py >> sh)) << 1);
    const float l1 = fabsf(dw.x) + fabsf(dw.y) + fabsf(dw.z);
    float u = dw.x / l1, v = dw.y / l1;
    if (dw.z < 0.f) {
        const float uu = (1.f - fabsf(v)) * (u >= 0.f ? 1.f : -1.f);
        v = (1.f - fabsf(u)) * (v >= 0.f ? 1.f : -1.f);
        u = uu;
    }
    const int nd = 1 << db;
    const int cu = min(nd - 1, max(0, (int)((u + 1.f) * (0.5f * nd))));
    const int cv = min(nd - 1, max(0, (int)((v + 1.f) * (0.5f * nd))));
    return base | (tile << (2 * db)) | (unsigned)(cv * nd + cu);
}

// In a launch of several requests (scenes, cameras) the buckets are request-major, each
// request getting kJobBuckets of them (8 x 8 tiles x 4 x 4 direction cells), so that a warp's
// rays come from one request and walk one tree; a single request uses all kRayBuckets.
#ifndef GRT_BATCH_JOB_MAJOR
#define GRT_BATCH_JOB_MAJOR 1
#endif
constexpr int kJobTileBits = 3, kJobDirBits = 2;
constexpr unsigned kJobBuckets = 1u << (2 * (kJobTileBits + kJobDirBits));
static_assert(kJobBuckets * 64 <= kRayBuckets, "request-major buckets of up to 64 requests");

// The bucket scan works in tiles of kScanTile counters: tile sums, their scan, then each
// tile's scan from its offset.
constexpr int kScanTile = 4096;
constexpr unsigned kScanTiles = (kAllBuckets + kScanTile - 1) / kScanTile;
constexpr unsigned kScanTilesPad = (kScanTiles + 3) & ~3u;
static_assert(kScanTiles <= 1024, "the tile sums are scanned by one block of 1024 threads");

// Buffers of the ray order over n slots (order_scratch_bytes(n) bytes from `base`):
// hist[kAllBuckets] bucket counts, then exclusive offsets; the scan's tile sums; per slot
// its bucket, its rank in the bucket, and order[] = the slots bucket by bucket.
struct RayOrder {
    unsigned *hist, *tsum, *key, *rank, *order;
};
inline size_t order_scratch_bytes(long long n) { return 4 * (3 * (size_t)n + kAllBuckets + kScanTilesPad); }
inline RayOrder ray_order_bufs(void* base, long long n, unsigned* order = nullptr) {
    RayOrder o;
    o.hist = static_cast<unsigned*>(base);
    o.tsum = o.hist + kAllBuckets;
    o.key = o.tsum + kScanTilesPad;
    o.rank = o.key + n;
    o.order = order ? order : o.rank + n;
    return o;
}

#ifndef GRT_SAMPLE_REMAP
#define GRT_SAMPLE_REMAP 1
#endif
// ray buffer entry: (direction, 1) for a traced sample, (0, 0, 0, 0) for none; with an
// order (o.key != nullptr), also the slot's bucket and its rank among the bucket's slots
template <int CAP>
__global__ void __launch_bounds__(kShadeThreads) k_sample_rays(const __grid_constant__ JobTable<CAP> T,
                                                               float4* __restrict__ dirs,
                                                               RayOrder o = RayOrder{nullptr, nullptr, nullptr,
                                                                                     nullptr}) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T.total_rays) return;
    const int job = T.find_ray(t);
    const ShadeJob& J = T.job[job];
    long long lr = t - J.ray_begin;
#if GRT_SAMPLE_REMAP
    // thread -> slot: a complete group of 4 pixels (4 Nr slots, Nr a multiple of 8) is drawn
    // by warps of 4 pixels x 8 consecutive samples, so that a warp draws from one proposal
    // when the allocations are multiples of 8 (a pixel's 32 samples in one warp went three
    // ways: 17 of 32 lanes active); a slot's direction depends only on (pixel, j)
    if ((J.Nr & 7) == 0) {
        const long long g = lr / (4 * J.Nr);
        if ((g + 1) * 4 <= J.n_pixels) {
            const int u = (int)(lr - g * 4 * J.Nr);
            lr = g * 4 * J.Nr + (long long)(u & 3) * J.Nr + (((u >> 5) << 3) | ((u & 31) >> 2));
        }
    }
#endif
    const long long r = J.ray_begin + lr;
    int li = (int)(lr / J.Nr), j = (int)(lr - (long long)li * J.Nr);
    int pix = pixel_of(J, li);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pix >= 0 && __ldg(J.gb.valid + pix)) {
        PixelState ps = load_pixel(J.gb, pix);
        f3 w;
        if (draw_direction(J.S, J.env, ps, pix, j, &w)) out = make_float4(w.x, w.y, w.z, 1.f);
    }
    dirs[r] = out;
    if (o.key) {
        const unsigned key = (GRT_BATCH_JOB_MAJOR && T.n_jobs > 1)
                                 ? ray_bucket(J.gb, pix, out, r, kJobTileBits, kJobDirBits, (unsigned)job * kJobBuckets)
                                 : ray_bucket(J.gb, pix, out, r, kTileBits, kDirBits, 0u);
        // one atomic per distinct key in the warp; its old value ranks the warp's slots
        const unsigned peers = __match_any_sync(__activemask(), key);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(o.hist + key, (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        o.key[r] = key;
        o.rank[r] = base + (unsigned)__popc(peers & ((1u << lane) - 1u));
    }
}

// Exclusive scan of the n bucket counters in place, in three launches: the sum of each tile of
// kScanTile counters (coalesced loads), the exclusive scan of the tile sums (one block), and
// each tile's own scan from its offset.  The offsets are exact integer prefix sums, so the ray
// order is the same as a serial scan's.  (One block of 1,024 threads over all counters, each
// thread walking its own run, took 54 us for 2^16 buckets and 0.2 ms for 2^18.)
__global__ void __launch_bounds__(256) k_bucket_tile_sums(const unsigned* __restrict__ hist, int n,
                                                          unsigned* __restrict__ tsum) {
    __shared__ unsigned ws[8];
    const int base = blockIdx.x * kScanTile;
    unsigned s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += 256) {
        const int k = base + i;
        if (k < n) s += hist[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        tsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_bucket_tile_scan(unsigned* __restrict__ tsum, int tiles) {
    __shared__ unsigned sh[1024];
    const unsigned v = (int)threadIdx.x < tiles ? tsum[threadIdx.x] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned a = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0u;
        __syncthreads();
        sh[threadIdx.x] += a;
        __syncthreads();
    }
    if ((int)threadIdx.x < tiles) tsum[threadIdx.x] = sh[threadIdx.x] - v;
}

__global__ void __launch_bounds__(256) k_bucket_tile_apply(unsigned* __restrict__ hist, int n,
                                                           const unsigned* __restrict__ tsum) {
    constexpr int kPer = kScanTile / 256;
    __shared__ unsigned ws[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kPer;
    unsigned v[kPer];
    unsigned tot = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const unsigned c = base + k < n ? hist[base + k] : 0u;
        v[k] = tot;
        tot += c;
    }
    unsigned x = tot;  // inclusive scan of the thread totals over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    unsigned off = tsum[blockIdx.x] + x - tot;
    for (int w = 0; w < warp; ++w) off += ws[w];
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        if (base + k < n) hist[base + k] = off + v[k];
}

// order[offset of the slot's bucket + its rank] = slot (hist holds the exclusive offsets).
__global__ void k_ray_scatter(long long n, RayOrder o) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    o.order[__ldg(o.hist + o.key[r]) + o.rank[r]] = (unsigned)r;
}

// Bucket offsets and the order, after k_sample_rays has filled hist, key and rank.
inline void launch_ray_order(const RayOrder& o, long long n, cudaStream_t st) {
    k_bucket_tile_sums<<<kScanTiles, 256, 0, st>>>(o.hist, (int)kAllBuckets, o.tsum);
    k_bucket_tile_scan<<<1, 1024, 0, st>>>(o.tsum, (int)kScanTiles);
    k_bucket_tile_apply<<<kScanTiles, 256, 0, st>>>(o.hist, (int)kAllBuckets, o.tsum);
    k_ray_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, o);
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
            int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
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


__global__ void k_zero_outputs(float* c, float* v, float* i, int n) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    c[3 * (size_t)t] = c[3 * (size_t)t + 1] = c[3 * (size_t)t + 2] = 0.f;
    if (v) v[t] = 0.f;
    if (i) i[3 * (size_t)t] = i[3 * (size_t)t + 1] = i[3 * (size_t)t + 2] = 0.f;
}

inline int make_job(const grt_bvh* b, const grt_surfels* s, const grt_gbuffer* g, const grt_envmap* e,
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
    J->mu = s->mu;
    J->quat = s->quat;
    J->scale = s->scale;
    J->opacity = s->opacity;
    J->attr = AttrSrc{b->normals, s->albedo, s->rough, s->metal};
    J->cdim = s->color_dim;
    J->gb = GbufDev{g->pos, g->normal, g->albedo, g->rough, g->metal, g->valid, g->eye[0], g->eye[1], g->eye[2], g->W, g->H};
    EnvLayout l = env_layout(e->W, e->H);
    const char* tb = (const char*)e->tables;
    J->env = EnvDev{(const float4*)(tb + l.texel), (const float*)(tb + l.marg), (const float*)(tb + l.cond), e->W, e->H,
                    (float)e->W * (float)e->H / (2.f * kPi * kPi)};
    J->S = Sampling{smp->n_cos, smp->n_ggx, smp->n_env, smp->brdf, (uint32_t)(smp->seed & 0xFFFFFFFFu),
                    (uint32_t)(smp->seed >> 32)};
    J->pixel_list = pixel_list;
    J->pixel_offset = 0;
    J->n_pixels = Nr > 0 ? n_pixels : 0;
    J->Nr = Nr > 0 ? Nr : 1;
    J->out_color = oc;
    J->out_vis = ov;
    J->out_ind = oi;
    J->out_light = nullptr;
    J->G = group_lanes(J->Nr);
    J->spl = (J->Nr + J->G - 1) / J->G;
    J->ray_begin = 0;
    J->unit_begin = 0;
    return GRT_OK;
}

// Caller-supplied device workspace of a shading call (NULL: the stream-ordered pool).
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

inline int workspace_arg(void* ptr, size_t bytes, Workspace* out) {
    if (ptr && ((uintptr_t)ptr & 255)) return set_error(GRT_ERR_ARG, "workspace must be 256-byte aligned");
    out->ptr = ptr;
    out->bytes = ptr ? bytes : 0;
    return GRT_OK;
}

// Ray buffers of a shading call over n ray slots: direction and (c_rt, T) per slot, the
// walk's ray counter, then (with the ray order) bucket counters and 12 bytes per slot.
inline size_t shade_ws_bytes(long long n, bool ord) {
    return sizeof(float4) * (2 * (size_t)n + 1) + (ord ? order_scratch_bytes(n) : 0);
}

// Keeps freed ray buffers in the device's stream-ordered pool between calls.
inline void keep_pool_memory() {
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


// Shading rays: origin = G-buffer point of the ray's pixel, direction from k_sample_rays;
// result (c_rt, T) per ray, T = -1 for "no ray".
template <int K, int CAP>
struct ShadeTrace {
    using Visitor = RadianceVisitor;
    const JobTable<CAP>* T;
    const float4* dirs;
    float4* res;
    __device__ __forceinline__ bool begin(long long r, WalkState<K>& ts, Visitor& cv, const DevBvh*& bvh) {
        float4 dw = __ldg(dirs + r);
        if (dw.w == 0.f) {
            res[r] = make_float4(0.f, 0.f, 0.f, -1.f);
            return false;
        }
        const ShadeJob& J = T->job[T->find_ray(r)];
        int li = (int)((r - J.ray_begin) / J.Nr);
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        f3 o = mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
                   __ldg(J.gb.pos + 3 * (size_t)pix + 2));
        f3 d = mk3(dw.x, dw.y, dw.z);
        bvh = &J.bvh;
        trace_begin(J.bvh, ts, o, d, T->P);
        cv = RadianceVisitor(J.color, J.cdim, d);
        return true;
    }
    __device__ __forceinline__ void end(long long r, const WalkState<K>& ts, Visitor& cv) {
        res[r] = make_float4(cv.c[0], cv.c[1], cv.c[2], ts.T);
    }
};

template <int K, int CAP>
__global__ void __launch_bounds__(kShadeThreads, K >= 32 ? 3 : GRT_TRACE_MIN_BLOCKS) k_trace_rays_ww(
    const __grid_constant__ JobTable<CAP> T, const float4* __restrict__ dirs, float4* __restrict__ res,
    unsigned long long* __restrict__ next_ray, const unsigned* __restrict__ order) {
    __shared__ int q[kQueue * kShadeThreads];
    ShadeTrace<K, CAP> task{&T, dirs, res};
    persistent_trace<K>(task, T.P, next_ray, T.total_rays, q + threadIdx.x, kShadeThreads, order);
}


// Forward record kept for the backward pass (grt_shade_pixels_save): per ray the number
// of composited hits and, slot-major ([slot][ray], coalesced across a warp), the surfel id,
// tau and alpha of its first L hits in compositing order.  Rays with more than L hits
// continue in an overflow area: the first ov_cap of them (in the order they reach hit L)
// each take an overflow slot holding hits L .. L + kOverflowHits - 1 ([k - L][slot]), the
// ray of slot s in ov_ray[s], the slots handed out counted in *ov_count (zeroed before the
// forward).  A ray that found no slot free has kNoSlot set in its hit count.
constexpr int kOverflowHits = 192;
constexpr int kNoSlot = 1 << 30;

struct SavedHits {
    int* nh;
    int* ids;
    float* tau;
    float* alpha;
    long long R;
    int L;
    int* ov_ray;
    int* ov_ids;
    float* ov_tau;
    float* ov_alpha;
    unsigned* ov_count;
    int ov_cap;
    unsigned* order;  // the forward walk's ray order: record row p is ray order[p] (NULL: row = ray)
};

// Overflow slots of a record over R rays: one ray in 256, at least 64 (0 without a record).
inline int overflow_slots(long long R, int L) {
    if (L <= 0) return 0;
    long long c = R / 256;
    return (int)(c < 64 ? 64 : (c > (1ll << 24) ? (1ll << 24) : c));
}

// Layout of the caller's saved-forward buffer: ray directions and traced (c_rt, T) as in
// the shading pass, the persistent kernel's ray counter, then the hit record and its
// overflow area.
struct SavedLayout {
    size_t dirs, res, next, nh, ids, tau, alpha, ov_count, ov_ray, ov_ids, ov_tau, ov_alpha, order, total;
    int ov_cap;
    bool has_order;
};

inline SavedLayout saved_layout(long long R, int L) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    SavedLayout o;
    size_t off = 0;
    o.dirs = off;
    off = up(off + 16 * (size_t)R);
    o.res = off;
    off = up(off + 16 * (size_t)R);
    o.next = off;
    off = up(off + 8);
    o.nh = off;
    off = up(off + 4 * (size_t)R);
    o.ids = off;
    off = up(off + 4 * (size_t)L * R);
    o.tau = off;
    off = up(off + 4 * (size_t)L * R);
    o.alpha = off;
    off = up(off + 4 * (size_t)L * R);
    o.ov_cap = overflow_slots(R, L);
    const size_t oh = (size_t)kOverflowHits * o.ov_cap;
    o.ov_count = off;
    off = up(off + 8);
    o.ov_ray = off;
    off = up(off + 4 * (size_t)o.ov_cap);
    o.ov_ids = off;
    off = up(off + 4 * oh);
    o.ov_tau = off;
    off = up(off + 4 * oh);
    o.ov_alpha = off;
    off = up(off + 4 * oh);
    // the coherent order in which the forward walked the rays, kept for the replay
    o.has_order = L > 0 && use_ray_order(R);
    o.order = off;
    if (o.has_order) off = up(off + 4 * (size_t)R);
    o.total = off;
    return o;
}

inline SavedHits saved_hits(char* base, const SavedLayout& L, long long R, int max_hits) {
    return SavedHits{reinterpret_cast<int*>(base + L.nh),        reinterpret_cast<int*>(base + L.ids),
                     reinterpret_cast<float*>(base + L.tau),     reinterpret_cast<float*>(base + L.alpha),
                     R,                                          max_hits,
                     reinterpret_cast<int*>(base + L.ov_ray),    reinterpret_cast<int*>(base + L.ov_ids),
                     reinterpret_cast<float*>(base + L.ov_tau),  reinterpret_cast<float*>(base + L.ov_alpha),
                     reinterpret_cast<unsigned*>(base + L.ov_count), L.ov_cap,
                     L.has_order ? reinterpret_cast<unsigned*>(base + L.order) : nullptr};
}

// Caller-owned buffers of grt_shade_pixels_save / grt_shade_backward_saved.
struct SaveBufs {
    float4* dirs;
    float4* res;
    unsigned long long* next;
    SavedHits hits;
};

// The saved-forward buffer checked against the layout of this call's rays.
inline int saved_buffers(const void* saved, size_t saved_bytes, int32_t n_pixels, const grt_sampling* smp,
                         int32_t max_hits, SaveBufs* out) {
    size_t need = grt_shade_saved_bytes(n_pixels, smp, max_hits);
    if (need == 0) return GRT_ERR_ARG;
    if (!saved || ((uintptr_t)saved & 255))
        return set_error(GRT_ERR_ARG, "saved must be a 256-byte aligned device pointer");
    if (saved_bytes < need) return set_error(GRT_ERR_ARG, "saved buffer holds %zu bytes, %zu needed", saved_bytes, need);
    const long long R = (long long)n_pixels * (smp->n_cos + smp->n_ggx + smp->n_env);
    SavedLayout L = saved_layout(R, max_hits);
    char* base = (char*)saved;
    out->dirs = reinterpret_cast<float4*>(base + L.dirs);
    out->res = reinterpret_cast<float4*>(base + L.res);
    out->next = reinterpret_cast<unsigned long long*>(base + L.next);
    out->hits = saved_hits(base, L, R, max_hits);
    return GRT_OK;
}

// Radiance visitor that also writes the composited hits of its ray into the record: the
// first L in place, the next kOverflowHits in an overflow slot taken at hit L.
// The record's rows follow the walk order: hit k of the ray at walk position p sits at
// k * R + p, so that the lanes of a warp, which walk neighbouring positions, write (and the
// replay, taking positions in order, reads) neighbouring words.  Overflow slots name the
// position too; the ray's slot is order[p].
struct SavingVisitor : RadianceVisitor {
    const SavedHits* sv;
    long long r;  // the ray's position in the walk order (its record row)
    int slot;     // overflow slot, -1 until hit L (and when none was left)
    __device__ __forceinline__ SavingVisitor() {}
    __device__ __forceinline__ SavingVisitor(const float* col, int cd, f3 dir, const SavedHits* s, long long pos)
        : RadianceVisitor(col, cd, dir), sv(s), r(pos), slot(-1) {}
    __device__ __forceinline__ void composite(int k, int id, float tau, float alpha, float Tb) {
        RadianceVisitor::composite(k, id, tau, alpha, Tb);
        record(k, id, tau, alpha);
    }
    __device__ __forceinline__ void record(int k, int id, float tau, float alpha) {
        if (k < sv->L) {
            const size_t i = (size_t)k * sv->R + r;
            sv->ids[i] = id;
            sv->tau[i] = tau;
            sv->alpha[i] = alpha;
            return;
        }
        if (sv->L == 0) return;
        if (k == sv->L) {
            const unsigned s = atomicAdd(sv->ov_count, 1u);
            slot = s < (unsigned)sv->ov_cap ? (int)s : -1;
            if (slot >= 0) sv->ov_ray[slot] = (int)r;
        }
        if (slot >= 0 && k - sv->L < kOverflowHits) {
            const size_t i = (size_t)(k - sv->L) * sv->ov_cap + slot;
            sv->ov_ids[i] = id;
            sv->ov_tau[i] = tau;
            sv->ov_alpha[i] = alpha;
        }
    }
};

template <int K, int CAP>
struct ShadeTraceSave {
    using Visitor = SavingVisitor;
    const JobTable<CAP>* T;
    const float4* dirs;
    float4* res;
    const SavedHits* sv;
    long long pos = 0;  // walk position of the ray begin() takes (set by the walk)
    __device__ __forceinline__ bool begin(long long r, WalkState<K>& ts, Visitor& cv, const DevBvh*& bvh) {
        float4 dw = __ldg(dirs + r);
        if (dw.w == 0.f) {
            res[r] = make_float4(0.f, 0.f, 0.f, -1.f);
            sv->nh[r] = 0;
            return false;
        }
        const ShadeJob& J = T->job[T->find_ray(r)];
        int li = (int)((r - J.ray_begin) / J.Nr);
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        f3 o = mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
                   __ldg(J.gb.pos + 3 * (size_t)pix + 2));
        f3 d = mk3(dw.x, dw.y, dw.z);
        bvh = &J.bvh;
        trace_begin(J.bvh, ts, o, d, T->P);
        cv = SavingVisitor(J.color, J.cdim, d, sv, pos);
        return true;
    }
    __device__ __forceinline__ void end(long long r, const WalkState<K>& ts, Visitor& cv) {
        res[r] = make_float4(cv.c[0], cv.c[1], cv.c[2], ts.T);
        sv->nh[r] = ts.ncomp | (ts.ncomp > sv->L && cv.slot < 0 ? kNoSlot : 0);
    }
};

template <int K, int CAP>
__global__ void __launch_bounds__(kShadeThreads, K >= 32 ? 3 : GRT_TRACE_MIN_BLOCKS) k_trace_rays_save(
    const __grid_constant__ JobTable<CAP> T, const float4* __restrict__ dirs, float4* __restrict__ res,
    const __grid_constant__ SavedHits sv, unsigned long long* __restrict__ next_ray,
    const unsigned* __restrict__ order) {
    __shared__ int q[kQueue * kShadeThreads];
    ShadeTraceSave<K, CAP> task{&T, dirs, res, &sv};
    persistent_trace<K>(task, T.P, next_ray, T.total_rays, q + threadIdx.x, kShadeThreads, order);
}

// Relighting rays (Eq. 15): the same rays, but Trace_attr (Eq. 14) instead of Trace; the
// result (( 1 - V_r) SplitSum(a_r, r_r, m_r, n_r, E), V_r) takes the place of (c_rt, T), so
// the accumulation forms V L_new + (1 - V) SplitSum exactly as it forms V L_env + c_rt.
template <int K, int CAP>
struct ShadeTraceRelight {
    using Visitor = AttrVisitor;
    const JobTable<CAP>* T;
    const float4* dirs;
    float4* res;
    const RelightDev* E;
    __device__ __forceinline__ bool begin(long long r, WalkState<K>& ts, Visitor& v, const DevBvh*& bvh) {
        float4 dw = __ldg(dirs + r);
        if (dw.w == 0.f) {
            res[r] = make_float4(0.f, 0.f, 0.f, -1.f);
            return false;
        }
        const ShadeJob& J = T->job[T->find_ray(r)];
        int li = (int)((r - J.ray_begin) / J.Nr);
        int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
        f3 o = mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
                   __ldg(J.gb.pos + 3 * (size_t)pix + 2));
        f3 d = mk3(dw.x, dw.y, dw.z);
        bvh = &J.bvh;
        trace_begin(J.bvh, ts, o, d, T->P);
        v = AttrVisitor(&J.attr, d);
        return true;
    }
    __device__ __forceinline__ void end(long long r, const WalkState<K>& ts, Visitor& v) {
        const float V = ts.T;
        float ss[3] = {0.f, 0.f, 0.f};
        if (V < 1.f) {
            v.resolve();
            const ShadeJob& J = T->job[T->find_ray(r)];
            splitsum_d(*E, J.env, v.a, v.r, v.m, mk3(v.n[0], v.n[1], v.n[2]), mk3(-v.d.x, -v.d.y, -v.d.z), ss);
        }
        const float o = 1.f - V;
        res[r] = make_float4(o * ss[0], o * ss[1], o * ss[2], V);
    }
};

template <int K, int CAP>
__global__ void __launch_bounds__(kShadeThreads, K >= 32 ? 3 : GRT_TRACE_MIN_BLOCKS) k_trace_rays_relight(
    const __grid_constant__ JobTable<CAP> T, const float4* __restrict__ dirs, float4* __restrict__ res,
    const __grid_constant__ RelightDev E, unsigned long long* __restrict__ next_ray,
    const unsigned* __restrict__ order) {
    __shared__ int q[kQueue * kShadeThreads];
    ShadeTraceRelight<K, CAP> task{&T, dirs, res, &E};
    persistent_trace<K>(task, T.P, next_ray, T.total_rays, q + threadIdx.x, kShadeThreads, order);
}

template <int K, int CAP>
inline void launch_trace_relight(const JobTable<CAP>& T, const float4* dirs, float4* res, const RelightDev& E,
                                 unsigned long long* next_ray, long long blocks_max, cudaStream_t st,
                                 const unsigned* order = nullptr) {
    cudaMemsetAsync(next_ray, 0, sizeof(unsigned long long), st);
    constexpr size_t smem = walk_smem_bytes<K>();
    const long long grid = persistent_grid(k_trace_rays_relight<K, CAP>, smem, blocks_max);
    k_trace_rays_relight<K, CAP><<<(unsigned)grid, kShadeThreads, smem, st>>>(T, dirs, res, E, next_ray, order);
}

// Relighting rays with the mesh backend of Eq. 14: closest triangle hit, one thread per
// ray (in bucket order when given); res = (SplitSum of the hit, 0) or (0, 0, 0, 1) for a miss.
template <int CAP>
__global__ void __launch_bounds__(kShadeThreads) k_trace_rays_mesh(const __grid_constant__ JobTable<CAP> T,
                                                                   const float4* __restrict__ dirs,
                                                                   float4* __restrict__ res,
                                                                   const __grid_constant__ RelightDev E,
                                                                   const __grid_constant__ MeshDev M,
                                                                   const unsigned* __restrict__ order) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.total_rays) return;
    const long long r = order ? (long long)__ldg(order + i) : i;
    const float4 dw = __ldg(dirs + r);
    if (dw.w == 0.f) {
        res[r] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    const ShadeJob& J = T.job[T.find_ray(r)];
    const int li = (int)((r - J.ray_begin) / J.Nr);
    const int pix = J.pixel_list ? __ldg(J.pixel_list + li) : J.pixel_offset + li;
    const f3 o = mk3(__ldg(J.gb.pos + 3 * (size_t)pix), __ldg(J.gb.pos + 3 * (size_t)pix + 1),
                     __ldg(J.gb.pos + 3 * (size_t)pix + 2));
    const f3 d = mk3(dw.x, dw.y, dw.z);
    const MeshHit h = mesh_closest(J.bvh, o, d, T.P.t_min, T.P.t_max);
    if (h.id < 0) {
        res[r] = make_float4(0.f, 0.f, 0.f, 1.f);
        return;
    }
    float a[3], rr, mm, ss[3];
    f3 n;
    mesh_attr(M, h, d, J.bvh.status, a, &rr, &mm, &n);
    splitsum_d(E, J.env, a, rr, mm, n, mk3(-d.x, -d.y, -d.z), ss);
    res[r] = make_float4(ss[0], ss[1], ss[2], 0.f);
}

// Persistent forward trace of every ray of the table (per-ray (c_rt, T) into res).
template <int K, int CAP>
inline void launch_trace_dyn(const JobTable<CAP>& T, const float4* dirs, float4* res, unsigned long long* next_ray,
                             long long blocks_max, cudaStream_t st, const unsigned* order = nullptr) {
    cudaMemsetAsync(next_ray, 0, sizeof(unsigned long long), st);
    constexpr size_t smem = walk_smem_bytes<K>();
    const long long grid = persistent_grid(k_trace_rays_ww<K, CAP>, smem, blocks_max);
    k_trace_rays_ww<K, CAP><<<(unsigned)grid, kShadeThreads, smem, st>>>(T, dirs, res, next_ray, order);
}

// Persistent forward trace that also keeps the per-ray hit record.
template <int K, int CAP>
inline void launch_trace_save(const JobTable<CAP>& T, const float4* dirs, float4* res, const SavedHits& sv,
                              unsigned long long* next_ray, long long blocks_max, cudaStream_t st,
                              const unsigned* order = nullptr) {
    cudaMemsetAsync(next_ray, 0, sizeof(unsigned long long), st);
    if (sv.ov_count) cudaMemsetAsync(sv.ov_count, 0, sizeof(unsigned), st);
    constexpr size_t smem = walk_smem_bytes<K>();
    const long long grid = persistent_grid(k_trace_rays_save<K, CAP>, smem, blocks_max);
    k_trace_rays_save<K, CAP><<<(unsigned)grid, kShadeThreads, smem, st>>>(T, dirs, res, sv, next_ray, order);
}

}  // namespace
}  // namespace grt
