// envmap.cu -- environment-light proposal tables (Sec. III-D, p_e).
//
// The proposal picks a texel with probability proportional to its luminance
// (0.2126 R + 0.7152 G + 0.0722 B): a row from the marginal CDF, then a column from that
// row's conditional CDF, then a uniform position inside the texel.  The CDFs are FP32
// prefix sums taken sequentially in texel order with explicitly rounded operations, so
// the texel a uniform selects is a pure function of the map.
//
// Table layout (each part 256-byte aligned):
//   texel[H*W]   float4 (R, G, B, p_texel = lum / total)
//   marg[H+2]    float  marginal CDF over rows, marg[0] = 0, marg[H] = 1; marg[H+1] = total
//   cond[H][W+1] float  conditional CDF of each row
#include "common_args.cuh"
#include "shade.cuh"

namespace grt {
namespace {

__device__ __forceinline__ float lum_d(const float* t) {
    float l = mul_d(0.2126f, t[0]);
    l = add_d(l, mul_d(0.7152f, t[1]));
    l = add_d(l, mul_d(0.0722f, t[2]));
    return l;
}

// One warp per row.  The row's luminances arrive 32 at a time (one coalesced load per lane)
// and are added to the running sum in column order, one explicitly rounded add per column
// exactly as in the sequential definition: every lane forms the same chain of sums from the
// shuffled values, and lane k keeps the sum through column k of the chunk.  (A thread per
// row waited on one dependent texel load per column: 0.31 ms for a 512x256 map.)
__global__ void k_env_rows(const float* __restrict__ rgb, int W, int H, float* __restrict__ marg,
                           float* __restrict__ cond) {
    const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (r >= H) return;  // whole warps
    float* cr = cond + (size_t)r * (W + 1);
    if (lane == 0) cr[0] = 0.f;
    float acc = 0.f;
    for (int c0 = 0; c0 < W; c0 += 32) {
        const int c = c0 + lane, n = min(32, W - c0);
        const float l = c < W ? lum_d(rgb + ((size_t)r * W + c) * 3) : 0.f;
        float mine = 0.f;
        for (int k = 0; k < n; ++k) {
            acc = add_d(acc, __shfl_sync(0xffffffffu, l, k));
            if (lane == k) mine = acc;
        }
        if (c < W) cr[c + 1] = mine;
    }
    // each lane normalises the entries it wrote
    for (int c = 1 + lane; c <= W; c += 32) cr[c] = acc > 0.f ? div_d(cr[c], acc) : div_d((float)c, (float)W);
    if (lane == 0) marg[r + 1] = acc;
}

// The marginal CDF in row order, by one warp in the same way.
__global__ void k_env_marg(float* __restrict__ marg, int H) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    if (lane == 0) marg[0] = 0.f;
    float tot = 0.f;
    for (int r0 = 1; r0 <= H; r0 += 32) {
        const int r = r0 + lane, n = min(32, H - r0 + 1);
        const float v = r <= H ? marg[r] : 0.f;
        float mine = 0.f;
        for (int k = 0; k < n; ++k) {
            tot = add_d(tot, __shfl_sync(0xffffffffu, v, k));
            if (lane == k) mine = tot;
        }
        if (r <= H) marg[r] = mine;
    }
    for (int r = 1 + lane; r <= H; r += 32) marg[r] = div_d(marg[r], tot);
    if (lane == 0) marg[H + 1] = tot;  // scratch slot past the CDF: total luminance
}

__global__ void k_env_texels(const float* __restrict__ rgb, int W, int H, const float* __restrict__ marg,
                             float4* __restrict__ texel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    float tot = marg[H + 1];
    const float* t = rgb + 3 * (size_t)i;
    float l = lum_d(t);
    texel[i] = make_float4(t[0], t[1], t[2], tot > 0.f ? l / tot : 0.f);
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" size_t grt_env_tables_bytes(int32_t W, int32_t H) {
    if (W <= 0 || H <= 0) return 0;
    return env_layout(W, H).total;
}

extern "C" int grt_env_prepare(const float* rgb, int32_t W, int32_t H, void* tables, void* stream) {
    if (!rgb || !tables) return set_error(GRT_ERR_ARG, "rgb or tables is NULL");
    if (W <= 0 || H <= 0 || W > 65536 || H > 65536) return set_error(GRT_ERR_ARG, "bad map size %dx%d", W, H);
    if ((uintptr_t)tables & 255) return set_error(GRT_ERR_ARG, "tables must be 256-byte aligned");
    EnvLayout l = env_layout(W, H);
    char* base = (char*)tables;
    float4* texel = (float4*)(base + l.texel);
    float* marg = (float*)(base + l.marg);
    float* cond = (float*)(base + l.cond);
    cudaStream_t st = (cudaStream_t)stream;
    k_env_rows<<<(H + 3) / 4, 128, 0, st>>>(rgb, W, H, marg, cond);  // a warp per row
    k_env_marg<<<1, 32, 0, st>>>(marg, H);
    k_env_texels<<<(W * H + 255) / 256, 256, 0, st>>>(rgb, W, H, marg, texel);
    return launch_error("grt_env_prepare");
}
