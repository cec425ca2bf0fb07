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

__global__ void k_env_rows(const float* __restrict__ rgb, int W, int H, float* __restrict__ marg,
                           float* __restrict__ cond) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    float* cr = cond + (size_t)r * (W + 1);
    float acc = 0.f;
    cr[0] = 0.f;
    for (int c = 0; c < W; ++c) {
        acc = add_d(acc, lum_d(rgb + ((size_t)r * W + c) * 3));
        cr[c + 1] = acc;
    }
    for (int c = 1; c <= W; ++c) cr[c] = acc > 0.f ? div_d(cr[c], acc) : div_d((float)c, (float)W);
    marg[r + 1] = acc;
}

__global__ void k_env_marg(float* __restrict__ marg, int H) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float tot = 0.f;
    marg[0] = 0.f;
    for (int r = 1; r <= H; ++r) {
        tot = add_d(tot, marg[r]);
        marg[r] = tot;
    }
    for (int r = 1; r <= H; ++r) marg[r] = div_d(marg[r], tot);
    marg[H + 1] = tot;  // scratch slot past the CDF: total luminance
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
    k_env_rows<<<(H + 63) / 64, 64, 0, st>>>(rgb, W, H, marg, cond);
    k_env_marg<<<1, 32, 0, st>>>(marg, H);
    k_env_texels<<<(W * H + 255) / 256, 256, 0, st>>>(rgb, W, H, marg, texel);
    return launch_error("grt_env_prepare");
}
