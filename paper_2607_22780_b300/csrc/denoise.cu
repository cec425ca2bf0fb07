// denoise.cu -- cross-bilateral denoiser for low-sample shading (Sec. III-D, "Denoising").
//
// c_den(p) = sum_{p' in Q(p)} B(p,p') c(p') / sum B(p,p'), with
//   B = exp(-|p-p'|^2 / (2 s_s^2))
//     * exp(-|D(p) - D(p')| / (s_d |grad D(p) . (p-p')| + e_d))
//     * max(0, N(p) . N(p'))^s_n,
// N normalised per pixel, grad D the screen-space depth derivative (central difference,
// one-sided next to an invalid or missing neighbour), Q(p) the valid pixels of the
// (2r+1)^2 window around p inside the image.  Invalid pixels, and valid pixels whose normal
// has zero length, keep their input colour.
//
// One block shades a 32x8 tile; the tile plus a halo of max(r, 1) pixels (colour, depth,
// unit normal, validity) and the spatial weights of the window are staged in shared memory,
// so every input pixel is read from HBM once per tile.  The kernel is bound by the
// transcendental functions of its (2r+1)^2 weights per pixel.
#include "common_args.cuh"

namespace grt {
namespace {

constexpr int kTileX = 32, kTileY = 8;

struct DenoiseArgs {
    const float *color, *depth, *normal;
    const int* valid;
    float* out;
    int W, H, r;
    float inv_2ss, sigma_d, sigma_n, eps_d;
};

__host__ __device__ __forceinline__ int tile_pixels(int r) {
    const int h = r > 1 ? r : 1;
    return (kTileX + 2 * h) * (kTileY + 2 * h);
}

__global__ void __launch_bounds__(kTileX * kTileY) k_denoise(DenoiseArgs a) {
    extern __shared__ float sm[];
    const int halo = a.r > 1 ? a.r : 1;
    const int TW = kTileX + 2 * halo, TN = tile_pixels(a.r), nw = (2 * a.r + 1) * (2 * a.r + 1);
    float* s_col = sm;             // [3][TN]
    float* s_dep = s_col + 3 * TN; // [TN]
    float* s_nrm = s_dep + TN;     // [3][TN], unit (zero where invalid)
    float* s_ws = s_nrm + 3 * TN;  // [nw] spatial weights
    int* s_val = reinterpret_cast<int*>(s_ws + nw);
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    const int x0 = blockIdx.x * kTileX - halo, y0 = blockIdx.y * kTileY - halo;
    for (int i = tid; i < TN; i += kTileX * kTileY) {
        const int gx = x0 + i % TW, gy = y0 + i / TW;
        int v = 0;
        float c[3] = {0.f, 0.f, 0.f}, n[3] = {0.f, 0.f, 0.f}, d = 0.f;
        if (gx >= 0 && gy >= 0 && gx < a.W && gy < a.H) {
            const size_t p = (size_t)gy * a.W + gx;
            v = a.valid[p] != 0;
            d = a.depth[p];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                c[k] = a.color[3 * p + k];
                n[k] = a.normal[3 * p + k];
            }
            const float l = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            const float il = l > 0.f ? 1.f / l : 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) n[k] *= il;
        }
        s_val[i] = v;
        s_dep[i] = d;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s_col[k * TN + i] = c[k];
            s_nrm[k * TN + i] = n[k];
        }
    }
    for (int i = tid; i < nw; i += kTileX * kTileY) {
        const int dx = i % (2 * a.r + 1) - a.r, dy = i / (2 * a.r + 1) - a.r;
        s_ws[i] = expf(-(float)(dx * dx + dy * dy) * a.inv_2ss);
    }
    __syncthreads();
    const int px = blockIdx.x * kTileX + threadIdx.x, py = blockIdx.y * kTileY + threadIdx.y;
    if (px >= a.W || py >= a.H) return;
    const int tx = threadIdx.x + halo, ty = threadIdx.y + halo, c0 = ty * TW + tx;
    const size_t p = (size_t)py * a.W + px;
    const float np0 = s_nrm[c0], np1 = s_nrm[TN + c0], np2 = s_nrm[2 * TN + c0];
    if (!s_val[c0] || (np0 == 0.f && np1 == 0.f && np2 == 0.f)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) a.out[3 * p + k] = s_col[k * TN + c0];
        return;
    }
    const float D = s_dep[c0];
    float g[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const int step = ax == 0 ? 1 : TW;
        const bool hm = s_val[c0 - step], hp = s_val[c0 + step];
        g[ax] = (hm && hp) ? 0.5f * (s_dep[c0 + step] - s_dep[c0 - step])
                           : (hp ? s_dep[c0 + step] - D : (hm ? D - s_dep[c0 - step] : 0.f));
    }
    float acc[3] = {0.f, 0.f, 0.f}, wsum = 0.f;
    for (int dy = -a.r; dy <= a.r; ++dy) {
        for (int dx = -a.r; dx <= a.r; ++dx) {
            const int q = c0 + dy * TW + dx;
            if (!s_val[q]) continue;
            const float cosn = np0 * s_nrm[q] + np1 * s_nrm[TN + q] + np2 * s_nrm[2 * TN + q];
            const float wn = cosn > 0.f ? powf(cosn, a.sigma_n) : 0.f;
            if (wn == 0.f) continue;
            const float den = a.sigma_d * fabsf(g[0] * (float)(-dx) + g[1] * (float)(-dy)) + a.eps_d;
            const float wd = expf(-fabsf(D - s_dep[q]) / den);
            const float w = s_ws[(dy + a.r) * (2 * a.r + 1) + dx + a.r] * wd * wn;
            acc[0] = fmaf(w, s_col[q], acc[0]);
            acc[1] = fmaf(w, s_col[TN + q], acc[1]);
            acc[2] = fmaf(w, s_col[2 * TN + q], acc[2]);
            wsum += w;
        }
    }
    const float iw = 1.f / wsum;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.out[3 * p + k] = acc[k] * iw;
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_denoise(const float* color, const float* depth, const float* normal, const int32_t* valid,
                           int32_t W, int32_t H, const grt_denoise_params* params, float* out, void* stream) {
    if (!params) return set_error(GRT_ERR_ARG, "params is NULL");
    if (W <= 0 || H <= 0 || (long long)W * H > (1LL << 30)) return set_error(GRT_ERR_ARG, "bad image size %dx%d", W, H);
    if (!color || !depth || !normal || !valid || !out)
        return set_error(GRT_ERR_ARG, "color, depth, normal, valid and out must be non-NULL");
    if (out == color) return set_error(GRT_ERR_ARG, "out must not alias color (the filter reads neighbours)");
    const grt_denoise_params& q = *params;
    if (q.radius < 0 || q.radius > GRT_DENOISE_MAX_RADIUS)
        return set_error(GRT_ERR_ARG, "radius %d outside [0, %d]", q.radius, GRT_DENOISE_MAX_RADIUS);
    if (!(q.sigma_s > 0.f) || !(q.sigma_d > 0.f) || !(q.sigma_n > 0.f) || !(q.eps_d > 0.f))
        return set_error(GRT_ERR_ARG, "sigma_s, sigma_d, sigma_n and eps_d must be > 0");
    DenoiseArgs a{color, depth, normal, valid, out, W, H, q.radius, 1.f / (2.f * q.sigma_s * q.sigma_s),
                  q.sigma_d, q.sigma_n, q.eps_d};
    const int nw = (2 * q.radius + 1) * (2 * q.radius + 1);
    const size_t smem = sizeof(float) * (7 * (size_t)tile_pixels(q.radius) + nw) + sizeof(int) * tile_pixels(q.radius);
    dim3 grid((W + kTileX - 1) / kTileX, (H + kTileY - 1) / kTileY), block(kTileX, kTileY);
    k_denoise<<<grid, block, smem, (cudaStream_t)stream>>>(a);
    return launch_error("k_denoise");
}
