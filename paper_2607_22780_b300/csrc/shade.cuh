// shade.cuh -- per-sample MIS shading (Sec. III-C/III-D, Eq. 4-5, Eq. 10-13) shared by the
// forward shading kernels and the shading adjoint.
#pragma once

#include "trace.cuh"

namespace grt {

struct EnvLayout {
    size_t texel, marg, cond, total;
};
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// Environment tables: texel[H*W] float4 | marg[H+1] + one slot (total luminance) |
// cond[H][W+1]; each part 256-byte aligned.
__host__ __device__ inline EnvLayout env_layout(int W, int H) {
    EnvLayout l;
    l.texel = 0;
    l.marg = align256(sizeof(float4) * (size_t)W * H);
    l.cond = l.marg + align256(sizeof(float) * (size_t)(H + 2));
    l.total = l.cond + align256(sizeof(float) * (size_t)H * (W + 1));
    return l;
}

struct EnvDev {
    const float4* texel;  // (R, G, B, p_texel)
    const float* marg;
    const float* cond;
    int W, H;
    float pe_scale;  // W H / (2 pi^2)
};

struct GbufDev {
    const float *pos, *normal, *albedo, *rough, *metal;
    const int* valid;
    float ex, ey, ez;
    int W, H;
};

struct Sampling {
    int n_cos, n_ggx, n_env, brdf;
    uint32_t k0, k1;
};

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;

// GGX normal distribution with a = max(r^2, 1e-4), written with sin^2 = |h x n|^2 so the
// peak keeps its precision for smooth surfaces: D = a^2 / (pi (s2 + c2 a^2)^2).
__device__ __forceinline__ float ggx_D(f3 h, f3 n, float hn, float a2) {
    f3 c = mk3(h.y * n.z - h.z * n.y, h.z * n.x - h.x * n.z, h.x * n.y - h.y * n.x);
    float s2 = dot3(c, c);
    float t = fmaf(hn * hn, a2, s2);
    return a2 / (kPi * t * t);
}
__device__ __forceinline__ float ggx_G1(float c, float a2) {
    return 2.f * c / (c + sqrtf(fmaf(1.f - a2, c * c, a2)));
}
__device__ __forceinline__ float ggx_alpha2(float rough) {
    float a = fmaxf(rough * rough, 1e-4f);
    return a * a;
}

// Visible-normal density of the reflected direction: G1(w_o) D(h) / (4 w_o.n).
__device__ __forceinline__ float pdf_ggx(f3 wo, f3 n, float won, float a2, f3 wi) {
    if (!(won > 0.f)) return 0.f;
    f3 hs = mk3(wo.x + wi.x, wo.y + wi.y, wo.z + wi.z);
    float hl2 = dot3(hs, hs);
    if (!(hl2 > 0.f)) return 0.f;
    float il = rsqrtf(hl2);
    f3 h = mk3(hs.x * il, hs.y * il, hs.z * il);
    float hn = dot3(h, n);
    if (!(hn > 0.f)) return 0.f;
    return ggx_G1(won, a2) * ggx_D(h, n, hn, a2) / (4.f * won);
}

// f = f_d + f_s (Eq. 4-5) or Lambert a/pi.
__device__ __forceinline__ void brdf_eval(int mode, f3 wo, f3 wi, f3 n, const float alb[3], float rough, float metal,
                                          float f[3]) {
    float kd = (mode == 0 ? 1.f : 1.f - metal) * kInvPi;
    f[0] = kd * alb[0];
    f[1] = kd * alb[1];
    f[2] = kd * alb[2];
    if (mode != 1) return;
    float won = dot3(wo, n), win = dot3(wi, n);
    if (!(won > 0.f) || !(win > 0.f)) return;
    f3 hs = mk3(wo.x + wi.x, wo.y + wi.y, wo.z + wi.z);
    float il = rsqrtf(dot3(hs, hs));
    f3 h = mk3(hs.x * il, hs.y * il, hs.z * il);
    float hn = dot3(h, n);
    if (!(hn > 0.f)) return;
    float a2 = ggx_alpha2(rough);
    float DG = ggx_D(h, n, hn, a2) * ggx_G1(win, a2) * ggx_G1(won, a2) / (4.f * win * won);
    float x = fmaxf(1.f - dot3(wi, h), 0.f);
    float x2 = x * x, x5 = x2 * x2 * x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float F0 = fmaf(metal, alb[c], 0.04f * (1.f - metal));
        f[c] = fmaf(DG, fmaf(1.f - F0, x5, F0), f[c]);
    }
}

// Partial derivatives of f (brdf_eval) per channel with respect to that channel's albedo
// (dfa), the metallic weight (dfm) and the roughness (dfr; zero where a = max(r^2, 1e-4)
// is clamped), written in a2 = a^2: dD/da2 = (1 - 2 a2 (h.n)^2 / t) / (pi t^2),
// dG1/da2 = -c (1 - c^2) / ((c + s)^2 s), s = sqrt(a2 + (1 - a2) c^2), da2/dr = 4 a r.
__device__ __forceinline__ void brdf_partials(int mode, f3 wo, f3 wi, f3 n, const float alb[3], float rough,
                                              float metal, float dfa[3], float dfm[3], float dfr[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dfa[c] = (mode == 0 ? 1.f : 1.f - metal) * kInvPi;
        dfm[c] = mode == 0 ? 0.f : -alb[c] * kInvPi;
        dfr[c] = 0.f;
    }
    if (mode != 1) return;
    float won = dot3(wo, n), win = dot3(wi, n);
    if (!(won > 0.f) || !(win > 0.f)) return;
    f3 hs = mk3(wo.x + wi.x, wo.y + wi.y, wo.z + wi.z);
    float il = rsqrtf(dot3(hs, hs));
    f3 h = mk3(hs.x * il, hs.y * il, hs.z * il);
    float hn = dot3(h, n);
    if (!(hn > 0.f)) return;
    const float a = fmaxf(rough * rough, 1e-4f), a2 = a * a;
    const float D = ggx_D(h, n, hn, a2), Gi = ggx_G1(win, a2), Go = ggx_G1(won, a2);
    const float DG = D * Gi * Go / (4.f * win * won);
    float x = fmaxf(1.f - dot3(wi, h), 0.f);
    float x2 = x * x, x5 = x2 * x2 * x;
    float dDG = 0.f;
    if (rough * rough > 1e-4f) {
        f3 cr = mk3(h.y * n.z - h.z * n.y, h.z * n.x - h.x * n.z, h.x * n.y - h.y * n.x);
        const float t = fmaf(hn * hn, a2, dot3(cr, cr));
        const float dD = (1.f - 2.f * a2 * hn * hn / t) / (kPi * t * t);
        const float si = sqrtf(fmaf(1.f - a2, win * win, a2)), so = sqrtf(fmaf(1.f - a2, won * won, a2));
        const float dGi = -win * (1.f - win * win) / ((win + si) * (win + si) * si);
        const float dGo = -won * (1.f - won * won) / ((won + so) * (won + so) * so);
        dDG = DG * (dD / D + dGi / Gi + dGo / Go) * 4.f * a * rough;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float F0 = fmaf(metal, alb[c], 0.04f * (1.f - metal));
        dfa[c] = fmaf(DG * metal, 1.f - x5, dfa[c]);
        dfm[c] = fmaf(DG * (1.f - x5), alb[c] - 0.04f, dfm[c]);
        dfr[c] = dDG * fmaf(1.f - F0, x5, F0);
    }
}

// Per-pixel shading state; decision quantities (n32, wo32, frame) drive the sampler.
struct PixelState {
    f3 x, n, wo, b1, b2;
    float alb[3], rough, metal;
};

__device__ __forceinline__ PixelState load_pixel(const GbufDev& g, int p) {
    PixelState s;
    s.x = mk3(__ldg(g.pos + 3 * (size_t)p), __ldg(g.pos + 3 * (size_t)p + 1), __ldg(g.pos + 3 * (size_t)p + 2));
    f3 nr = mk3(__ldg(g.normal + 3 * (size_t)p), __ldg(g.normal + 3 * (size_t)p + 1), __ldg(g.normal + 3 * (size_t)p + 2));
    s.n = norm_d(nr);
    frame_d(s.n, &s.b1, &s.b2);
    s.wo = norm_d(mk3(sub_d(g.ex, s.x.x), sub_d(g.ey, s.x.y), sub_d(g.ez, s.x.z)));
    s.alb[0] = __ldg(g.albedo + 3 * (size_t)p);
    s.alb[1] = __ldg(g.albedo + 3 * (size_t)p + 1);
    s.alb[2] = __ldg(g.albedo + 3 * (size_t)p + 2);
    s.rough = __ldg(g.rough + p);
    s.metal = __ldg(g.metal + p);
    return s;
}

// Draws the direction of sample j (Sec. III-D allocation order: cosine, GGX, environment).
// Returns false when the sample contributes nothing (w_o below the surface for GGX, or the
// direction below the horizon).
__device__ __forceinline__ bool draw_direction(const Sampling& S, const EnvDev& E, const PixelState& ps, int pix, int j,
                                               f3* w) {
    uint4 rn = philox4x32_10(make_uint4((uint32_t)pix, (uint32_t)j, 0u, 0u), S.k0, S.k1);
    float u0 = unif24(rn.x), u1 = unif24(rn.y);
    bool ok = true;
    if (j < S.n_cos) {
        *w = sample_cos_d(ps.n, ps.b1, ps.b2, u0, u1);
    } else if (j < S.n_cos + S.n_ggx) {
        ok = sample_ggx_d(ps.n, ps.b1, ps.b2, ps.wo, ps.rough, u0, u1, w);
    } else {
        int row = cdf_search(E.marg, E.H, u0);
        int col = cdf_search(E.cond + (size_t)row * (E.W + 1), E.W, u1);
        *w = env_dir_d(row, col, unif24(rn.z), unif24(rn.w), E.W, E.H);
    }
    return ok && dot_d(*w, ps.n) > 0.f;
}

// Integrand weight of a traced sample: g = f cos / q per channel, cos / q, and L_env(w)
// with its texel index.
struct SampleWeight {
    float g[3];
    float L[3];
    float cq;
    int texel;
};

__device__ __forceinline__ SampleWeight sample_weight(const Sampling& S, const EnvDev& E, const PixelState& ps, f3 w) {
    SampleWeight sw;
    int row, col;
    texel_of_d(w, E.W, E.H, &row, &col);
    sw.texel = row * E.W + col;
    float4 tx = __ldg(E.texel + (size_t)row * E.W + col);
    sw.L[0] = tx.x;
    sw.L[1] = tx.y;
    sw.L[2] = tx.z;
    float cosn = fmaxf(dot3(w, ps.n), 0.f);
    float Nr = (float)(S.n_cos + S.n_ggx + S.n_env);
    float q = S.n_cos ? S.n_cos * cosn * kInvPi : 0.f;
    if (S.n_ggx) q = fmaf((float)S.n_ggx, pdf_ggx(ps.wo, ps.n, dot3(ps.wo, ps.n), ggx_alpha2(ps.rough), w), q);
    if (S.n_env) {
        float st = sqrtf(fmaf(w.x, w.x, w.z * w.z));
        q = fmaf((float)S.n_env, tx.w * E.pe_scale / fmaxf(st, 1e-12f), q);
    }
    q /= Nr;
    float f[3];
    brdf_eval(S.brdf, ps.wo, w, ps.n, ps.alb, ps.rough, ps.metal, f);
    float s = q > 0.f ? cosn / q : 0.f;
    sw.cq = s;
    sw.g[0] = f[0] * s;
    sw.g[1] = f[1] * s;
    sw.g[2] = f[2] * s;
    return sw;
}

// Lane layout of a pixel group: G lanes (power of two <= 32) share a pixel, each takes
// samples j = lane_in_group + m G, m = 0 .. S-1.
__host__ __device__ inline int group_lanes(int Nr) {
    int g = 1;
    while (g < Nr && g < 32) g <<= 1;
    return g;
}

}  // namespace grt
