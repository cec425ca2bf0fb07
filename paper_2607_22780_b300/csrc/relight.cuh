// relight.cuh -- relighting under a novel map (Sec. III-E, Eq. 14-15).
//
// Trace_attr (Eq. 14), Gaussian backend: along a secondary ray the same admitted hits, in
// the same order and with the same termination as Trace (Eq. 8), are blended with weights
// w_k = T_k a_k into the material state a_r, r_r, m_r (weighted means) and n_r (normalised
// weighted sum of the surfel normals turned towards the ray origin); V_r is the final
// transmittance.  The relit incident radiance (Eq. 15) is
//   L = V_r L_new(w) + (1 - V_r) SplitSum(a_r, r_r, m_r, n_r, E),  seen from v = -w:
//   SplitSum = a (1 - m) E_diff(n) + E_spec(R, r) (F0 A(n.v, r) + B(n.v, r)),
//   R = 2 (n.v) n - v,  F0 = 0.04 (1 - m) + a m,  n.v clamped to [1e-4, 1].
// E (left open by the paper) is tabulated by grt_env_prefilter on equirectangular grids
// (cell centres, the novel map's layout): E_diff = cosine-convolved radiance / pi on 32 x 16,
// E_spec = GGX-lobe (n = v = R) normalised average on 64 x 32 for r = 0.2, 0.4, ..., 1 (level
// r = 0 is the map itself), and the split-sum BRDF table A, B on 32 x 32 (n.v, r) cell
// centres by a 256 x 256 midpoint rule over GGX half vectors.  Lookups are bilinear
// (wrapping in phi) and linear across roughness levels; inside the half-cell caps around
// the poles, where phi has no meaning, they fade linearly in theta towards the mean of the
// pole row (precomputed with the tables), so every lookup is continuous on the sphere.
#pragma once

#include "shade.cuh"

namespace grt {

constexpr int kDiffW = 32, kDiffH = 16, kSpecW = 64, kSpecH = 32, kSpecLevels = 6, kLutN = 32, kLutM = 256;

// Float offsets of the tables in a prefiltered buffer.  poles: for the diffuse grid, each
// specular level and the map itself, the mean of the top row then of the bottom row (rgb).
struct PrefLayout {
    size_t diff, spec, lut, poles, total;
};
__host__ __device__ __forceinline__ PrefLayout pref_layout() {
    PrefLayout l;
    l.diff = 0;
    l.spec = l.diff + 3 * kDiffW * kDiffH;
    l.lut = l.spec + 3 * (size_t)(kSpecLevels - 1) * kSpecW * kSpecH;
    l.poles = l.lut + 2 * kLutN * kLutN;
    l.total = l.poles + 6 * (kSpecLevels + 1);
    return l;
}

struct RelightDev {
    const float* diff;   // [kDiffH][kDiffW][3]
    const float* spec;   // [kSpecLevels - 1][kSpecH][kSpecW][3]
    const float* lut;    // [kLutN (n.v)][kLutN (r)][2]
    const float* poles;  // [diff, spec levels 1.., map][top, bottom][3]
};

// Direction through the centre of cell (row, col) of a W x H equirectangular grid.
__device__ __forceinline__ f3 grid_dir(int row, int col, int W, int H) {
    float sp, cp, st, ct;
    sincospif(2.f * ((float)col + 0.5f) / (float)W, &sp, &cp);
    sincospif(((float)row + 0.5f) / (float)H, &st, &ct);
    return mk3(st * sp, ct, st * cp);
}

// Lookup in direction w: `get(row, col, ch)` reads a cell, pole[6] = top and bottom row means.
template <class Get>
__device__ __forceinline__ void grid_lookup(Get get, const float* pole, int W, int H, f3 w, float out[3]) {
    float ph = atan2f(w.x, w.z);
    if (ph < 0.f) ph += 2.f * kPi;
    const float th = atan2f(sqrtf(w.x * w.x + w.z * w.z), w.y);
    const float u = ph * (0.5f * kInvPi) * (float)W - 0.5f, v = th * kInvPi * (float)H - 0.5f;
    const float fi = floorf(u), fu = u - fi;
    int i0 = (int)fi % W;
    if (i0 < 0) i0 += W;
    const int i1 = i0 + 1 < W ? i0 + 1 : 0;
    int j0, j1, pole_row = -1;
    float fv, tp = 1.f;
    if (v <= 0.f) {
        j0 = j1 = 0;
        fv = 0.f;
        pole_row = 0;
        tp = 2.f * v + 1.f;
    } else if (v >= (float)(H - 1)) {
        j0 = j1 = H - 1;
        fv = 0.f;
        pole_row = 1;
        tp = 2.f * (((float)H - 0.5f) - v);
    } else {
        j0 = (int)floorf(v);
        j1 = j0 + 1;
        fv = v - (float)j0;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        out[ch] = (1.f - fv) * ((1.f - fu) * get(j0, i0, ch) + fu * get(j0, i1, ch)) +
                  fv * ((1.f - fu) * get(j1, i0, ch) + fu * get(j1, i1, ch));
        if (pole_row >= 0) out[ch] = (1.f - tp) * __ldg(pole + 3 * pole_row + ch) + tp * out[ch];
    }
}

__device__ __forceinline__ void splitsum_d(const RelightDev& E, const EnvDev& env, const float a[3], float r, float m,
                                           f3 n, f3 v, float out[3]) {
    const float nv = fminf(fmaxf(dot3(n, v), 1e-4f), 1.f);
    const f3 R = mk3(2.f * nv * n.x - v.x, 2.f * nv * n.y - v.y, 2.f * nv * n.z - v.z);
    float ed[3], e0[3], e1[3];
    grid_lookup([&](int j, int i, int ch) { return __ldg(E.diff + 3 * (j * kDiffW + i) + ch); }, E.poles, kDiffW,
                kDiffH, n, ed);
    const float rc = fminf(fmaxf(r, 0.f), 1.f);
    const float t = rc * (float)(kSpecLevels - 1);
    int l0 = (int)floorf(t);
    if (l0 > kSpecLevels - 2) l0 = kSpecLevels - 2;
    const float f = t - (float)l0;
    if (l0 == 0) {
        grid_lookup(
            [&](int j, int i, int ch) {
                const float4 x = __ldg(env.texel + (size_t)j * env.W + i);
                return ch == 0 ? x.x : (ch == 1 ? x.y : x.z);
            },
            E.poles + 6 * kSpecLevels, env.W, env.H, R, e0);
    } else {
        const float* s0 = E.spec + 3 * (size_t)(l0 - 1) * kSpecW * kSpecH;
        grid_lookup([&](int j, int i, int ch) { return __ldg(s0 + 3 * (j * kSpecW + i) + ch); }, E.poles + 6 * l0,
                    kSpecW, kSpecH, R, e0);
    }
    const float* s1 = E.spec + 3 * (size_t)l0 * kSpecW * kSpecH;
    grid_lookup([&](int j, int i, int ch) { return __ldg(s1 + 3 * (j * kSpecW + i) + ch); }, E.poles + 6 * (l0 + 1),
                kSpecW, kSpecH, R, e1);
    const float x = fminf(fmaxf(nv * (float)kLutN - 0.5f, 0.f), (float)(kLutN - 1));
    const float y = fminf(fmaxf(rc * (float)kLutN - 0.5f, 0.f), (float)(kLutN - 1));
    const int x0 = (int)floorf(x), y0 = (int)floorf(y);
    const int x1 = x0 + 1 < kLutN ? x0 + 1 : x0, y1 = y0 + 1 < kLutN ? y0 + 1 : y0;
    const float fx = x - (float)x0, fy = y - (float)y0;
    float AB[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
        AB[k] = (1.f - fx) * ((1.f - fy) * __ldg(E.lut + 2 * (x0 * kLutN + y0) + k) +
                              fy * __ldg(E.lut + 2 * (x0 * kLutN + y1) + k)) +
                fx * ((1.f - fy) * __ldg(E.lut + 2 * (x1 * kLutN + y0) + k) +
                      fy * __ldg(E.lut + 2 * (x1 * kLutN + y1) + k));
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float kd = a[ch] * (1.f - m), F0 = 0.04f * (1.f - m) + a[ch] * m;
        const float es = (1.f - f) * e0[ch] + f * e1[ch];
        out[ch] = kd * ed[ch] + es * (F0 * AB[0] + AB[1]);
    }
}

// Surfel material arrays read by the attribute visitor.
struct AttrSrc {
    const float4* nrm;  // the tree's decision normals (R(q/|q|) third column, by surfel id)
    const float *albedo, *rough, *metal;
};

// Trace_attr visitor: blends the material state of the composited hits.
struct AttrVisitor {
    const AttrSrc* src;
    f3 d;
    float wsum, a[3], r, m, n[3];
    __device__ __forceinline__ AttrVisitor() {}
    __device__ __forceinline__ AttrVisitor(const AttrSrc* s, f3 dir) : src(s), d(dir), wsum(0.f), r(0.f), m(0.f) {
        a[0] = a[1] = a[2] = 0.f;
        n[0] = n[1] = n[2] = 0.f;
    }
    // one call site: the walks' in-order compositing loop
    __device__ __forceinline__ void composite(int, int id, float, float alpha, float Tb) {
        const float w = Tb * alpha;
        const float4 nv = __ldg(src->nrm + id);
        const f3 nn = mk3(nv.x, nv.y, nv.z);
        const float sw = dot_d(nn, d) > 0.f ? -w : w;  // turned towards the ray origin
        n[0] = fmaf(sw, nn.x, n[0]);
        n[1] = fmaf(sw, nn.y, n[1]);
        n[2] = fmaf(sw, nn.z, n[2]);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) a[ch] = fmaf(w, __ldg(src->albedo + 3 * (size_t)id + ch), a[ch]);
        r = fmaf(w, __ldg(src->rough + id), r);
        m = fmaf(w, __ldg(src->metal + id), m);
        wsum += w;
    }
    __device__ __forceinline__ void finish(float) {}
    // Normalised state after the walk: weighted means and unit normal (zeros without hits).
    __device__ __forceinline__ void resolve() {
        const float iw = wsum > 0.f ? 1.f / wsum : 0.f;
        a[0] *= iw;
        a[1] *= iw;
        a[2] *= iw;
        r *= iw;
        m *= iw;
        const float nl = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const float in = nl > 0.f ? 1.f / nl : 0.f;
        n[0] *= in;
        n[1] *= in;
        n[2] *= in;
    }
};

}  // namespace grt
