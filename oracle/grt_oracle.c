/*
 * grt_oracle.c -- brute-force CPU oracle for differentiable 2D Gaussian ray tracing
 * (2DGRT) of secondary rays with multiple-importance-sampled shading.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header or table with
 * the CUDA path and never calls it.
 *
 * What it computes (paper sections / equations of arXiv 2607.22780):
 *   - surfel frame from a quaternion; t_u, t_v, n = columns of R     (Sec. III-A, 2DGS)
 *   - ray-surfel intersection tau = n.(mu-o)/(n.d), local (u,v),
 *     G = exp(-(u^2+v^2)/2), alpha = min(alpha_max, o*G) kept iff
 *     alpha >= alpha_min                                             (Eq. 7, Sec. III-B)
 *   - every ray is tested against every surfel, all hits are sorted by
 *     (tau, surfel id) and composited front to back,
 *     c_rt = sum T_k a_k c_k, o_rt = sum T_k a_k, stopping after the hit
 *     whose remaining transmittance falls below T_min                (Eq. 8, Eq. 2)
 *   - SH degree-3 colour evaluated at the ray direction, max(0, SH+0.5)
 *   - primary G-buffer with normalised weights w_i = T_i a_i / sum T_j a_j  (Eq. 9)
 *   - MIS: cosine, GGX visible-normal and environment proposals, deterministic
 *     mixture q = (1/N_r) sum_l N_l p_l, c_pbr = (1/N_r) sum g/q       (Eq. 12, Eq. 13)
 *   - light L_i = V L_env + L_ind with (L_ind, 1-V) = Trace           (Eq. 10, Eq. 11)
 *   - metallic microfacet BRDF f = (1-m)a/pi + DFG/(4 cos_i cos_o),
 *     F0 = 0.04(1-m) + m a                                            (Eq. 4, Eq. 5)
 *   - analytic adjoint of Eq. 8 chained to surfel position, rotation, scale,
 *     opacity and colour.
 *
 * Precision.  Continuous quantities are FP64.  Where floating point decides an
 * integer outcome -- the depth order of hits and the plane test that admits a hit
 * (tau in (t_min, t_max), |n.d| >= eps_nd), the sampled secondary direction that
 * decides which surfels a ray meets, and the environment texel a direction falls
 * in -- the decision is taken in FP32 through one fixed sequence of correctly
 * rounded +,-,*,/,sqrt operations (part A below), which the kernel uses too.  The
 * two remaining FP-decided outcomes, alpha >= alpha_min and T < T_min, are taken
 * in FP64 here and reported as "near-boundary" flags when they are within 1e-4
 * (relative) of the threshold.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_FLAG_ALPHA_MIN 1u  /* an admitted/rejected hit had o*G within 1e-4 of alpha_min */
#define OR_FLAG_ALPHA_MAX 2u  /* o*G within 1e-6 of the alpha_max clamp                  */
#define OR_FLAG_T_MIN 4u      /* a transmittance within 1e-4 of T_min                      */
#define OR_FLAG_VALID 8u      /* primary opacity within 1e-5 of the 0.5 validity threshold */

/* ========================================================================== *
 * Part A: decisions in FP32 (fixed order of correctly rounded operations).    *
 * ========================================================================== */

typedef struct { float x, y, z; } f3;

static inline f3 mk3(float x, float y, float z) { f3 r; r.x = x; r.y = y; r.z = z; return r; }

/* ((a.x*b.x + a.y*b.y) + a.z*b.z), every product and sum rounded. */
static inline float dotf(f3 a, f3 b) {
    float s = a.x * b.x;
    s = s + a.y * b.y;
    s = s + a.z * b.z;
    return s;
}

static inline f3 normf(f3 a) {
    float l = sqrtf(dotf(a, a));
    return mk3(a.x / l, a.y / l, a.z / l);
}

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
 * multiplies with the published multipliers and Weyl key increments. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1): the top 24 bits times 2^-24 (exact in FP32 and FP64). */
static inline float unif24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

/* sin and cos of 2*pi*t for t in [0,1]: octant reduction (exact), then Taylor
 * polynomials of sin and cos on [0, pi/4] (truncation below 2e-9). */
void or_sincos2pi(float t, float* s_out, float* c_out) {
    float y = t * 8.0f;
    float kf = floorf(y);
    int k = ((int)kf) & 7;
    float f = y - kf;
    float g = (k & 1) ? (1.0f - f) : f;
    float x = g * 0.785398163397448309616f;
    float x2 = x * x;
    float ps = 2.7557319223985890653e-6f;             /*  1/9!  */
    ps = ps * x2 + -1.9841269841269841270e-4f;        /* -1/7!  */
    ps = ps * x2 + 8.3333333333333333333e-3f;         /*  1/5!  */
    ps = ps * x2 + -1.6666666666666666667e-1f;        /* -1/3!  */
    float s0 = x + (x * x2) * ps;
    float pc = -2.7557319223985890653e-7f;            /* -1/10! */
    pc = pc * x2 + 2.4801587301587301587e-5f;         /*  1/8!  */
    pc = pc * x2 + -1.3888888888888888889e-3f;        /* -1/6!  */
    pc = pc * x2 + 4.1666666666666666667e-2f;         /*  1/4!  */
    pc = pc * x2 + -0.5f;                             /* -1/2!  */
    float c0 = 1.0f + x2 * pc;
    float s, c;
    switch (k) {
        case 0: s = s0; c = c0; break;
        case 1: s = c0; c = s0; break;
        case 2: s = c0; c = -s0; break;
        case 3: s = s0; c = -c0; break;
        case 4: s = -s0; c = -c0; break;
        case 5: s = -c0; c = -s0; break;
        case 6: s = -c0; c = s0; break;
        default: s = -s0; c = c0; break;
    }
    *s_out = s; *c_out = c;
}

/* atan2(y, x) in radians: reduce to a = min/max in [0,1], then to |t| <= tan(pi/8)
 * via atan(a) = pi/4 + atan((a-1)/(a+1)), then the Taylor series of atan to t^15. */
float or_atan2f(float y, float x) {
    float ax = fabsf(x), ay = fabsf(y);
    float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float a = mn / mx;
    float base = 0.0f, t = a;
    if (a > 0.414213562373095f) { t = (a - 1.0f) / (a + 1.0f); base = 0.785398163397448309616f; }
    float t2 = t * t;
    float p = -6.6666666666666666667e-2f;             /* -1/15 */
    p = p * t2 + 7.6923076923076923077e-2f;           /*  1/13 */
    p = p * t2 + -9.0909090909090909091e-2f;          /* -1/11 */
    p = p * t2 + 1.1111111111111111111e-1f;           /*  1/9  */
    p = p * t2 + -1.4285714285714285714e-1f;          /* -1/7  */
    p = p * t2 + 2.0e-1f;                             /*  1/5  */
    p = p * t2 + -3.3333333333333333333e-1f;          /* -1/3  */
    float r = base + (t + (t * t2) * p);
    if (ay > ax) r = 1.57079632679489661923f - r;
    if (x < 0.0f) r = 3.14159265358979323846f - r;
    if (y < 0.0f) r = -r;
    return r;
}

/* Surfel normal n = third column of R(q/|q|), (w,x,y,z) Hamilton convention. */
static f3 normal_from_quat_f(const float* q) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float s2 = w * w;
    s2 = s2 + x * x;
    s2 = s2 + y * y;
    s2 = s2 + z * z;
    float s = sqrtf(s2);
    w = w / s; x = x / s; y = y / s; z = z / s;
    float nx = x * z; nx = nx + w * y; nx = 2.0f * nx;
    float ny = y * z; ny = ny - w * x; ny = 2.0f * ny;
    float nz = x * x; nz = nz + y * y; nz = 1.0f - 2.0f * nz;
    return mk3(nx, ny, nz);
}

/* Plane test of Eq. 7 in FP32: admits tau in (t_min, t_max) when |n.d| >= eps_nd. */
static int plane_test_f(f3 n, f3 mu, f3 o, f3 d, float t_min, float t_max,
                        float eps_nd, float* tau_out, float* den_out) {
    f3 w = mk3(mu.x - o.x, mu.y - o.y, mu.z - o.z);
    float num = dotf(n, w);
    float den = dotf(n, d);
    *den_out = den;
    if (!(fabsf(den) >= eps_nd)) return 0;
    float t = num / den;
    if (!(t > t_min && t < t_max)) return 0;
    *tau_out = t;
    return 1;
}

/* Orthonormal basis (b1, b2, n) of Duff et al., "Building an Orthonormal Basis,
 * Revisited" (JCGT 2017). */
static void frame_f(f3 n, f3* b1, f3* b2) {
    float sign = n.z >= 0.0f ? 1.0f : -1.0f;
    float a = -1.0f / (sign + n.z);
    float b = (n.x * n.y) * a;
    *b1 = mk3(1.0f + ((sign * n.x) * n.x) * a, sign * b, -sign * n.x);
    *b2 = mk3(b, sign + (n.y * n.y) * a, -n.y);
}

static inline f3 to_world_f(f3 b1, f3 b2, f3 n, f3 l) {
    return mk3((b1.x * l.x + b2.x * l.y) + n.x * l.z,
               (b1.y * l.x + b2.y * l.y) + n.y * l.z,
               (b1.z * l.x + b2.z * l.y) + n.z * l.z);
}

/* Cosine-weighted hemisphere direction (Malley's method). */
static f3 sample_cos_f(f3 n, f3 b1, f3 b2, float u0, float u1) {
    float r = sqrtf(u0);
    float s, c;
    or_sincos2pi(u1, &s, &c);
    float lz = 1.0f - u0;
    lz = sqrtf(lz > 0.0f ? lz : 0.0f);
    return to_world_f(b1, b2, n, mk3(r * c, r * s, lz));
}

/* GGX visible-normal sampling (Heitz, "Sampling the GGX Distribution of Visible
 * Normals", JCGT 2018) followed by reflection of w_o about the sampled normal.
 * Returns 0 when w_o is below the shading hemisphere. */
static int sample_ggx_f(f3 n, f3 b1, f3 b2, f3 wo, float rough, float u0, float u1, f3* out) {
    f3 v = mk3(dotf(wo, b1), dotf(wo, b2), dotf(wo, n));
    if (!(v.z > 0.0f)) return 0;
    float a = rough * rough;
    if (a < 1e-4f) a = 1e-4f;
    f3 vh = normf(mk3(a * v.x, a * v.y, v.z));
    float lensq = vh.x * vh.x + vh.y * vh.y;
    f3 T1;
    if (lensq > 0.0f) {
        float l = sqrtf(lensq);
        T1 = mk3(-vh.y / l, vh.x / l, 0.0f);
    } else {
        T1 = mk3(1.0f, 0.0f, 0.0f);
    }
    f3 T2 = mk3(vh.y * T1.z - vh.z * T1.y, vh.z * T1.x - vh.x * T1.z, vh.x * T1.y - vh.y * T1.x);
    float r = sqrtf(u0);
    float s, c;
    or_sincos2pi(u1, &s, &c);
    float t1 = r * c, t2 = r * s;
    float sh = 0.5f * (1.0f + vh.z);
    float q1 = 1.0f - t1 * t1;
    t2 = (1.0f - sh) * sqrtf(q1 > 0.0f ? q1 : 0.0f) + sh * t2;
    float q2 = q1 - t2 * t2;
    float nz = sqrtf(q2 > 0.0f ? q2 : 0.0f);
    f3 nh = mk3((t1 * T1.x + t2 * T2.x) + nz * vh.x,
                (t1 * T1.y + t2 * T2.y) + nz * vh.y,
                (t1 * T1.z + t2 * T2.z) + nz * vh.z);
    f3 ne = mk3(a * nh.x, a * nh.y, nh.z > 0.0f ? nh.z : 0.0f);
    float ll = dotf(ne, ne);
    if (ll > 0.0f) ne = normf(ne); else ne = mk3(0.0f, 0.0f, 1.0f);
    float d2 = 2.0f * dotf(v, ne);
    f3 wl = mk3(d2 * ne.x - v.x, d2 * ne.y - v.y, d2 * ne.z - v.z);
    *out = to_world_f(b1, b2, n, wl);
    return 1;
}

/* Environment sampling tables in FP32, summed sequentially in texel order:
 * lum = (0.2126 R + 0.7152 G) + 0.0722 B per texel; cond[r][c] = prefix/rowsum
 * (uniform when a row is black), marg[r] = prefix of row sums / total. */
void or_env_tables_f32(int W, int H, const float* rgb, float* marg, float* cond) {
    float total = 0.0f;
    float* rowsum = (float*)malloc(sizeof(float) * (size_t)H);
    for (int r = 0; r < H; ++r) {
        float acc = 0.0f;
        float* cr = cond + (size_t)r * (W + 1);
        cr[0] = 0.0f;
        for (int c = 0; c < W; ++c) {
            const float* t = rgb + ((size_t)r * W + c) * 3;
            float l = 0.2126f * t[0];
            l = l + 0.7152f * t[1];
            l = l + 0.0722f * t[2];
            acc = acc + l;
            cr[c + 1] = acc;
        }
        rowsum[r] = acc;
        for (int c = 1; c <= W; ++c) cr[c] = acc > 0.0f ? cr[c] / acc : (float)c / (float)W;
    }
    marg[0] = 0.0f;
    for (int r = 0; r < H; ++r) { total = total + rowsum[r]; marg[r + 1] = total; }
    for (int r = 1; r <= H; ++r) marg[r] = marg[r] / total;
    free(rowsum);
}

/* Largest i in [0, n-1] with cdf[i] <= u (cdf[0] = 0 <= u < cdf[n] = 1). */
static int cdf_search(const float* cdf, int n, float u) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (cdf[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

/* Equirectangular texel of a direction (theta from +y, phi = atan2(x, z)). */
void or_texel_of(float dx, float dy, float dz, int W, int H, int* row, int* col) {
    float phi = or_atan2f(dx, dz);
    if (phi < 0.0f) phi = phi + 6.28318530717958647692f;
    float cf = (phi * 0.159154943091895335769f) * (float)W;
    int c = (int)floorf(cf);
    if (c < 0) c = 0;
    if (c > W - 1) c = W - 1;
    float sxz = sqrtf(dx * dx + dz * dz);
    float th = or_atan2f(sxz, dy);
    float rf = (th * 0.318309886183790671538f) * (float)H;
    int r = (int)floorf(rf);
    if (r < 0) r = 0;
    if (r > H - 1) r = H - 1;
    *row = r; *col = c;
}

/* Direction through texel (row, col) at offsets (u_row, u_col) within it. */
static f3 env_dir_f(int row, int col, float u_row, float u_col, int W, int H) {
    float xp = ((float)col + u_col) / (float)W;
    float xt = ((float)row + u_row) / (float)H;
    float sp, cp, st, ct;
    or_sincos2pi(xp, &sp, &cp);
    or_sincos2pi(xt * 0.5f, &st, &ct);
    return mk3(st * sp, ct, st * cp);
}

/* Primary ray direction through the centre of pixel (px, py); row 0 at the top.
 * cam = eye[3], target[3], up[3], tan(fovy/2). */
static void camera_ray_f(const float* cam, int W, int H, int px, int py, f3* o, f3* d) {
    f3 eye = mk3(cam[0], cam[1], cam[2]);
    f3 fwd = normf(mk3(cam[3] - cam[0], cam[4] - cam[1], cam[5] - cam[2]));
    f3 up = mk3(cam[6], cam[7], cam[8]);
    f3 right = normf(mk3(fwd.y * up.z - fwd.z * up.y, fwd.z * up.x - fwd.x * up.z,
                         fwd.x * up.y - fwd.y * up.x));
    f3 up2 = mk3(right.y * fwd.z - right.z * fwd.y, right.z * fwd.x - right.x * fwd.z,
                 right.x * fwd.y - right.y * fwd.x);
    float th = cam[9];
    float aspect = (float)W / (float)H;
    float sx = ((2.0f * ((float)px + 0.5f)) / (float)W - 1.0f) * th * aspect;
    float sy = (1.0f - (2.0f * ((float)py + 0.5f)) / (float)H) * th;
    f3 dd = mk3((fwd.x + sx * right.x) + sy * up2.x, (fwd.y + sx * right.y) + sy * up2.y,
                (fwd.z + sx * right.z) + sy * up2.z);
    *o = eye;
    *d = normf(dd);
}

/* ========================================================================== *
 * Part B: FP64 continuous arithmetic.                                         *
 * ========================================================================== */

typedef struct { double x, y, z; } d3;
static inline d3 md3(double x, double y, double z) { d3 r; r.x = x; r.y = y; r.z = z; return r; }
static inline double dotd(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline d3 addd(d3 a, d3 b) { return md3(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline d3 subd(d3 a, d3 b) { return md3(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline d3 muld(d3 a, double s) { return md3(a.x * s, a.y * s, a.z * s); }
static inline d3 normd(d3 a) { double l = sqrt(dotd(a, a)); return muld(a, 1.0 / l); }
static inline d3 f2d(f3 a) { return md3(a.x, a.y, a.z); }

/* Surfel parameters in FP64 (FP32 inputs convert exactly; finite differences
 * perturb them in FP64).  Decisions read their FP32 roundings. */
typedef struct {
    int n, color_dim;
    const double *mu, *quat, *scale, *opacity, *color, *albedo, *rough, *metal;
} or_scene;

typedef struct { float alpha_min, alpha_max, t_min, t_max, T_min, eps_nd; } or_params;

typedef struct {
    const float *pos, *normal, *albedo, *rough, *metal; /* [P][3],[P][3],[P][3],[P],[P] */
    const int32_t* valid;                              /* [P] */
    const float* eye;                                  /* [3] */
    int W, H;
} or_gbuf;

typedef struct {
    int W, H;
    const float* rgb;     /* [H][W][3] */
} or_env;

typedef struct { int n_cos, n_ggx, n_env; uint32_t seed_lo, seed_hi; int brdf; } or_sampling;

/* Per-surfel precomputation: FP32 normal for decisions, FP64 frame for arithmetic. */
typedef struct { f3 n32, mu32; d3 tu, tv, n; double qn[4]; double qlen; } surf_pre;

static void frame_from_quat_d(const double* q, surf_pre* s) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double l = sqrt(w * w + x * x + y * y + z * z);
    s->qlen = l;
    w /= l; x /= l; y /= l; z /= l;
    s->qn[0] = w; s->qn[1] = x; s->qn[2] = y; s->qn[3] = z;
    s->tu = md3(1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y));
    s->tv = md3(2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x));
    s->n = md3(2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y));
}

static surf_pre* precompute(const or_scene* sc) {
    surf_pre* p = (surf_pre*)malloc(sizeof(surf_pre) * (size_t)(sc->n > 0 ? sc->n : 1));
    for (int i = 0; i < sc->n; ++i) {
        const double* q = sc->quat + 4 * (size_t)i;
        const double* m = sc->mu + 3 * (size_t)i;
        float q32[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
        p[i].n32 = normal_from_quat_f(q32);
        p[i].mu32 = mk3((float)m[0], (float)m[1], (float)m[2]);
        frame_from_quat_d(q, &p[i]);
    }
    return p;
}

/* Real spherical harmonics to degree 3 (16 functions) at unit direction d, with the
 * normalisation constants written from their closed forms sqrt((2l+1)/(4 pi) ...). */
void or_sh_basis(double x, double y, double z, double* Y) {
    const double pi = 3.14159265358979323846;
    double c0 = sqrt(1.0 / (4 * pi));
    double c1 = sqrt(3.0 / (4 * pi));
    double c2a = sqrt(15.0 / (4 * pi)), c2b = sqrt(5.0 / (16 * pi)), c2c = sqrt(15.0 / (16 * pi));
    double c3a = sqrt(35.0 / (32 * pi)), c3b = sqrt(105.0 / (4 * pi)), c3c = sqrt(21.0 / (32 * pi));
    double c3d = sqrt(7.0 / (16 * pi)), c3e = sqrt(105.0 / (16 * pi));
    double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c0;
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    Y[4] = c2a * x * y; Y[5] = -c2a * y * z; Y[6] = c2b * (2 * zz - xx - yy);
    Y[7] = -c2a * x * z; Y[8] = c2c * (xx - yy);
    Y[9] = -c3a * y * (3 * xx - yy); Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4 * zz - xx - yy); Y[12] = c3d * z * (2 * zz - 3 * xx - 3 * yy);
    Y[13] = -c3c * x * (4 * zz - xx - yy); Y[14] = c3e * z * (xx - yy);
    Y[15] = -c3a * x * (xx - 3 * yy);
}

/* Surfel colour seen along direction d: RGB as stored, or max(0, SH(d) + 0.5). */
static void surfel_colour(const or_scene* sc, int id, d3 d, double c[3], int live[3], double Y[16]) {
    const double* col = sc->color + (size_t)id * sc->color_dim;
    if (sc->color_dim == 3) {
        for (int ch = 0; ch < 3; ++ch) { c[ch] = col[ch]; live[ch] = 1; }
        return;
    }
    or_sh_basis(d.x, d.y, d.z, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int l = 0; l < 16; ++l) s += col[l * 3 + ch] * Y[l];
        live[ch] = s > 0.0;
        c[ch] = s > 0.0 ? s : 0.0;
    }
}

typedef struct {
    float tau32;
    int id;
    float den32;
    double tau, alpha, G, u, v, oG;
    int clamped;
} hit_t;

static int hit_cmp(const void* pa, const void* pb) {
    const hit_t* a = (const hit_t*)pa;
    const hit_t* b = (const hit_t*)pb;
    if (a->tau32 < b->tau32) return -1;
    if (a->tau32 > b->tau32) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* All admitted hits of one ray (brute force over all surfels), sorted by (tau, id). */
static int collect_hits(const or_scene* sc, const surf_pre* pre, const or_params* P, f3 o32,
                        f3 d32, hit_t** buf, int* cap, uint32_t* flags) {
    int nh = 0;
    d3 o = f2d(o32), d = f2d(d32);
    for (int i = 0; i < sc->n; ++i) {
        float tau32, den32;
        if (!plane_test_f(pre[i].n32, pre[i].mu32, o32, d32, P->t_min, P->t_max,
                          P->eps_nd, &tau32, &den32))
            continue;
        const double* m = sc->mu + 3 * (size_t)i;
        d3 mu = md3(m[0], m[1], m[2]);
        d3 n = pre[i].n;
        double nd = dotd(n, d);
        double tau = dotd(n, subd(mu, o)) / nd;
        d3 dp = subd(addd(o, muld(d, tau)), mu);
        double su = sc->scale[2 * (size_t)i], sv = sc->scale[2 * (size_t)i + 1];
        double u = dotd(dp, pre[i].tu) / su, v = dotd(dp, pre[i].tv) / sv;
        double G = exp(-0.5 * (u * u + v * v));
        double oG = (double)sc->opacity[i] * G;
        double amin = P->alpha_min;
        if (fabs(oG / amin - 1.0) < 1e-4) *flags |= OR_FLAG_ALPHA_MIN;
        if (!(oG >= amin)) continue;
        double amax = P->alpha_max;
        if (fabs(oG - amax) < 1e-6) *flags |= OR_FLAG_ALPHA_MAX;
        if (nh == *cap) {
            *cap = *cap ? 2 * *cap : 64;
            *buf = (hit_t*)realloc(*buf, sizeof(hit_t) * (size_t)*cap);
        }
        hit_t* h = &(*buf)[nh++];
        h->tau32 = tau32; h->id = i; h->den32 = den32; h->tau = tau; h->G = G; h->u = u; h->v = v;
        h->oG = oG;
        h->clamped = oG > amax;
        h->alpha = h->clamped ? amax : oG;
    }
    qsort(*buf, (size_t)nh, sizeof(hit_t), hit_cmp);
    return nh;
}

/* Number of leading hits composited before termination; T_k per hit into Tk. */
static int composite_count(const hit_t* h, int nh, const or_params* P, double* Tk, double* Tfinal,
                           uint32_t* flags) {
    double T = 1.0;
    int k = 0;
    for (; k < nh; ++k) {
        Tk[k] = T;
        T *= (1.0 - h[k].alpha);
        if (fabs(T / (double)P->T_min - 1.0) < 1e-4) *flags |= OR_FLAG_T_MIN;
        if (T < (double)P->T_min) { ++k; break; }
    }
    *Tfinal = T;
    return k;
}

typedef struct { hit_t* buf; int cap; double* Tk; int tcap; } ray_ws;

static void ws_ensure(ray_ws* ws, int n) {
    if (ws->tcap < n) {
        ws->tcap = n > 64 ? n : 64;
        ws->Tk = (double*)realloc(ws->Tk, sizeof(double) * (size_t)ws->tcap);
    }
}

/* Trace (Eq. 8): c_rt, o_rt, T_final and the composited hit ids. */
static void trace_one(const or_scene* sc, const surf_pre* pre, const or_params* P, f3 o32, f3 d32,
                      ray_ws* ws, double rgb[3], double* op, double* Tf, int max_hits,
                      int32_t* hits, int32_t* nhits, uint32_t* flags) {
    int nh = collect_hits(sc, pre, P, o32, d32, &ws->buf, &ws->cap, flags);
    ws_ensure(ws, nh + 1);
    double T;
    int K = composite_count(ws->buf, nh, P, ws->Tk, &T, flags);
    d3 d = f2d(d32);
    double c[3], Y[16];
    int live[3];
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    double o = 0.0;
    for (int k = 0; k < K; ++k) {
        const hit_t* h = &ws->buf[k];
        surfel_colour(sc, h->id, d, c, live, Y);
        double w = ws->Tk[k] * h->alpha;
        for (int ch = 0; ch < 3; ++ch) rgb[ch] += w * c[ch];
        o += w;
        if (hits && k < max_hits) hits[k] = h->id;
    }
    *op = o;
    *Tf = T;
    if (nhits) *nhits = K;
}

static int nthreads_or_default(int nt) {
#ifdef _OPENMP
    return nt > 0 ? nt : omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* Ray mode: R rays given by origin and direction (FP32 inputs). */
int or_trace_rays(const or_scene* sc, const or_params* P, int R, const float* ray_o,
                  const float* ray_d, double* out_rgb, double* out_opacity, double* out_T,
                  int max_hits, int32_t* out_hits, int32_t* out_nhits, uint32_t* out_flags,
                  int nthreads) {
    surf_pre* pre = precompute(sc);
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 8)
        for (int r = 0; r < R; ++r) {
            f3 o = mk3(ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]);
            f3 d = mk3(ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]);
            uint32_t fl = 0;
            double rgb[3], op, T;
            trace_one(sc, pre, P, o, d, &ws, rgb, &op, &T, max_hits,
                      out_hits ? out_hits + (size_t)r * max_hits : NULL,
                      out_nhits ? out_nhits + r : NULL, &fl);
            out_rgb[3 * r] = rgb[0]; out_rgb[3 * r + 1] = rgb[1]; out_rgb[3 * r + 2] = rgb[2];
            out_opacity[r] = op;
            if (out_T) out_T[r] = T;
            if (out_flags) out_flags[r] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    free(pre);
    return 0;
}

/* Primary G-buffer (Eq. 9 with a traced camera ray): normalised blend of depth,
 * camera-facing normal, albedo, roughness, metallic; valid iff opacity >= 0.5.
 * Output row i is pixel pixels[i] (all W*H pixels in raster order when pixels is NULL). */
int or_gbuffer(const or_scene* sc, const or_params* P, const float* cam, int W, int H,
               const int32_t* pixels, int n_out,
               double* pos, double* normal, double* albedo, double* rough, double* metal,
               double* alpha, double* depth, int32_t* valid, uint32_t* flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 8)
        for (int i = 0; i < n_out; ++i) {
            const int p = pixels ? pixels[i] : i;
            f3 o32, d32;
            camera_ray_f(cam, W, H, p % W, p / W, &o32, &d32);
            uint32_t fl = 0;
            int nh = collect_hits(sc, pre, P, o32, d32, &ws.buf, &ws.cap, &fl);
            ws_ensure(&ws, nh + 1);
            double T;
            int K = composite_count(ws.buf, nh, P, ws.Tk, &T, &fl);
            double D = 0, a = 0, al[3] = {0, 0, 0}, ro = 0, me = 0;
            d3 N = md3(0, 0, 0);
            for (int k = 0; k < K; ++k) {
                const hit_t* h = &ws.buf[k];
                double w = ws.Tk[k] * h->alpha;
                d3 ni = pre[h->id].n;
                if (h->den32 > 0.0f) ni = muld(ni, -1.0);
                D += w * h->tau;
                N = addd(N, muld(ni, w));
                for (int ch = 0; ch < 3; ++ch) al[ch] += w * sc->albedo[3 * (size_t)h->id + ch];
                ro += w * sc->rough[h->id];
                me += w * sc->metal[h->id];
                a += w;
            }
            double nl = sqrt(dotd(N, N));
            int ok = a >= 0.5 && nl > 1e-12;
            if (fabs(a - 0.5) < 1e-5) fl |= OR_FLAG_VALID;
            valid[i] = ok;
            alpha[i] = a;
            if (ok) {
                D /= a;
                depth[i] = D;
                d3 x = addd(f2d(o32), muld(f2d(d32), D));
                pos[3 * i] = x.x; pos[3 * i + 1] = x.y; pos[3 * i + 2] = x.z;
                normal[3 * i] = N.x / nl; normal[3 * i + 1] = N.y / nl; normal[3 * i + 2] = N.z / nl;
                for (int ch = 0; ch < 3; ++ch) albedo[3 * i + ch] = al[ch] / a;
                rough[i] = ro / a;
                metal[i] = me / a;
            } else {
                depth[i] = 0;
                for (int ch = 0; ch < 3; ++ch) { pos[3 * i + ch] = 0; normal[3 * i + ch] = 0; albedo[3 * i + ch] = 0; }
                rough[i] = 0; metal[i] = 0;
            }
            if (flags) flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    free(pre);
    return 0;
}

/* ---------------------------------------------------------------- shading (FP64) */

static const double PI_D = 3.14159265358979323846;

static double ggx_alpha(double rough) {
    double a = rough * rough;
    return a < 1e-4 ? 1e-4 : a;
}

/* Exact Smith G1 for GGX. */
static double ggx_G1(double cosv, double a) {
    double a2 = a * a;
    return 2.0 * cosv / (cosv + sqrt(a2 + (1.0 - a2) * cosv * cosv));
}

static double ggx_D(double hn, double a) {
    double a2 = a * a;
    double t = hn * hn * (a2 - 1.0) + 1.0;
    return a2 / (PI_D * t * t);
}

/* Density of the GGX visible-normal proposal over incident directions:
 * p(w_i) = G1(w_o) D(h) / (4 w_o.n). */
double or_pdf_ggx(const double* wo_, const double* n_, double rough, const double* wi_) {
    d3 wo = md3(wo_[0], wo_[1], wo_[2]), n = md3(n_[0], n_[1], n_[2]), wi = md3(wi_[0], wi_[1], wi_[2]);
    double won = dotd(wo, n);
    if (!(won > 0.0)) return 0.0;
    d3 hs = addd(wo, wi);
    double hl = sqrt(dotd(hs, hs));
    if (hl == 0.0) return 0.0;
    d3 h = muld(hs, 1.0 / hl);
    double hn = dotd(h, n);
    if (!(hn > 0.0)) return 0.0;
    double a = ggx_alpha(rough);
    return ggx_G1(won, a) * ggx_D(hn, a) / (4.0 * won);
}

/* Metallic microfacet BRDF of Eq. 4-5 (brdf=1) or Lambert a/pi (brdf=0). */
void or_brdf(const double* wo_, const double* wi_, const double* n_, const double* alb, double rough,
             double metal, int brdf, double* f) {
    d3 wo = md3(wo_[0], wo_[1], wo_[2]), wi = md3(wi_[0], wi_[1], wi_[2]), n = md3(n_[0], n_[1], n_[2]);
    if (brdf == 0) {
        for (int ch = 0; ch < 3; ++ch) f[ch] = alb[ch] / PI_D;
        return;
    }
    for (int ch = 0; ch < 3; ++ch) f[ch] = (1.0 - metal) * alb[ch] / PI_D;
    double won = dotd(wo, n), win = dotd(wi, n);
    if (!(won > 0.0) || !(win > 0.0)) return;
    d3 h = normd(addd(wo, wi));
    double hn = dotd(h, n), ih = dotd(wi, h);
    if (!(hn > 0.0)) return;
    double a = ggx_alpha(rough);
    double D = ggx_D(hn, a);
    double G = ggx_G1(win, a) * ggx_G1(won, a);
    double x = 1.0 - ih;
    if (x < 0) x = 0;
    double x5 = x * x * x * x * x;
    for (int ch = 0; ch < 3; ++ch) {
        double F0 = 0.04 * (1.0 - metal) + metal * alb[ch];
        double F = F0 + (1.0 - F0) * x5;
        f[ch] += D * F * G / (4.0 * win * won);
    }
}

typedef struct {
    float* marg;    /* [H+1] FP32 decision table */
    float* cond;    /* [H][W+1] FP32 decision table */
    double* ptex;   /* [H][W] FP64 texel probability lum/total */
} env_tab;

static void env_tab_build(const or_env* env, env_tab* t) {
    int W = env->W, H = env->H;
    t->marg = (float*)malloc(sizeof(float) * (size_t)(H + 1));
    t->cond = (float*)malloc(sizeof(float) * (size_t)H * (W + 1));
    t->ptex = (double*)malloc(sizeof(double) * (size_t)H * W);
    or_env_tables_f32(W, H, env->rgb, t->marg, t->cond);
    double tot = 0.0;
    for (size_t i = 0; i < (size_t)H * W; ++i) {
        const float* c = env->rgb + 3 * i;
        t->ptex[i] = 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2];
        tot += t->ptex[i];
    }
    for (size_t i = 0; i < (size_t)H * W; ++i) t->ptex[i] = tot > 0 ? t->ptex[i] / tot : 0.0;
}

static void env_tab_free(env_tab* t) { free(t->marg); free(t->cond); free(t->ptex); }

/* Environment proposal density over directions: texel probability times the
 * inverse Jacobian W H / (2 pi^2 sin(theta)) of the equirectangular map. */
static double pdf_env(const or_env* env, const env_tab* t, f3 w32, d3 w) {
    int row, col;
    or_texel_of(w32.x, w32.y, w32.z, env->W, env->H, &row, &col);
    double st = sqrt(w.x * w.x + w.z * w.z);
    if (st < 1e-12) st = 1e-12;
    return t->ptex[(size_t)row * env->W + col] * (double)env->W * env->H / (2.0 * PI_D * PI_D * st);
}

/* One Monte Carlo sample of pixel p: direction, its proposal, and whether it was drawn. */
typedef struct { f3 w32; int ok; } sample_t;

static sample_t draw_sample(const or_sampling* S, const env_tab* et, const or_env* env, int pix, int j,
                            f3 n32, f3 b1, f3 b2, f3 wo32, float rough) {
    uint32_t ctr[4] = {(uint32_t)pix, (uint32_t)j, 0u, 0u}, key[2] = {S->seed_lo, S->seed_hi}, r[4];
    or_philox4x32_10(ctr, key, r);
    float u0 = unif24(r[0]), u1 = unif24(r[1]), u2 = unif24(r[2]), u3 = unif24(r[3]);
    sample_t s;
    s.ok = 1;
    if (j < S->n_cos) {
        s.w32 = sample_cos_f(n32, b1, b2, u0, u1);
    } else if (j < S->n_cos + S->n_ggx) {
        s.ok = sample_ggx_f(n32, b1, b2, wo32, rough, u0, u1, &s.w32);
    } else {
        int row = cdf_search(et->marg, env->H, u0);
        int col = cdf_search(et->cond + (size_t)row * (env->W + 1), env->W, u1);
        s.w32 = env_dir_f(row, col, u2, u3, env->W, env->H);
    }
    if (s.ok && !(dotf(s.w32, n32) > 0.0f)) s.ok = 0;
    return s;
}

typedef struct {
    double g[3];        /* f * cos / q, per channel, for this sample */
    double cq;          /* cos / q */
    double Lenv[3];
    int row, col;       /* environment texel of the direction */
    double rgb[3], op, T;
} sample_eval;

/* Environment radiance along the sample, mixture pdf q and BRDF weight g = f cos / q. */
static void sample_weights(const or_env* env, const env_tab* et, const or_sampling* S, f3 w32, d3 n, d3 wo,
                           const double* alb, double rough, double metal, sample_eval* e) {
    d3 w = normd(f2d(w32));
    int row, col;
    or_texel_of(w32.x, w32.y, w32.z, env->W, env->H, &row, &col);
    e->row = row;
    e->col = col;
    const float* L = env->rgb + ((size_t)row * env->W + col) * 3;
    for (int ch = 0; ch < 3; ++ch) e->Lenv[ch] = L[ch];
    int Nr = S->n_cos + S->n_ggx + S->n_env;
    double cosn = dotd(w, n);
    if (cosn < 0) cosn = 0;
    double pc = cosn / PI_D;
    double wo_a[3] = {wo.x, wo.y, wo.z}, n_a[3] = {n.x, n.y, n.z}, w_a[3] = {w.x, w.y, w.z};
    double pg = S->n_ggx > 0 ? or_pdf_ggx(wo_a, n_a, rough, w_a) : 0.0;
    double pe = S->n_env > 0 ? pdf_env(env, et, w32, w) : 0.0;
    double q = (S->n_cos * pc + S->n_ggx * pg + S->n_env * pe) / Nr;
    double f[3];
    or_brdf(wo_a, w_a, n_a, alb, rough, metal, S->brdf, f);
    e->cq = q > 0 ? cosn / q : 0.0;
    for (int ch = 0; ch < 3; ++ch) e->g[ch] = q > 0 ? f[ch] * cosn / q : 0.0;
}

/* Evaluate the sample: trace, environment, pdfs, BRDF. */
static void eval_sample(const or_scene* sc, const surf_pre* pre, const or_params* P, const or_env* env,
                        const env_tab* et, const or_sampling* S, ray_ws* ws, f3 x32, f3 w32,
                        d3 n, d3 wo, const double* alb, double rough, double metal,
                        sample_eval* e, uint32_t* flags) {
    trace_one(sc, pre, P, x32, w32, ws, e->rgb, &e->op, &e->T, 0, NULL, NULL, flags);
    sample_weights(env, et, S, w32, n, wo, alb, rough, metal, e);
}

static void pixel_setup(const or_gbuf* gb, int p, f3* x32, f3* n32, f3* b1, f3* b2, f3* wo32, d3* n,
                        d3* wo) {
    const float* ps = gb->pos + 3 * (size_t)p;
    const float* ns = gb->normal + 3 * (size_t)p;
    *x32 = mk3(ps[0], ps[1], ps[2]);
    *n32 = normf(mk3(ns[0], ns[1], ns[2]));
    frame_f(*n32, b1, b2);
    *wo32 = normf(mk3(gb->eye[0] - ps[0], gb->eye[1] - ps[1], gb->eye[2] - ps[2]));
    *n = normd(md3(ns[0], ns[1], ns[2]));
    *wo = normd(md3((double)gb->eye[0] - ps[0], (double)gb->eye[1] - ps[1], (double)gb->eye[2] - ps[2]));
}

/* MIS shading of Eq. 13 for a list of pixels (or all W*H when pixel_list is NULL):
 * colour = (1/N_r) sum g/q, visibility = (1/N_r) sum V, indirect = (1/N_r) sum L_ind,
 * light (optional) = (1/N_r) sum L_i, the mean incident radiance of Eq. 16.
 * Samples below the horizon contribute nothing (V = 0, L_ind = 0). */
int or_shade_pixels(const or_scene* sc, const or_params* P, const or_gbuf* gb, const or_env* env,
                    const or_sampling* S, const int32_t* pixel_list, int n_pixels, double* out_color,
                    double* out_vis, double* out_ind, double* out_light, uint32_t* out_flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    env_tab et;
    env_tab_build(env, &et);
    int Nr = S->n_cos + S->n_ggx + S->n_env;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_pixels; ++i) {
            int p = pixel_list ? pixel_list[i] : i;
            double col[3] = {0, 0, 0}, vis = 0, ind[3] = {0, 0, 0}, light[3] = {0, 0, 0};
            uint32_t fl = 0;
            if (gb->valid[p] && Nr > 0) {
                f3 x32, n32, b1, b2, wo32;
                d3 n, wo;
                pixel_setup(gb, p, &x32, &n32, &b1, &b2, &wo32, &n, &wo);
                double alb[3] = {gb->albedo[3 * (size_t)p], gb->albedo[3 * (size_t)p + 1], gb->albedo[3 * (size_t)p + 2]};
                for (int j = 0; j < Nr; ++j) {
                    sample_t s = draw_sample(S, &et, env, p, j, n32, b1, b2, wo32, gb->rough[p]);
                    if (!s.ok) continue;
                    sample_eval e;
                    eval_sample(sc, pre, P, env, &et, S, &ws, x32, s.w32, n, wo, alb, gb->rough[p],
                                gb->metal[p], &e, &fl);
                    double V = 1.0 - e.op;
                    for (int ch = 0; ch < 3; ++ch) {
                        double Li = V * e.Lenv[ch] + e.rgb[ch];
                        col[ch] += e.g[ch] * Li;
                        ind[ch] += e.rgb[ch];
                        light[ch] += Li;
                    }
                    vis += V;
                }
                for (int ch = 0; ch < 3; ++ch) { col[ch] /= Nr; ind[ch] /= Nr; light[ch] /= Nr; }
                vis /= Nr;
            }
            for (int ch = 0; ch < 3; ++ch) { out_color[3 * (size_t)i + ch] = col[ch]; out_ind[3 * (size_t)i + ch] = ind[ch]; }
            if (out_light)
                for (int ch = 0; ch < 3; ++ch) out_light[3 * (size_t)i + ch] = light[ch];
            out_vis[i] = vis;
            if (out_flags) out_flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    env_tab_free(&et);
    free(pre);
    return 0;
}

/* ---------------------------------------------------------------- backward (FP64) */

typedef struct { double *g_mu, *g_quat, *g_scale, *g_opacity, *g_color; } or_grads;

static inline void atomic_add_d(double* p, double v) {
#pragma omp atomic
    *p += v;
}

/* Adjoint of Eq. 8 for one ray given dL/dc_rt (Gc) and dL/do_rt (Go):
 *   dL/dc_k = Gc T_k a_k,
 *   dL/da_k = Gc.(T_k c_k - S_k/(1-a_k)) + Go T_final/(1-a_k),  S_k = sum_{j>k} T_j a_j c_j,
 * then a = o G, G = exp(-(u^2+v^2)/2), u = (p-mu).t_u/s_u, v = (p-mu).t_v/s_v,
 * p = o_ray + tau d, tau = n.(mu-o_ray)/(n.d), into mu, q (through R(q/|q|)), s, o, colour. */
static void backward_one(const or_scene* sc, const surf_pre* pre, const or_params* P, f3 o32, f3 d32,
                         const double Gc[3], double Go, ray_ws* ws, const or_grads* g, uint32_t* flags) {
    int nh = collect_hits(sc, pre, P, o32, d32, &ws->buf, &ws->cap, flags);
    ws_ensure(ws, nh + 1);
    double Tf;
    int K = composite_count(ws->buf, nh, P, ws->Tk, &Tf, flags);
    if (K == 0) return;
    d3 d = f2d(d32), o = f2d(o32);
    double* wc = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    double* cc = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    int* lv = (int*)malloc(sizeof(int) * 3 * (size_t)K);
    double Y[16];
    for (int k = 0; k < K; ++k) {
        surfel_colour(sc, ws->buf[k].id, d, cc + 3 * k, lv + 3 * k, Y);
        double w = ws->Tk[k] * ws->buf[k].alpha;
        for (int ch = 0; ch < 3; ++ch) wc[3 * k + ch] = w * cc[3 * k + ch];
    }
    double S[3] = {0, 0, 0};
    for (int k = K - 1; k >= 0; --k) {
        const hit_t* h = &ws->buf[k];
        int id = h->id;
        double a = h->alpha, Tk = ws->Tk[k];
        double dLda = Go * Tf / (1.0 - a);
        for (int ch = 0; ch < 3; ++ch) dLda += Gc[ch] * (Tk * cc[3 * k + ch] - S[ch] / (1.0 - a));
        for (int ch = 0; ch < 3; ++ch) S[ch] += wc[3 * k + ch];
        /* colour */
        double dLdc[3];
        for (int ch = 0; ch < 3; ++ch) dLdc[ch] = Gc[ch] * Tk * a;
        if (sc->color_dim == 3) {
            for (int ch = 0; ch < 3; ++ch) atomic_add_d(&g->g_color[3 * (size_t)id + ch], dLdc[ch]);
        } else {
            or_sh_basis(d.x, d.y, d.z, Y);
            for (int ch = 0; ch < 3; ++ch) {
                if (!lv[3 * k + ch]) continue;
                for (int l = 0; l < 16; ++l)
                    atomic_add_d(&g->g_color[(size_t)id * 48 + l * 3 + ch], dLdc[ch] * Y[l]);
            }
        }
        if (h->clamped) continue;
        atomic_add_d(&g->g_opacity[id], dLda * h->G);
        double dLdu = -dLda * a * h->u, dLdv = -dLda * a * h->v;
        double su = sc->scale[2 * (size_t)id], sv = sc->scale[2 * (size_t)id + 1];
        atomic_add_d(&g->g_scale[2 * (size_t)id], -dLdu * h->u / su);
        atomic_add_d(&g->g_scale[2 * (size_t)id + 1], -dLdv * h->v / sv);
        const surf_pre* sp = &pre[id];
        double nd = dotd(sp->n, d);
        double tud = dotd(sp->tu, d), tvd = dotd(sp->tv, d);
        const double* m = sc->mu + 3 * (size_t)id;
        d3 mu = md3(m[0], m[1], m[2]);
        d3 dp = subd(addd(o, muld(d, h->tau)), mu);
        /* d u / d mu = (t_u.d / (s_u n.d)) n - t_u / s_u ; likewise v */
        d3 gmu = addd(muld(sp->n, dLdu * tud / (su * nd) + dLdv * tvd / (sv * nd)),
                      addd(muld(sp->tu, -dLdu / su), muld(sp->tv, -dLdv / sv)));
        atomic_add_d(&g->g_mu[3 * (size_t)id], gmu.x);
        atomic_add_d(&g->g_mu[3 * (size_t)id + 1], gmu.y);
        atomic_add_d(&g->g_mu[3 * (size_t)id + 2], gmu.z);
        /* gradients with respect to the columns of R */
        d3 gtu = muld(dp, dLdu / su), gtv = muld(dp, dLdv / sv);
        d3 gn = muld(dp, -(dLdu * tud / su + dLdv * tvd / sv) / nd);
        double G00 = gtu.x, G10 = gtu.y, G20 = gtu.z;
        double G01 = gtv.x, G11 = gtv.y, G21 = gtv.z;
        double G02 = gn.x, G12 = gn.y, G22 = gn.z;
        double w = sp->qn[0], x = sp->qn[1], y = sp->qn[2], z = sp->qn[3];
        double gw = 2 * (-z * G01 + y * G02 + z * G10 - x * G12 - y * G20 + x * G21);
        double gx = 2 * (y * G01 + z * G02 + y * G10 - 2 * x * G11 - w * G12 + z * G20 + w * G21 - 2 * x * G22);
        double gy = 2 * (-2 * y * G00 + x * G01 + w * G02 + x * G10 + z * G12 - w * G20 + z * G21 - 2 * y * G22);
        double gz = 2 * (-2 * z * G00 - w * G01 + x * G02 + w * G10 - 2 * z * G11 + y * G12 + x * G20 + y * G21);
        double qd = w * gw + x * gx + y * gy + z * gz;
        double il = 1.0 / sp->qlen;
        atomic_add_d(&g->g_quat[4 * (size_t)id], (gw - w * qd) * il);
        atomic_add_d(&g->g_quat[4 * (size_t)id + 1], (gx - x * qd) * il);
        atomic_add_d(&g->g_quat[4 * (size_t)id + 2], (gy - y * qd) * il);
        atomic_add_d(&g->g_quat[4 * (size_t)id + 3], (gz - z * qd) * il);
    }
    free(wc); free(cc); free(lv);
}

/* Ray-mode backward: gradients accumulate (+=) into the caller's zeroed arrays. */
int or_backward_rays(const or_scene* sc, const or_params* P, int R, const float* ray_o, const float* ray_d,
                     const double* dL_drgb, const double* dL_dop, const or_grads* g, uint32_t* out_flags,
                     int nthreads) {
    surf_pre* pre = precompute(sc);
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 8)
        for (int r = 0; r < R; ++r) {
            f3 o = mk3(ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]);
            f3 d = mk3(ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]);
            uint32_t fl = 0;
            backward_one(sc, pre, P, o, d, dL_drgb + 3 * (size_t)r, dL_dop[r], &ws, g, &fl);
            if (out_flags) out_flags[r] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    free(pre);
    return 0;
}

/* Pixel-mode backward of the shaded outputs: per traced sample,
 *   dL/dc_rt = dL/dcolor * g / N_r + dL/dind / N_r,
 *   dL/do_rt = -(sum_ch dL/dcolor_ch g_ch Lenv_ch) / N_r - dL/dvis / N_r,
 * with g = f cos / q; dL_dvis and dL_dind may be NULL. */
int or_backward_pixels(const or_scene* sc, const or_params* P, const or_gbuf* gb, const or_env* env,
                       const or_sampling* S, const int32_t* pixel_list, int n_pixels, const double* dL_dcolor,
                       const double* dL_dvis, const double* dL_dind, const or_grads* g, uint32_t* out_flags,
                       int nthreads) {
    surf_pre* pre = precompute(sc);
    env_tab et;
    env_tab_build(env, &et);
    int Nr = S->n_cos + S->n_ggx + S->n_env;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_pixels; ++i) {
            int p = pixel_list ? pixel_list[i] : i;
            uint32_t fl = 0;
            if (gb->valid[p] && Nr > 0) {
                f3 x32, n32, b1, b2, wo32;
                d3 n, wo;
                pixel_setup(gb, p, &x32, &n32, &b1, &b2, &wo32, &n, &wo);
                double alb[3] = {gb->albedo[3 * (size_t)p], gb->albedo[3 * (size_t)p + 1], gb->albedo[3 * (size_t)p + 2]};
                const double* dc = dL_dcolor + 3 * (size_t)i;
                for (int j = 0; j < Nr; ++j) {
                    sample_t s = draw_sample(S, &et, env, p, j, n32, b1, b2, wo32, gb->rough[p]);
                    if (!s.ok) continue;
                    sample_eval e;
                    eval_sample(sc, pre, P, env, &et, S, &ws, x32, s.w32, n, wo, alb, gb->rough[p],
                                gb->metal[p], &e, &fl);
                    double Gc[3], Go = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        Gc[ch] = dc[ch] * e.g[ch] / Nr + (dL_dind ? dL_dind[3 * (size_t)i + ch] / Nr : 0.0);
                        Go -= dc[ch] * e.g[ch] * e.Lenv[ch] / Nr;
                    }
                    if (dL_dvis) Go -= dL_dvis[i] / Nr;
                    backward_one(sc, pre, P, x32, s.w32, Gc, Go, &ws, g, &fl);
                }
            }
            if (out_flags) out_flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    env_tab_free(&et);
    free(pre);
    return 0;
}

/* ---------------------------------------------------------------- exposed helpers */

/* Sampled direction of sample j of a pixel (for distribution tests).  Returns 1 when a
 * direction was drawn above the horizon. */
int or_sample_direction(const or_sampling* S, const or_env* env, const float* pos, const float* nrm,
                        const float* eye, float rough, int pix, int j, float* w_out) {
    env_tab et;
    env_tab_build(env, &et);
    f3 n32 = normf(mk3(nrm[0], nrm[1], nrm[2])), b1, b2;
    frame_f(n32, &b1, &b2);
    f3 wo32 = normf(mk3(eye[0] - pos[0], eye[1] - pos[1], eye[2] - pos[2]));
    sample_t s = draw_sample(S, &et, env, pix, j, n32, b1, b2, wo32, rough);
    env_tab_free(&et);
    w_out[0] = s.w32.x; w_out[1] = s.w32.y; w_out[2] = s.w32.z;
    return s.ok;
}

/* Many directions of one proposal at one shading point, drawn without the horizon cut. */
void or_sample_many(int proposal, const or_env* env, const float* nrm, const float* wo, float rough,
                    uint32_t seed, int count, float* w_out, int32_t* ok_out) {
    env_tab et;
    env_tab_build(env, &et);
    f3 n32 = normf(mk3(nrm[0], nrm[1], nrm[2])), b1, b2;
    frame_f(n32, &b1, &b2);
    f3 wo32 = normf(mk3(wo[0], wo[1], wo[2]));
    for (int i = 0; i < count; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 7u, 0u}, key[2] = {seed, 0x5EEDu}, r[4];
        or_philox4x32_10(ctr, key, r);
        float u0 = unif24(r[0]), u1 = unif24(r[1]), u2 = unif24(r[2]), u3 = unif24(r[3]);
        f3 w = mk3(0, 0, 0);
        int ok = 1;
        if (proposal == 0) w = sample_cos_f(n32, b1, b2, u0, u1);
        else if (proposal == 1) ok = sample_ggx_f(n32, b1, b2, wo32, rough, u0, u1, &w);
        else {
            int row = cdf_search(et.marg, env->H, u0);
            int col = cdf_search(et.cond + (size_t)row * (env->W + 1), env->W, u1);
            w = env_dir_f(row, col, u2, u3, env->W, env->H);
        }
        w_out[3 * i] = w.x; w_out[3 * i + 1] = w.y; w_out[3 * i + 2] = w.z;
        ok_out[i] = ok;
    }
    env_tab_free(&et);
}

double or_pdf_env_dir(const or_env* env, const float* w) {
    env_tab et;
    env_tab_build(env, &et);
    f3 w32 = mk3(w[0], w[1], w[2]);
    double r = pdf_env(env, &et, w32, normd(f2d(w32)));
    env_tab_free(&et);
    return r;
}

void or_camera_ray(const float* cam, int W, int H, int px, int py, float* o, float* d) {
    f3 oo, dd;
    camera_ray_f(cam, W, H, px, py, &oo, &dd);
    o[0] = oo.x; o[1] = oo.y; o[2] = oo.z;
    d[0] = dd.x; d[1] = dd.y; d[2] = dd.z;
}

void or_normal_from_quat(const float* q, float* n) {
    f3 r = normal_from_quat_f(q);
    n[0] = r.x; n[1] = r.y; n[2] = r.z;
}

/* ---------------------------------------------------------------- denoiser (FP64) */

/* Screen-space depth derivative along one axis at pixel (x, y): central difference when
 * both neighbours are valid, one-sided when only one is, 0 otherwise. */
static double depth_slope(const double* D, const int32_t* valid, int W, int H, int x, int y, int ax) {
    int xm = x - (ax == 0), ym = y - (ax == 1), xp = x + (ax == 0), yp = y + (ax == 1);
    int has_m = xm >= 0 && ym >= 0 && valid[ym * W + xm];
    int has_p = xp < W && yp < H && valid[yp * W + xp];
    if (has_m && has_p) return 0.5 * (D[yp * W + xp] - D[ym * W + xm]);
    if (has_p) return D[yp * W + xp] - D[y * W + x];
    if (has_m) return D[y * W + x] - D[ym * W + xm];
    return 0.0;
}

/* Cross-bilateral denoiser (Sec. III-D): c_den(p) = sum_{p' in Q(p)} B(p,p') c(p') /
 * sum B(p,p'), B = exp(-|p-p'|^2 / (2 s_s^2)) * exp(-|D(p)-D(p')| / (s_d |grad D(p).(p-p')|
 * + e_d)) * max(0, N(p).N(p'))^s_n, with N normalised per pixel; Q(p) = the valid pixels of
 * the (2r+1)^2 window around p inside the image.  Invalid pixels, and valid pixels whose
 * normal has zero length (nothing to compare with), keep their input. */
int or_denoise(const double* color, const double* depth, const double* normal, const int32_t* valid, int W, int H,
               int radius, double sigma_s, double sigma_d, double sigma_n, double eps_d, double* out,
               int nthreads) {
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int p = 0; p < W * H; ++p) {
        int x = p % W, y = p / W;
        double nl = sqrt(normal[3 * p] * normal[3 * p] + normal[3 * p + 1] * normal[3 * p + 1] +
                         normal[3 * p + 2] * normal[3 * p + 2]);
        if (!valid[p] || nl == 0.0) {  /* no surface, or no normal to compare with */
            for (int c = 0; c < 3; ++c) out[3 * p + c] = color[3 * p + c];
            continue;
        }
        double gx = depth_slope(depth, valid, W, H, x, y, 0), gy = depth_slope(depth, valid, W, H, x, y, 1);
        double np[3] = {normal[3 * p] / nl, normal[3 * p + 1] / nl, normal[3 * p + 2] / nl};
        double acc[3] = {0, 0, 0}, wsum = 0;
        for (int dy = -radius; dy <= radius; ++dy) {
            for (int dx = -radius; dx <= radius; ++dx) {
                int xq = x + dx, yq = y + dy;
                if (xq < 0 || yq < 0 || xq >= W || yq >= H) continue;
                int q = yq * W + xq;
                if (!valid[q]) continue;
                double nq_l = sqrt(normal[3 * q] * normal[3 * q] + normal[3 * q + 1] * normal[3 * q + 1] +
                                   normal[3 * q + 2] * normal[3 * q + 2]);
                double cosn = nq_l > 0 ? (np[0] * normal[3 * q] + np[1] * normal[3 * q + 1] + np[2] * normal[3 * q + 2]) / nq_l
                                       : 0.0;
                /* p - p' = (-dx, -dy) */
                double ws = exp(-(double)(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s));
                double wd = exp(-fabs(depth[p] - depth[q]) / (sigma_d * fabs(gx * (-dx) + gy * (-dy)) + eps_d));
                double wn = pow(cosn > 0 ? cosn : 0.0, sigma_n);
                double w = ws * wd * wn;
                for (int c = 0; c < 3; ++c) acc[c] += w * color[3 * q + c];
                wsum += w;
            }
        }
        for (int c = 0; c < 3; ++c) out[3 * p + c] = acc[c] / wsum;
    }
    return 0;
}

/* ---------------------------------------------------------------- relighting (FP64) */
/* Sec. III-E: Trace_attr (Eq. 14) returns the visibility V_r of the novel environment and
 * the material state (a_r, r_r, m_r, n_r) met along a secondary ray; the incident radiance
 * under the novel map is L = V_r L_new(w) + (1 - V_r) SplitSum(a_r, r_r, m_r, n_r, E)
 * (Eq. 15), substituted for L_i in the MIS estimate.  E, left open by the paper, is:
 *   E_diff(n)    = (1/pi) sum_t L_t max(0, n.w_t) dW_t                 on a 32 x 16 grid,
 *   E_spec(R, r) = sum_t L_t w_t / sum_t w_t, w_t = D(R.h_t) max(0, R.w_t) dW_t,
 *                  h_t = normalize(w_t + R) (the split-sum lobe with n = v = R),
 *                  levels r = l/5, l = 1..5 on 64 x 32 grids; level 0 is the map itself,
 *   A, B(nv, r)  = split-sum BRDF integrals of the specular lobe of Eq. 5 (D, Smith G,
 *                  Schlick F = F0 + (1 - F0)(1 - v.h)^5 split as F0 A + B), midpoint rule
 *                  over 256 x 256 GGX half-vector samples, 32 x 32 cell centres,
 * texels t of the novel map with centre directions w_t and solid angles dW_t.  All grids
 * use the map's equirectangular layout with cell centres; lookups are bilinear (wrapping
 * in phi; towards the pole-row mean inside the polar half-cell caps) and linear across
 * roughness levels. */
#define OR_DIFF_W 32
#define OR_DIFF_H 16
#define OR_SPEC_W 64
#define OR_SPEC_H 32
#define OR_SPEC_LEVELS 6
#define OR_LUT_N 32
#define OR_LUT_M 256

typedef struct {
    int W, H;                 /* novel map */
    const float* rgb;         /* [H][W][3] */
    const double* diff;       /* [OR_DIFF_H][OR_DIFF_W][3] */
    const double* spec;       /* [OR_SPEC_LEVELS - 1][OR_SPEC_H][OR_SPEC_W][3] */
    const double* lut;        /* [OR_LUT_N (nv)][OR_LUT_N (r)][2] */
} or_prefiltered;

static d3 grid_dir(int row, int col, int W, int H) {
    double ph = 2.0 * PI_D * (col + 0.5) / W, th = PI_D * (row + 0.5) / H;
    return md3(sin(th) * sin(ph), cos(th), sin(th) * cos(ph));
}

void or_env_prefilter(int W, int H, const float* rgb, double* diff, double* spec, double* lut) {
    int n = W * H;
    d3* dir = (d3*)malloc(sizeof(d3) * (size_t)n);
    double* dw = (double*)malloc(sizeof(double) * (size_t)n);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            dir[r * W + c] = grid_dir(r, c, W, H);
            dw[r * W + c] = (2.0 * PI_D / W) * (cos(PI_D * r / H) - cos(PI_D * (r + 1) / H));
        }
#pragma omp parallel for schedule(dynamic, 1)
    for (int g = 0; g < OR_DIFF_W * OR_DIFF_H; ++g) {
        d3 nn = grid_dir(g / OR_DIFF_W, g % OR_DIFF_W, OR_DIFF_W, OR_DIFF_H);
        double acc[3] = {0, 0, 0};
        for (int t = 0; t < n; ++t) {
            double c = dotd(nn, dir[t]);
            if (c <= 0) continue;
            for (int ch = 0; ch < 3; ++ch) acc[ch] += rgb[3 * (size_t)t + ch] * c * dw[t];
        }
        for (int ch = 0; ch < 3; ++ch) diff[3 * g + ch] = acc[ch] / PI_D;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int g = 0; g < (OR_SPEC_LEVELS - 1) * OR_SPEC_W * OR_SPEC_H; ++g) {
        int lev = 1 + g / (OR_SPEC_W * OR_SPEC_H), cell = g % (OR_SPEC_W * OR_SPEC_H);
        double a = ggx_alpha((double)lev / (OR_SPEC_LEVELS - 1));
        d3 R = grid_dir(cell / OR_SPEC_W, cell % OR_SPEC_W, OR_SPEC_W, OR_SPEC_H);
        double acc[3] = {0, 0, 0}, wsum = 0;
        for (int t = 0; t < n; ++t) {
            double c = dotd(R, dir[t]);
            if (c <= 0) continue;
            d3 h = normd(addd(dir[t], R));
            double w = ggx_D(dotd(R, h), a) * c * dw[t];
            for (int ch = 0; ch < 3; ++ch) acc[ch] += rgb[3 * (size_t)t + ch] * w;
            wsum += w;
        }
        for (int ch = 0; ch < 3; ++ch) spec[3 * (size_t)g + ch] = wsum > 0 ? acc[ch] / wsum : 0.0;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int ij = 0; ij < OR_LUT_N * OR_LUT_N; ++ij) {
        {
            int i = ij / OR_LUT_N, j = ij % OR_LUT_N;
            double nv = (i + 0.5) / OR_LUT_N, a = ggx_alpha((j + 0.5) / OR_LUT_N);
            d3 v = md3(sqrt(1.0 - nv * nv), 0.0, nv);
            double A = 0, B = 0;
            for (int p = 0; p < OR_LUT_M; ++p) {
                for (int q = 0; q < OR_LUT_M; ++q) {
                    double u1 = (p + 0.5) / OR_LUT_M, u2 = (q + 0.5) / OR_LUT_M;
                    double th = atan(a * sqrt(u1 / (1.0 - u1))), ph = 2.0 * PI_D * u2;
                    d3 h = md3(sin(th) * cos(ph), sin(th) * sin(ph), cos(th));
                    double vh = dotd(v, h);
                    if (vh <= 0) continue;
                    d3 l = addd(muld(h, 2.0 * vh), muld(v, -1.0));
                    if (l.z <= 0) continue;
                    double Gv = ggx_G1(nv, a) * ggx_G1(l.z, a) * vh / (nv * h.z);
                    double x = 1.0 - vh, x5 = x * x * x * x * x;
                    A += Gv * (1.0 - x5);
                    B += Gv * x5;
                }
            }
            lut[2 * (i * OR_LUT_N + j)] = A / (OR_LUT_M * OR_LUT_M);
            lut[2 * (i * OR_LUT_N + j) + 1] = B / (OR_LUT_M * OR_LUT_M);
        }
    }
    free(dir);
    free(dw);
}

/* Lookup of an equirectangular grid (cell centres) in direction w: bilinear between cell
 * centres (wrapping in phi); inside the half-cell caps around the poles, where phi loses
 * its meaning, linear in theta from the pole-row value towards the mean of that row at the
 * pole itself, so the lookup is continuous on the whole sphere. */
static void grid_lookup_d(const double* g, const float* gf, int W, int H, d3 w, double out[3]) {
    double ph = atan2(w.x, w.z);
    if (ph < 0) ph += 2.0 * PI_D;
    double th = atan2(sqrt(w.x * w.x + w.z * w.z), w.y);
    double u = ph / (2.0 * PI_D) * W - 0.5, v = th / PI_D * H - 0.5;
    double fi = floor(u), fu = u - fi;
    int i0 = ((int)fi % W + W) % W, i1 = (i0 + 1) % W;
    int j0, j1, pole = -1;
    double fv, tp = 1.0;
    if (v <= 0) { j0 = j1 = 0; fv = 0; pole = 0; tp = 2.0 * v + 1.0; }
    else if (v >= H - 1) { j0 = j1 = H - 1; fv = 0; pole = H - 1; tp = 2.0 * ((H - 0.5) - v); }
    else { j0 = (int)floor(v); j1 = j0 + 1; fv = v - j0; }
    for (int ch = 0; ch < 3; ++ch) {
#define OR_G(j, i) (g ? g[3 * ((size_t)(j) * W + (i)) + ch] : (double)gf[3 * ((size_t)(j) * W + (i)) + ch])
        out[ch] = (1 - fv) * ((1 - fu) * OR_G(j0, i0) + fu * OR_G(j0, i1)) + fv * ((1 - fu) * OR_G(j1, i0) + fu * OR_G(j1, i1));
        if (pole >= 0) {
            double mean = 0;
            for (int i = 0; i < W; ++i) mean += OR_G(pole, i);
            mean /= W;
            out[ch] = (1 - tp) * mean + tp * out[ch];
        }
#undef OR_G
    }
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* SplitSum(a, r, m, n, E) seen from direction v (unit, towards the viewer of the hit). */
static void splitsum(const or_prefiltered* E, const double a[3], double r, double m, d3 n, d3 v, double out[3]) {
    double nv = clampd(dotd(n, v), 1e-4, 1.0);
    d3 R = addd(muld(n, 2.0 * nv), muld(v, -1.0));
    double ed[3], e0[3], e1[3];
    grid_lookup_d(E->diff, NULL, OR_DIFF_W, OR_DIFF_H, n, ed);
    double t = clampd(r, 0.0, 1.0) * (OR_SPEC_LEVELS - 1);
    int l0 = (int)floor(t);
    if (l0 > OR_SPEC_LEVELS - 2) l0 = OR_SPEC_LEVELS - 2;
    double f = t - l0;
    if (l0 == 0) grid_lookup_d(NULL, E->rgb, E->W, E->H, R, e0);
    else grid_lookup_d(E->spec + 3 * (size_t)(l0 - 1) * OR_SPEC_W * OR_SPEC_H, NULL, OR_SPEC_W, OR_SPEC_H, R, e0);
    grid_lookup_d(E->spec + 3 * (size_t)l0 * OR_SPEC_W * OR_SPEC_H, NULL, OR_SPEC_W, OR_SPEC_H, R, e1);
    double x = clampd(nv * OR_LUT_N - 0.5, 0.0, OR_LUT_N - 1.0), y = clampd(clampd(r, 0.0, 1.0) * OR_LUT_N - 0.5, 0.0, OR_LUT_N - 1.0);
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < OR_LUT_N ? x0 + 1 : x0, y1 = y0 + 1 < OR_LUT_N ? y0 + 1 : y0;
    double fx = x - x0, fy = y - y0, AB[2];
    for (int k = 0; k < 2; ++k)
        AB[k] = (1 - fx) * ((1 - fy) * E->lut[2 * (x0 * OR_LUT_N + y0) + k] + fy * E->lut[2 * (x0 * OR_LUT_N + y1) + k]) +
                fx * ((1 - fy) * E->lut[2 * (x1 * OR_LUT_N + y0) + k] + fy * E->lut[2 * (x1 * OR_LUT_N + y1) + k]);
    for (int ch = 0; ch < 3; ++ch) {
        double kd = a[ch] * (1.0 - m), F0 = 0.04 * (1.0 - m) + a[ch] * m;
        double es = (1 - f) * e0[ch] + f * e1[ch];
        out[ch] = kd * ed[ch] + es * (F0 * AB[0] + AB[1]);
    }
}

void or_splitsum_many(int n, const double* a, const double* r, const double* m, const double* nrm, const double* v,
                      int W, int H, const float* rgb, const double* diff, const double* spec, const double* lut,
                      double* out) {
    or_prefiltered E = {W, H, rgb, diff, spec, lut};
    for (int i = 0; i < n; ++i)
        splitsum(&E, a + 3 * i, r[i], m[i], md3(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]),
                 md3(v[3 * i], v[3 * i + 1], v[3 * i + 2]), out + 3 * i);
}

/* Trace_attr (Eq. 14), Gaussian backend: the hits and order of Trace (Eq. 8); V_r = the
 * final transmittance; a_r, r_r, m_r = T_k a_k-weighted means of the surfels' albedo,
 * roughness, metallic; n_r = normalised weighted sum of their normals turned towards the
 * ray origin.  No hit: V_r = 1 and zero attributes. */
static void trace_attr_one(const or_scene* sc, const surf_pre* pre, const or_params* P, f3 o32, f3 d32,
                           ray_ws* ws, double* V, double a[3], double* r, double* m, double n[3], uint32_t* flags) {
    int nh = collect_hits(sc, pre, P, o32, d32, &ws->buf, &ws->cap, flags);
    ws_ensure(ws, nh + 1);
    double T;
    int K = composite_count(ws->buf, nh, P, ws->Tk, &T, flags);
    double wsum = 0, acc[3] = {0, 0, 0}, ra = 0, ma = 0;
    d3 nacc = md3(0, 0, 0);
    for (int k = 0; k < K; ++k) {
        const hit_t* h = &ws->buf[k];
        double w = ws->Tk[k] * h->alpha;
        for (int ch = 0; ch < 3; ++ch) acc[ch] += w * sc->albedo[3 * (size_t)h->id + ch];
        ra += w * sc->rough[h->id];
        ma += w * sc->metal[h->id];
        d3 ni = pre[h->id].n;
        if (h->den32 > 0.0f) ni = muld(ni, -1.0);
        nacc = addd(nacc, muld(ni, w));
        wsum += w;
    }
    *V = T;
    double nl = sqrt(dotd(nacc, nacc));
    for (int ch = 0; ch < 3; ++ch) a[ch] = wsum > 0 ? acc[ch] / wsum : 0.0;
    *r = wsum > 0 ? ra / wsum : 0.0;
    *m = wsum > 0 ? ma / wsum : 0.0;
    n[0] = nl > 0 ? nacc.x / nl : 0.0;
    n[1] = nl > 0 ? nacc.y / nl : 0.0;
    n[2] = nl > 0 ? nacc.z / nl : 0.0;
}

int or_trace_attr(const or_scene* sc, const or_params* P, int R, const float* ray_o, const float* ray_d,
                  double* out_V, double* out_a, double* out_r, double* out_m, double* out_n, uint32_t* out_flags,
                  int nthreads) {
    surf_pre* pre = precompute(sc);
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 8)
        for (int i = 0; i < R; ++i) {
            uint32_t fl = 0;
            f3 o = mk3(ray_o[3 * i], ray_o[3 * i + 1], ray_o[3 * i + 2]);
            f3 d = mk3(ray_d[3 * i], ray_d[3 * i + 1], ray_d[3 * i + 2]);
            trace_attr_one(sc, pre, P, o, d, &ws, out_V + i, out_a + 3 * (size_t)i, out_r + i, out_m + i,
                           out_n + 3 * (size_t)i, &fl);
            if (out_flags) out_flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    free(pre);
    return 0;
}

/* MIS relighting (Eq. 15 in Eq. 13): as or_shade_pixels with L_i = V_r L_new(w) +
 * (1 - V_r) SplitSum(a_r, r_r, m_r, n_r, E) seen from v = -w; indirect output = the mean
 * of (1 - V_r) SplitSum.  `env` is the novel map (its proposal tables drive the samples). */
/* Backend of the secondary query of Eq. 14: the Gaussian trace or the mesh closest hit. */
typedef struct {
    const or_scene* sc;
    const surf_pre* pre;
    const struct or_mesh_s* mesh;
} attr_backend;

static void mesh_attr_one(const struct or_mesh_s* m, const or_params* P, f3 o32, f3 d32, double* V, double a[3],
                          double* r, double* mm, double n[3], uint32_t* flags);

static void relight_pixels(const attr_backend* B, const or_params* P, const or_gbuf* gb, const or_env* env,
                           const double* diff, const double* spec, const double* lut, const or_sampling* S,
                           const int32_t* pixel_list, int n_pixels, double* out_color, double* out_vis,
                           double* out_ind, uint32_t* out_flags, int nthreads) {
    env_tab et;
    env_tab_build(env, &et);
    or_prefiltered E = {env->W, env->H, env->rgb, diff, spec, lut};
    int Nr = S->n_cos + S->n_ggx + S->n_env;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_pixels; ++i) {
            int p = pixel_list ? pixel_list[i] : i;
            double col[3] = {0, 0, 0}, vis = 0, ind[3] = {0, 0, 0};
            uint32_t fl = 0;
            if (gb->valid[p] && Nr > 0) {
                f3 x32, n32, b1, b2, wo32;
                d3 n, wo;
                pixel_setup(gb, p, &x32, &n32, &b1, &b2, &wo32, &n, &wo);
                double alb[3] = {gb->albedo[3 * (size_t)p], gb->albedo[3 * (size_t)p + 1], gb->albedo[3 * (size_t)p + 2]};
                for (int j = 0; j < Nr; ++j) {
                    sample_t s = draw_sample(S, &et, env, p, j, n32, b1, b2, wo32, gb->rough[p]);
                    if (!s.ok) continue;
                    double V, ar[3], rr, mr, nr[3];
                    if (B->mesh)
                        mesh_attr_one(B->mesh, P, x32, s.w32, &V, ar, &rr, &mr, nr, &fl);
                    else
                        trace_attr_one(B->sc, B->pre, P, x32, s.w32, &ws, &V, ar, &rr, &mr, nr, &fl);
                    sample_eval e;
                    sample_weights(env, &et, S, s.w32, n, wo, alb, gb->rough[p], gb->metal[p], &e);
                    double ss[3] = {0, 0, 0};
                    if (V < 1.0) {
                        d3 w = normd(f2d(s.w32));
                        splitsum(&E, ar, rr, mr, md3(nr[0], nr[1], nr[2]), muld(w, -1.0), ss);
                    }
                    for (int ch = 0; ch < 3; ++ch) {
                        double Lind = (1.0 - V) * ss[ch];
                        col[ch] += e.g[ch] * (V * e.Lenv[ch] + Lind);
                        ind[ch] += Lind;
                    }
                    vis += V;
                }
                for (int ch = 0; ch < 3; ++ch) { col[ch] /= Nr; ind[ch] /= Nr; }
                vis /= Nr;
            }
            for (int ch = 0; ch < 3; ++ch) { out_color[3 * (size_t)i + ch] = col[ch]; out_ind[3 * (size_t)i + ch] = ind[ch]; }
            out_vis[i] = vis;
            if (out_flags) out_flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    env_tab_free(&et);
}

int or_shade_relight(const or_scene* sc, const or_params* P, const or_gbuf* gb, const or_env* env,
                     const double* diff, const double* spec, const double* lut, const or_sampling* S,
                     const int32_t* pixel_list, int n_pixels, double* out_color, double* out_vis, double* out_ind,
                     uint32_t* out_flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    attr_backend B = {sc, pre, NULL};
    relight_pixels(&B, P, gb, env, diff, spec, lut, S, pixel_list, n_pixels, out_color, out_vis, out_ind, out_flags,
                   nthreads);
    free(pre);
    return 0;
}

/* ---------------------------------------------------------------- material and map adjoint (FP64) */

/* Partial derivatives of the BRDF (Eq. 4-5; Lambert for brdf = 0) per channel with respect
 * to the albedo of that channel (dfa), the metallic weight (dfm) and the roughness (dfr),
 * alpha = max(r^2, 1e-4) (no roughness derivative where the clamp holds). */
static void brdf_partials(d3 wo, d3 wi, d3 n, const double* alb, double rough, double metal, int brdf,
                          double dfa[3], double dfm[3], double dfr[3]) {
    for (int ch = 0; ch < 3; ++ch) {
        dfa[ch] = (brdf == 0 ? 1.0 : 1.0 - metal) / PI_D;
        dfm[ch] = brdf == 0 ? 0.0 : -alb[ch] / PI_D;
        dfr[ch] = 0.0;
    }
    if (brdf == 0) return;
    double won = dotd(wo, n), win = dotd(wi, n);
    if (!(won > 0.0) || !(win > 0.0)) return;
    d3 h = normd(addd(wo, wi));
    double hn = dotd(h, n), ih = dotd(wi, h);
    if (!(hn > 0.0)) return;
    double a = ggx_alpha(rough);
    double D = ggx_D(hn, a), Gi = ggx_G1(win, a), Go = ggx_G1(won, a);
    double DG = D * Gi * Go / (4.0 * win * won);
    double x = 1.0 - ih;
    if (x < 0) x = 0;
    double x5 = x * x * x * x * x;
    double dDG_dr = 0.0;
    if (rough * rough > 1e-4) {
        double t = hn * hn * (a * a - 1.0) + 1.0;
        double dD = 2.0 * a / (PI_D * t * t) * (1.0 - 2.0 * a * a * hn * hn / t);
        double si = sqrt(a * a + (1.0 - a * a) * win * win), so = sqrt(a * a + (1.0 - a * a) * won * won);
        double dGi = -2.0 * win / ((win + si) * (win + si)) * a * (1.0 - win * win) / si;
        double dGo = -2.0 * won / ((won + so) * (won + so)) * a * (1.0 - won * won) / so;
        dDG_dr = DG * (dD / D + dGi / Gi + dGo / Go) * 2.0 * rough;
    }
    for (int ch = 0; ch < 3; ++ch) {
        double F0 = 0.04 * (1.0 - metal) + metal * alb[ch];
        double F = F0 + (1.0 - F0) * x5;
        dfa[ch] += DG * metal * (1.0 - x5);
        dfm[ch] += DG * (1.0 - x5) * (alb[ch] - 0.04);
        dfr[ch] = dDG_dr * F;
    }
}

/* Adjoint of the MIS estimate (Eq. 13) and of the mean incident radiance of Eq. 16 with
 * respect to the environment map and the per-pixel materials, the sampled directions and
 * the proposal density q held fixed: given dL/dcolor and dL/dlight per listed pixel,
 *   dL/dL_env[t] += (1/N_r) sum_{j: w_j in t} (dL/dc g_j + dL/dlight) V_j,
 *   dL/da_c      += (1/N_r) sum_j dL/dc_c (df_c/da_c) (cos/q)_j L_i,j,c   (and m, r alike),
 * with L_i = V L_env + L_ind.  Map gradients accumulate in grad_env[H][W][3]; material
 * gradients are written per list entry (grad_albedo[n][3], grad_rough[n], grad_metal[n]). */
int or_backward_material(const or_scene* sc, const or_params* P, const or_gbuf* gb, const or_env* env,
                         const or_sampling* S, const int32_t* pixel_list, int n_pixels, const double* dL_dcolor,
                         const double* dL_dlight, double* grad_env, double* grad_albedo, double* grad_rough,
                         double* grad_metal, uint32_t* out_flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    env_tab et;
    env_tab_build(env, &et);
    int Nr = S->n_cos + S->n_ggx + S->n_env;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        ray_ws ws = {0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_pixels; ++i) {
            int p = pixel_list ? pixel_list[i] : i;
            double ga[3] = {0, 0, 0}, gr = 0, gm = 0;
            uint32_t fl = 0;
            if (gb->valid[p] && Nr > 0) {
                f3 x32, n32, b1, b2, wo32;
                d3 n, wo;
                pixel_setup(gb, p, &x32, &n32, &b1, &b2, &wo32, &n, &wo);
                double alb[3] = {gb->albedo[3 * (size_t)p], gb->albedo[3 * (size_t)p + 1], gb->albedo[3 * (size_t)p + 2]};
                const double* dc = dL_dcolor + 3 * (size_t)i;
                double dl[3] = {0, 0, 0};
                if (dL_dlight)
                    for (int ch = 0; ch < 3; ++ch) dl[ch] = dL_dlight[3 * (size_t)i + ch];
                for (int j = 0; j < Nr; ++j) {
                    sample_t s = draw_sample(S, &et, env, p, j, n32, b1, b2, wo32, gb->rough[p]);
                    if (!s.ok) continue;
                    sample_eval e;
                    eval_sample(sc, pre, P, env, &et, S, &ws, x32, s.w32, n, wo, alb, gb->rough[p], gb->metal[p],
                                &e, &fl);
                    double V = 1.0 - e.op;
                    d3 w = normd(f2d(s.w32));
                    double dfa[3], dfm[3], dfr[3];
                    brdf_partials(wo, w, n, alb, gb->rough[p], gb->metal[p], S->brdf, dfa, dfm, dfr);
                    for (int ch = 0; ch < 3; ++ch) {
                        double Li = V * e.Lenv[ch] + e.rgb[ch];
                        ga[ch] += dc[ch] * dfa[ch] * e.cq * Li;
                        gm += dc[ch] * dfm[ch] * e.cq * Li;
                        gr += dc[ch] * dfr[ch] * e.cq * Li;
                        if (grad_env) {
                            double v = (dc[ch] * e.g[ch] + dl[ch]) * V / Nr;
                            atomic_add_d(grad_env + 3 * ((size_t)e.row * env->W + e.col) + ch, v);
                        }
                    }
                }
                for (int ch = 0; ch < 3; ++ch) ga[ch] /= Nr;
                gr /= Nr;
                gm /= Nr;
            }
            if (grad_albedo)
                for (int ch = 0; ch < 3; ++ch) grad_albedo[3 * (size_t)i + ch] = ga[ch];
            if (grad_rough) grad_rough[i] = gr;
            if (grad_metal) grad_metal[i] = gm;
            if (out_flags) out_flags[i] = fl;
        }
        free(ws.buf);
        free(ws.Tk);
    }
    env_tab_free(&et);
    free(pre);
    return 0;
}

/* ---------------------------------------------------------------- mesh backend */
/* Sec. III-E: the mesh backend answers Eq. 14 with the closest hit of the ray against a
 * triangle mesh: a miss gives V_r = 1 and zero attributes; a hit gives V_r = 0 and the
 * barycentric interpolation of the hit triangle's per-vertex albedo, roughness, metallic
 * and normal (normalised, turned towards the ray origin).  Every triangle is tested; the
 * nearest t in (t_min, t_max) wins, equal t by triangle index.
 *
 * Which triangle a ray hits is an integer outcome, so (part A) it is decided in FP32 by
 * one fixed sequence of correctly rounded operations, the kernel's too: the watertight
 * ray/triangle test of Woop, Benthin and Wald (JCGT 2(1), 2013), two-sided:
 *   kz = the axis of the largest |d| (the first on ties), kx = kz+1 mod 3, ky = kx+1 mod 3;
 *   Sx = d[kx]/d[kz], Sy = d[ky]/d[kz], Sz = 1/d[kz];
 *   A = v0 - o, B = v1 - o, C = v2 - o; for P in {A, B, C}: Px = P[kx] - Sx P[kz],
 *   Py = P[ky] - Sy P[kz];
 *   U = Cx By - Cy Bx, V = Ax Cy - Ay Cx, W = Bx Ay - By Ax (two rounded products, then
 *   their rounded difference); if one of U, V, W is 0 all three are recomputed from the
 *   same FP32 operands by Kahan's difference of products in FP32 with fused multiply-adds
 *   (w = c d, e = fma(-c, d, w), (fma(a, b, -w)) + e; relative error below 2 ulp after
 *   Jeannerod, Louvet and Muller, Math. Comp. 2013, so its sign and zeros are exact);
 *   a hit needs U, V, W of one sign (zeros allowed) and det = (U + V) + W != 0;
 *   t = ((U (Sz A[kz]) + V (Sz B[kz])) + W (Sz C[kz])) / det in (t_min, t_max).
 * An edge shared by two triangles is evaluated from the same vertex values in both: the
 * plain difference to the same magnitude with opposite sign, and when it is 0 in one it is
 * 0 in both and both take the exact-sign difference, so no ray passes between them.  The barycentric
 * weights of (v0, v1, v2), continuous quantities, come from FP64 Moeller-Trumbore on the
 * chosen triangle. */
typedef struct or_mesh_s {
    int nv, nt;
    const float *pos;
    const int32_t* tri;
    const float *normal, *albedo, *rough, *metal;
} or_mesh;

static d3 crossd(d3 a, d3 b) { return md3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }

/* a b - c d by Kahan's algorithm (exact sign; see above). */
static inline float diff_prod(float a, float b, float c, float d) {
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

static inline float f3c(f3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* The ray's shear (kx, ky, kz, Sx, Sy, Sz). */
typedef struct { f3 o; int kx, ky, kz; float Sx, Sy, Sz; } wt_ray;

static wt_ray wt_setup(f3 o, f3 d) {
    wt_ray r;
    r.o = o;
    int kz = 0;
    if (fabsf(d.y) > fabsf(f3c(d, kz))) kz = 1;
    if (fabsf(d.z) > fabsf(f3c(d, kz))) kz = 2;
    r.kz = kz; r.kx = (kz + 1) % 3; r.ky = (r.kx + 1) % 3;
    float dz = f3c(d, kz);
    r.Sx = f3c(d, r.kx) / dz;
    r.Sy = f3c(d, r.ky) / dz;
    r.Sz = 1.0f / dz;
    return r;
}

/* 1 and (t, U, V, W, det) for a hit with t in (t_min, t_max); 0 otherwise. */
static int wt_hit(const wt_ray* r, const float* p0, const float* p1, const float* p2, float tmin, float tmax,
                  float* t_out, float* U_out, float* V_out, float* W_out, float* det_out) {
    f3 A = mk3(p0[0] - r->o.x, p0[1] - r->o.y, p0[2] - r->o.z);
    f3 B = mk3(p1[0] - r->o.x, p1[1] - r->o.y, p1[2] - r->o.z);
    f3 C = mk3(p2[0] - r->o.x, p2[1] - r->o.y, p2[2] - r->o.z);
    float Az = f3c(A, r->kz), Bz = f3c(B, r->kz), Cz = f3c(C, r->kz);
    float Ax = f3c(A, r->kx) - r->Sx * Az, Ay = f3c(A, r->ky) - r->Sy * Az;
    float Bx = f3c(B, r->kx) - r->Sx * Bz, By = f3c(B, r->ky) - r->Sy * Bz;
    float Cx = f3c(C, r->kx) - r->Sx * Cz, Cy = f3c(C, r->ky) - r->Sy * Cz;
    float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = diff_prod(Cx, By, Cy, Bx);
        V = diff_prod(Ax, Cy, Ay, Cx);
        W = diff_prod(Bx, Ay, By, Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;
    float det = (U + V) + W;
    if (det == 0.0f) return 0;
    float T = (U * (r->Sz * Az) + V * (r->Sz * Bz)) + W * (r->Sz * Cz);
    float t = T / det;
    if (!(t > tmin && t < tmax)) return 0;
    *t_out = t; *U_out = U; *V_out = V; *W_out = W; *det_out = det;
    return 1;
}

static void mesh_attr_one(const or_mesh* m, const or_params* P, f3 o32, f3 d32, double* V, double a[3],
                          double* r, double* mm, double n[3], uint32_t* flags) {
    (void)flags;
    wt_ray ray = wt_setup(o32, d32);
    float best = P->t_max, bU = 0, bV = 0, bW = 0, bdet = 1;
    int bt = -1;
    for (int t = 0; t < m->nt; ++t) {
        const float* p0 = m->pos + 3 * (size_t)m->tri[3 * t];
        const float* p1 = m->pos + 3 * (size_t)m->tri[3 * t + 1];
        const float* p2 = m->pos + 3 * (size_t)m->tri[3 * t + 2];
        float tt, U, Vv, W, det;
        if (!wt_hit(&ray, p0, p1, p2, P->t_min, best, &tt, &U, &Vv, &W, &det)) continue;
        best = tt; bU = U; bV = Vv; bW = W; bdet = det; bt = t;   /* strict <: the lower index keeps a tie */
    }
    if (bt < 0) {
        *V = 1.0;
        a[0] = a[1] = a[2] = 0; *r = 0; *mm = 0; n[0] = n[1] = n[2] = 0;
        return;
    }
    *V = 0.0;
    const int32_t* tv = m->tri + 3 * bt;
    /* the weights are continuous: FP64 Moeller-Trumbore on the chosen triangle */
    double w[3] = {(double)bU / bdet, (double)bV / bdet, (double)bW / bdet};
    {
        const float *p0 = m->pos + 3 * (size_t)tv[0], *p1 = m->pos + 3 * (size_t)tv[1], *p2 = m->pos + 3 * (size_t)tv[2];
        d3 v0 = md3(p0[0], p0[1], p0[2]), d = f2d(d32);
        d3 e1 = md3((double)p1[0] - v0.x, (double)p1[1] - v0.y, (double)p1[2] - v0.z);
        d3 e2 = md3((double)p2[0] - v0.x, (double)p2[1] - v0.y, (double)p2[2] - v0.z);
        d3 pv = crossd(d, e2), sv = addd(f2d(o32), muld(v0, -1.0)), qv = crossd(sv, e1);
        double det = dotd(e1, pv);
        if (det != 0.0) {
            w[1] = dotd(sv, pv) / det;
            w[2] = dotd(d, qv) / det;
            w[0] = 1.0 - w[1] - w[2];
        }
    }
    double na[3] = {0, 0, 0};
    a[0] = a[1] = a[2] = 0; *r = 0; *mm = 0;
    for (int k = 0; k < 3; ++k) {
        int vi = tv[k];
        for (int ch = 0; ch < 3; ++ch) {
            a[ch] += w[k] * m->albedo[3 * (size_t)vi + ch];
            na[ch] += w[k] * m->normal[3 * (size_t)vi + ch];
        }
        *r += w[k] * m->rough[vi];
        *mm += w[k] * m->metal[vi];
    }
    double nl = sqrt(na[0] * na[0] + na[1] * na[1] + na[2] * na[2]);
    double sgn = (na[0] * (double)d32.x + na[1] * (double)d32.y + na[2] * (double)d32.z) > 0 ? -1.0 : 1.0;
    for (int ch = 0; ch < 3; ++ch) n[ch] = nl > 0 ? sgn * na[ch] / nl : 0.0;
}

int or_mesh_trace_attr(const or_mesh* m, const or_params* P, int R, const float* ray_o, const float* ray_d,
                       double* out_V, double* out_a, double* out_r, double* out_m, double* out_n, uint32_t* out_flags,
                       int nthreads) {
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 8)
    for (int i = 0; i < R; ++i) {
        uint32_t fl = 0;
        f3 o = mk3(ray_o[3 * i], ray_o[3 * i + 1], ray_o[3 * i + 2]);
        f3 d = mk3(ray_d[3 * i], ray_d[3 * i + 1], ray_d[3 * i + 2]);
        mesh_attr_one(m, P, o, d, out_V + i, out_a + 3 * (size_t)i, out_r + i, out_m + i, out_n + 3 * (size_t)i, &fl);
        if (out_flags) out_flags[i] = fl;
    }
    return 0;
}

int or_shade_relight_mesh(const or_mesh* m, const or_params* P, const or_gbuf* gb, const or_env* env,
                          const double* diff, const double* spec, const double* lut, const or_sampling* S,
                          const int32_t* pixel_list, int n_pixels, double* out_color, double* out_vis,
                          double* out_ind, uint32_t* out_flags, int nthreads) {
    attr_backend B = {NULL, NULL, m};
    relight_pixels(&B, P, gb, env, diff, spec, lut, S, pixel_list, n_pixels, out_color, out_vis, out_ind, out_flags,
                   nthreads);
    return 0;
}

/* ========================================================================== *
 * Audit of the FP32 decisions.  The same rays with every decision of Part A    *
 * taken in FP64 instead -- the plane test and depth order of Eq. 7-8 from the  *
 * FP64 surfel frame, and the sampled direction of Sec. III-D from FP64 frames  *
 * and libm trigonometry (the texel of an environment sample is still chosen    *
 * from the FP32 tables with the same uniforms) -- so that the FP32 decision    *
 * reading can be checked against the FP64 one.  A ray whose two composited     *
 * lists differ must be near a boundary; the flags below say which, each with   *
 * an a-priori bound on the FP32 error of the quantity that decides.            *
 * ========================================================================== */

#define OR_AUDIT_TIE 16u        /* consecutive hits whose FP64 depths lie within their FP32 depth errors */
#define OR_AUDIT_PLANE_TIE 32u  /* such a tie between coplanar surfels: geometry leaves their order open   */
#define OR_AUDIT_RANGE 64u      /* a depth within its FP32 error of t_min or t_max                          */
#define OR_AUDIT_GRAZE 128u     /* |n.d| within its FP32 error of eps_nd                                   */
#define OR_AUDIT_HORIZON 256u   /* a sampled direction (or w_o for GGX) within 1e-6 of the horizon         */
#define OR_AUDIT_DIR 512u       /* an alpha_min decision flips between the FP32 and the FP64 direction     */

static const double U32_D = 5.9604644775390625e-08; /* 2^-24, unit roundoff of FP32 */

/* Duff et al.'s orthonormal basis in FP64. */
static void frame_d64(d3 n, d3* b1, d3* b2) {
    double sign = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n.z);
    double b = n.x * n.y * a;
    *b1 = md3(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
    *b2 = md3(b, sign + n.y * n.y * a, -n.y);
}

static d3 to_world_d64(d3 b1, d3 b2, d3 n, d3 l) {
    return md3(b1.x * l.x + b2.x * l.y + n.x * l.z, b1.y * l.x + b2.y * l.y + n.y * l.z,
               b1.z * l.x + b2.z * l.y + n.z * l.z);
}

/* The samplers of Part A (Malley's cosine sampling; Heitz's visible normals) in FP64. */
static d3 sample_cos_d64(d3 n, d3 b1, d3 b2, double u0, double u1) {
    double r = sqrt(u0), ph = 2.0 * PI_D * u1;
    double lz = 1.0 - u0;
    return to_world_d64(b1, b2, n, md3(r * cos(ph), r * sin(ph), sqrt(lz > 0.0 ? lz : 0.0)));
}

static int sample_ggx_d64(d3 n, d3 b1, d3 b2, d3 wo, double rough, double u0, double u1, d3* out, uint32_t* fl) {
    d3 v = md3(dotd(wo, b1), dotd(wo, b2), dotd(wo, n));
    if (fabs(v.z) <= 1e-6) *fl |= OR_AUDIT_HORIZON;
    if (!(v.z > 0.0)) return 0;
    double a = rough * rough;
    if (a < 1e-4) a = 1e-4;
    d3 vh = normd(md3(a * v.x, a * v.y, v.z));
    double lensq = vh.x * vh.x + vh.y * vh.y;
    d3 T1 = lensq > 0.0 ? md3(-vh.y / sqrt(lensq), vh.x / sqrt(lensq), 0.0) : md3(1.0, 0.0, 0.0);
    d3 T2 = md3(vh.y * T1.z - vh.z * T1.y, vh.z * T1.x - vh.x * T1.z, vh.x * T1.y - vh.y * T1.x);
    double r = sqrt(u0), ph = 2.0 * PI_D * u1;
    double t1 = r * cos(ph), t2 = r * sin(ph);
    double sh = 0.5 * (1.0 + vh.z);
    double q1 = 1.0 - t1 * t1;
    t2 = (1.0 - sh) * sqrt(q1 > 0.0 ? q1 : 0.0) + sh * t2;
    double q2 = q1 - t2 * t2;
    double nz = sqrt(q2 > 0.0 ? q2 : 0.0);
    d3 nh = md3(t1 * T1.x + t2 * T2.x + nz * vh.x, t1 * T1.y + t2 * T2.y + nz * vh.y, t1 * T1.z + t2 * T2.z + nz * vh.z);
    d3 ne = md3(a * nh.x, a * nh.y, nh.z > 0.0 ? nh.z : 0.0);
    ne = dotd(ne, ne) > 0.0 ? normd(ne) : md3(0.0, 0.0, 1.0);
    double d2 = 2.0 * dotd(v, ne);
    *out = to_world_d64(b1, b2, n, md3(d2 * ne.x - v.x, d2 * ne.y - v.y, d2 * ne.z - v.z));
    return 1;
}

/* Sample j of pixel p with FP64 directions (same uniforms and texel choice as draw_sample). */
static int draw_sample_d64(const or_sampling* S, const env_tab* et, const or_env* env, int pix, int j, d3 n, d3 b1,
                           d3 b2, d3 wo, double rough, d3* w, uint32_t* fl) {
    uint32_t ctr[4] = {(uint32_t)pix, (uint32_t)j, 0u, 0u}, key[2] = {S->seed_lo, S->seed_hi}, r[4];
    or_philox4x32_10(ctr, key, r);
    float u0 = unif24(r[0]), u1 = unif24(r[1]), u2 = unif24(r[2]), u3 = unif24(r[3]);
    int ok = 1;
    if (j < S->n_cos) {
        *w = sample_cos_d64(n, b1, b2, u0, u1);
    } else if (j < S->n_cos + S->n_ggx) {
        ok = sample_ggx_d64(n, b1, b2, wo, rough, u0, u1, w, fl);
    } else {
        int row = cdf_search(et->marg, env->H, u0);
        int col = cdf_search(et->cond + (size_t)row * (env->W + 1), env->W, u1);
        double ph = 2.0 * PI_D * (((double)col + u3) / env->W), th = PI_D * (((double)row + u2) / env->H);
        *w = md3(sin(th) * sin(ph), cos(th), sin(th) * cos(ph));
    }
    if (ok) {
        double c = dotd(*w, n);
        if (fabs(c) <= 1e-6) *fl |= OR_AUDIT_HORIZON;
        if (!(c > 0.0)) ok = 0;
    }
    return ok;
}

typedef struct { double tau, alpha, err; int id; } ahit_t;

static int ahit_cmp(const void* pa, const void* pb) {
    const ahit_t* a = (const ahit_t*)pa;
    const ahit_t* b = (const ahit_t*)pb;
    if (a->tau < b->tau) return -1;
    if (a->tau > b->tau) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct { double tau; uint32_t flag; } aevent_t;

typedef struct {
    hit_t* A; int capA;
    ahit_t* B; int capB;
    aevent_t* E; int capE;
    double* Tk; int capT;
} audit_ws;

static void* grow(void* p, int* cap, int need, size_t elem) {
    if (need <= *cap) return p;
    while (*cap < need) *cap = *cap ? 2 * *cap : 64;
    return realloc(p, elem * (size_t)*cap);
}

/* One ray: list A with the FP32 decisions of Part A along d32 (as trace_one), list B with
 * the plane test and depth order in FP64 along d64.  Both admit a hit by o G >= alpha_min
 * in FP64 along their own direction and composite with FP64 alphas.  Writes the first
 * maxl composited ids of each, the composited counts, and the audit flags. */
static void audit_ray(const or_scene* sc, const surf_pre* pre, const or_params* P, f3 o32, f3 d32, d3 d64,
                      audit_ws* ws, int maxl, int32_t* la, int32_t* na, int32_t* lb, int32_t* nb, uint32_t* flags) {
    const d3 o = f2d(o32), dA = f2d(d32);
    const double amin = P->alpha_min;
    int nA = 0, nB = 0, nE = 0;
    uint32_t fl = 0, dummy = 0;
    for (int i = 0; i < sc->n; ++i) {
        const double* m = sc->mu + 3 * (size_t)i;
        const d3 mu = md3(m[0], m[1], m[2]), n = pre[i].n, w = subd(mu, o);
        const double su = sc->scale[2 * (size_t)i], sv = sc->scale[2 * (size_t)i + 1];
        /* world B: FP64 plane test along d64, with the FP32 error bound of its quantities */
        const double den = dotd(n, d64), num = dotd(n, w);
        const double sn = fabs(n.x * w.x) + fabs(n.y * w.y) + fabs(n.z * w.z);
        const double sd = fabs(n.x * d64.x) + fabs(n.y * d64.y) + fabs(n.z * d64.z);
        const double dd = fabs(n.x) * fabs(dA.x - d64.x) + fabs(n.y) * fabs(dA.y - d64.y) +
                          fabs(n.z) * fabs(dA.z - d64.z);
        const double den_err = 16.0 * U32_D * sd + dd;
        const double tauB = den != 0.0 ? num / den : INFINITY;
        const double tau_err = fabs(den) > 0.0 ? (16.0 * U32_D * sn + fabs(tauB) * den_err) / fabs(den) +
                                                     4.0 * U32_D * fabs(tauB) : INFINITY;
        const int planeB = fabs(den) >= P->eps_nd && tauB > P->t_min && tauB < P->t_max;
        /* world A: the FP32 plane test of Part A along d32 */
        float tau32 = 0.f, den32 = 0.f;
        const int planeA = plane_test_f(pre[i].n32, pre[i].mu32, o32, d32, P->t_min, P->t_max, P->eps_nd, &tau32,
                                        &den32);
        if (!planeA && !planeB) continue;
        /* alpha along each direction (FP64 geometry) */
        double oG[2];
        const d3 dirs[2] = {dA, d64};
        for (int k = 0; k < 2; ++k) {
            const double nd = dotd(n, dirs[k]);
            const double t = num / nd;
            const d3 dp = subd(addd(o, muld(dirs[k], t)), mu);
            const double u = dotd(dp, pre[i].tu) / su, v = dotd(dp, pre[i].tv) / sv;
            oG[k] = sc->opacity[i] * exp(-0.5 * (u * u + v * v));
        }
        /* the plane decisions matter only for a surfel that the Gaussian admits */
        uint32_t pf = 0;
        if (oG[0] >= amin * (1.0 - 1e-4) || oG[1] >= amin * (1.0 - 1e-4)) {
            if (fabs(fabs(den) - P->eps_nd) <= den_err) pf |= OR_AUDIT_GRAZE;
            if (fabs(tauB - P->t_min) <= tau_err || fabs(tauB - P->t_max) <= tau_err) pf |= OR_AUDIT_RANGE;
        }
        if (pf) {
            ws->E = grow(ws->E, &ws->capE, nE + 1, sizeof(aevent_t));
            ws->E[nE++] = (aevent_t){tauB, pf};
        }
        uint32_t af = 0;
        if (fabs(oG[1] / amin - 1.0) < 1e-4) af |= OR_FLAG_ALPHA_MIN;
        if ((oG[0] >= amin) != (oG[1] >= amin)) af |= OR_AUDIT_DIR;
        if (af) {
            ws->E = grow(ws->E, &ws->capE, nE + 1, sizeof(aevent_t));
            ws->E[nE++] = (aevent_t){tauB, af};
        }
        const double amax = P->alpha_max;
        if (planeA && oG[0] >= amin) {
            ws->A = grow(ws->A, &ws->capA, nA + 1, sizeof(hit_t));
            hit_t* h = &ws->A[nA++];
            memset(h, 0, sizeof(*h));
            h->tau32 = tau32; h->id = i; h->alpha = oG[0] > amax ? amax : oG[0];
        }
        if (planeB && oG[1] >= amin) {
            ws->B = grow(ws->B, &ws->capB, nB + 1, sizeof(ahit_t));
            ws->B[nB++] = (ahit_t){tauB, oG[1] > amax ? amax : oG[1], tau_err, i};
        }
    }
    qsort(ws->A, (size_t)nA, sizeof(hit_t), hit_cmp);
    qsort(ws->B, (size_t)nB, sizeof(ahit_t), ahit_cmp);
    ws->Tk = grow(ws->Tk, &ws->capT, (nA > nB ? nA : nB) + 1, sizeof(double));
    double T;
    const int KA = composite_count(ws->A, nA, P, ws->Tk, &T, &dummy);
    /* list B: the same termination rule, T_min flags from the FP64 decisions */
    double TB = 1.0;
    int KB = 0;
    for (; KB < nB; ++KB) {
        TB *= 1.0 - ws->B[KB].alpha;
        if (fabs(TB / (double)P->T_min - 1.0) < 1e-4) fl |= OR_FLAG_T_MIN;
        if (TB < (double)P->T_min) { ++KB; break; }
    }
    /* events count up to the depth where either list stops (one hit beyond) */
    double stop = INFINITY;
    if (KB < nB || KA < nA) {
        double sb = KB < nB ? ws->B[KB].tau + ws->B[KB].err : INFINITY;
        double sa = KA < nA ? (double)ws->A[KA].tau32 : INFINITY;
        stop = sb > sa ? sb : sa;
        if (!isfinite(stop)) stop = INFINITY;
    }
    for (int e = 0; e < nE; ++e)
        if (ws->E[e].tau <= stop) fl |= ws->E[e].flag;
    for (int k = 0; k + 1 < nB && k <= KB; ++k) {
        const ahit_t* h0 = &ws->B[k];
        const ahit_t* h1 = &ws->B[k + 1];
        if (h1->tau - h0->tau <= h0->err + h1->err) {
            fl |= OR_AUDIT_TIE;
            const surf_pre* p0 = &pre[h0->id];
            const surf_pre* p1 = &pre[h1->id];
            const double* m0 = sc->mu + 3 * (size_t)h0->id;
            const double* m1 = sc->mu + 3 * (size_t)h1->id;
            const d3 dm = md3(m1[0] - m0[0], m1[1] - m0[1], m1[2] - m0[2]);
            if (fabs(dotd(p0->n, p1->n)) >= 1.0 - 1e-12 && fabs(dotd(p0->n, dm)) <= 1e-6) fl |= OR_AUDIT_PLANE_TIE;
        }
    }
    for (int k = 0; k < maxl; ++k) {
        la[k] = k < KA ? ws->A[k].id : -1;
        lb[k] = k < KB ? ws->B[k].id : -1;
    }
    *na = KA;
    *nb = KB;
    *flags = fl;
}

static void audit_ws_free(audit_ws* ws) { free(ws->A); free(ws->B); free(ws->E); free(ws->Tk); }

/* Audit of R given rays: d32 the FP32 direction both lists start from (d64 = d32 exactly
 * when ray_d64 is NULL). */
int or_audit_rays(const or_scene* sc, const or_params* P, int R, const float* ray_o, const float* ray_d,
                  const double* ray_d64, int maxl, int32_t* list_a, int32_t* n_a, int32_t* list_b, int32_t* n_b,
                  uint32_t* out_flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        audit_ws ws = {0};
#pragma omp for schedule(dynamic, 4)
        for (int r = 0; r < R; ++r) {
            f3 o = mk3(ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]);
            f3 d = mk3(ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]);
            d3 d64 = ray_d64 ? md3(ray_d64[3 * r], ray_d64[3 * r + 1], ray_d64[3 * r + 2]) : f2d(d);
            audit_ray(sc, pre, P, o, d, d64, &ws, maxl, list_a + (size_t)r * maxl, n_a + r,
                      list_b + (size_t)r * maxl, n_b + r, out_flags + r);
        }
        audit_ws_free(&ws);
    }
    free(pre);
    return 0;
}

/* Audit of the shading rays of a pixel list: slot i * N_r + j holds sample j of pixel
 * pixel_list[i], drawn by the FP32 sampler of Part A (list A) and by its FP64 restatement
 * (list B).  A slot without a sample on one side and one on the other gets an empty list
 * there; n_a = n_b = -1 marks a slot without a sample on both sides. */
int or_audit_pixels(const or_scene* sc, const or_params* P, const or_gbuf* gb, const or_env* env,
                    const or_sampling* S, const int32_t* pixel_list, int n_pixels, int maxl, int32_t* list_a,
                    int32_t* n_a, int32_t* list_b, int32_t* n_b, uint32_t* out_flags, int nthreads) {
    surf_pre* pre = precompute(sc);
    env_tab et;
    env_tab_build(env, &et);
    const int Nr = S->n_cos + S->n_ggx + S->n_env;
    int nt = nthreads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
    {
        audit_ws ws = {0};
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_pixels; ++i) {
            const int p = pixel_list[i];
            f3 x32, n32, b1, b2, wo32;
            d3 n, wo;
            pixel_setup(gb, p, &x32, &n32, &b1, &b2, &wo32, &n, &wo);
            d3 c1, c2;
            frame_d64(n, &c1, &c2);
            for (int j = 0; j < Nr; ++j) {
                const size_t s = (size_t)i * Nr + j;
                int32_t* la = list_a + s * maxl;
                int32_t* lb = list_b + s * maxl;
                uint32_t fl = 0;
                sample_t a = gb->valid[p] ? draw_sample(S, &et, env, p, j, n32, b1, b2, wo32, gb->rough[p])
                                          : (sample_t){mk3(0, 0, 0), 0};
                d3 w64 = md3(0, 0, 0);
                int okb = gb->valid[p] ? draw_sample_d64(S, &et, env, p, j, n, c1, c2, wo, gb->rough[p], &w64, &fl) : 0;
                if (!a.ok && !okb) {
                    for (int k = 0; k < maxl; ++k) la[k] = lb[k] = -1;
                    n_a[s] = n_b[s] = -1;
                    out_flags[s] = fl;
                    continue;
                }
                uint32_t rf = 0;
                int32_t ka = 0, kb = 0;
                audit_ray(sc, pre, P, x32, a.ok ? a.w32 : mk3((float)w64.x, (float)w64.y, (float)w64.z),
                          okb ? w64 : f2d(a.w32), &ws, maxl, la, &ka, lb, &kb, &rf);
                if (!a.ok) { for (int k = 0; k < maxl; ++k) la[k] = -1; ka = 0; }
                if (!okb) { for (int k = 0; k < maxl; ++k) lb[k] = -1; kb = 0; }
                n_a[s] = ka;
                n_b[s] = kb;
                out_flags[s] = fl | rf;
            }
        }
        audit_ws_free(&ws);
    }
    env_tab_free(&et);
    free(pre);
    return 0;
}

/* Sample j of a pixel drawn by the audit's FP64 sampler (for checks against the FP32
 * sampler of or_sample_direction).  Returns 1 when a direction was drawn above the horizon;
 * *flags gets OR_AUDIT_HORIZON for a direction (or GGX w_o) within 1e-6 of the horizon. */
int or_sample_direction_d64(const or_sampling* S, const or_env* env, const float* pos, const float* nrm,
                            const float* eye, float rough, int pix, int j, double* w_out, uint32_t* flags) {
    env_tab et;
    env_tab_build(env, &et);
    d3 n = normd(md3(nrm[0], nrm[1], nrm[2])), b1, b2;
    frame_d64(n, &b1, &b2);
    d3 wo = normd(md3((double)eye[0] - pos[0], (double)eye[1] - pos[1], (double)eye[2] - pos[2]));
    d3 w = md3(0, 0, 0);
    uint32_t fl = 0;
    int ok = draw_sample_d64(S, &et, env, pix, j, n, b1, b2, wo, rough, &w, &fl);
    env_tab_free(&et);
    w_out[0] = w.x; w_out[1] = w.y; w_out[2] = w.z;
    *flags = fl;
    return ok;
}
