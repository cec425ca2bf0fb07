/*
 * grt.h -- C ABI of libgrt: differentiable 2D Gaussian ray tracing (2DGRT) of secondary
 * rays against 2D Gaussian surfels, with multiple-importance-sampled shading, for
 * NVIDIA B300 (sm_103a).
 *
 * Paper: "IRGS++" (arXiv 2607.22780).  The operations below are the paper's
 *   Trace(r_o, r_d) -> (c_rt, o_rt)                      Sec. III-B, Eq. 7-8
 *   G-buffer {D, N, A, R, M} with normalised weights      Sec. III-C, Eq. 9
 *   L_i = V L_dir + L_ind, (L_ind, 1-V) = Trace(x, w)     Eq. 10-11
 *   c_pbr = (1/N_r) sum g(w)/q(w), MIS mixture q           Eq. 12-13, Sec. III-D
 *   metallic microfacet BRDF                               Eq. 4-5
 *   gradients through Trace                                Sec. III-B ("Trace operator")
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous, row-major,
 *     FP32 unless stated.  Host-side structs (grt_surfels, grt_trace_params, ...) are
 *     read during the call only.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every call is
 *     asynchronous on that stream unless stated.
 *   - Return value: GRT_OK (0) or a GRT_ERR_* code; grt_last_error() gives the message
 *     of the calling thread's last failure.  No call throws or aborts.
 *   - Device-side anomalies (traversal stack overflow, non-finite inputs) set a status
 *     word in the BVH that grt_bvh_status() reads back.
 *   - Gradient outputs accumulate (+=) into caller-zeroed arrays.
 */
#ifndef GRT_H
#define GRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRT_OK 0
#define GRT_ERR_ARG 1         /* invalid argument (null pointer, bad size, bad enum) */
#define GRT_ERR_OOM 2         /* device allocation failed                            */
#define GRT_ERR_CUDA 3        /* a CUDA runtime call or kernel launch failed         */
#define GRT_ERR_OVERFLOW 4    /* device status: traversal stack overflow             */
#define GRT_ERR_TIMEOUT 5     /* a bounded device wait gave up                       */
#define GRT_ERR_UNSUPPORTED 6 /* option not built in (e.g. k not in {4,8,16,32})     */

/* Device status bits reported by grt_bvh_status(). */
#define GRT_STATUS_STACK_OVERFLOW 1  /* a traversal stack filled; deeper nodes were dropped  */
#define GRT_STATUS_NONFINITE 2  /* a ray with a NaN or infinite origin or direction was traced as a miss */
#define GRT_STATUS_BAD_TREE 4   /* node reference out of range or walk longer than the tree */
#define GRT_STATUS_BAD_INDEX 8  /* a pixel index outside the G-buffer was skipped            */

/* Surfels (Sec. III-A "2D Gaussian splatting"; Sec. III-B "Bounding proxy").
 * mu[n][3] centre; quat[n][4] rotation (w,x,y,z), any non-zero norm, normalised inside:
 * the columns of R(q/|q|) are (t_u, t_v, n); scale[n][2] = (s_u, s_v) > 0;
 * opacity[n] = o in (0,1]; color[n][color_dim]: color_dim 3 = RGB outgoing radiance,
 * 48 = real SH degree 3 laid out [16 basis][3 channels], evaluated at the ray direction
 * as max(0, SH + 0.5); albedo[n][3], rough[n], metal[n] feed only the primary G-buffer
 * and may be NULL otherwise. */
typedef struct {
    int32_t n;
    int32_t color_dim;
    const float* mu;
    const float* quat;
    const float* scale;
    const float* opacity;
    const float* color;
    const float* albedo;
    const float* rough;
    const float* metal;
} grt_surfels;

/* Trace parameters (Eq. 7-8).  A hit is admitted iff |n.d| >= eps_nd, tau in
 * (t_min, t_max) and o*G >= alpha_min; alpha = min(o*G, alpha_max).  Hits are
 * composited in ascending (tau, surfel id) and a ray stops after the hit that drops its
 * transmittance below T_min.  k is the per-ray k-buffer size (4, 8, 16 or 32); results
 * do not depend on k, only speed does.  build_passes (0 to GRT_MAX_BUILD_PASSES) is read
 * by the tree builds only: the number of treelet-restructuring passes applied to the
 * radix tree before its 4-wide collapse (0 = the plain LBVH; each pass costs about
 * 0.5 ms per 300k surfels and lowers the traversal's node visits: 32.4 -> 25.7 -> 25.3
 * per secondary ray on a 300k-surfel scene); like k, it changes speed, not results.
 * gbuffer_k is the k-buffer size of grt_gbuffer_primary's walk: 4, 8, 16 or 32, or 0 to
 * choose by frame size -- 32 for frames of at most GRT_GBUFFER_SMALL_FRAME pixels, k for
 * larger ones.  Most of a small frame's time is the tail of its slowest warps, which
 * fewer k-buffer rounds shorten (300k surfels, 200x200: 0.71 ms at k = 16, 0.57 ms at
 * 32; 800x800: 1.16 and 1.13 ms), while a large frame is bound by throughput, which
 * k = 16's five blocks per SM serve better (1024x1024: 1.52 against 1.61 ms; 1600x1600:
 * 2.99 against 3.46 ms).  Results do not depend on it.  Typical: 1/255, 0.99, 0.01, 3e38, 1e-4, 1e-6, 16, 1, 0. */
#define GRT_MAX_BUILD_PASSES 4
#define GRT_GBUFFER_SMALL_FRAME (3 << 18)
typedef struct {
    float alpha_min, alpha_max, t_min, t_max, T_min, eps_nd;
    int32_t k;
    int32_t build_passes;
    int32_t gbuffer_k;
} grt_trace_params;

typedef struct grt_bvh grt_bvh; /* opaque: LBVH nodes + packed surfel records (device) */

typedef struct {
    int32_t n_surfels;
    int32_t n_nodes;        /* internal nodes, n_surfels - 1 */
    size_t device_bytes;    /* bytes the BVH holds on the device */
    float bounds[6];        /* scene AABB of the surfel bounds (lo xyz, hi xyz); valid after sync */
} grt_bvh_info_t;

/* Build a linear BVH (Morton codes of the cut-off-ellipse AABB centres, LSD radix
 * sort, hierarchy from the sorted codes, bottom-up box refit, params->build_passes passes
 * of treelet restructuring, and the collapse to 4-wide nodes by the surface-area-optimal
 * cut) over the surfels.  Each surfel is bounded by the exact box of its alpha_min ellipse
 * u^2+v^2 <= 2 ln(o/alpha_min) (the same region the icosahedron proxy of Eq. 6 encloses),
 * padded for FP32.  Only params->alpha_min and params->build_passes are read.  Allocates
 * device memory; asynchronous on `stream`.
 * *out stays valid until grt_bvh_destroy().  n == 0 is allowed (every ray misses). */
int grt_build_bvh(const grt_surfels* surfels, const grt_trace_params* params, grt_bvh** out,
                  void* stream);

/* Recompute boxes and packed records after the surfel parameters changed, keeping the
 * topology (the caller keeps n and color_dim).  Asynchronous on `stream`. */
int grt_refit_bvh(grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                  void* stream);

/* Full rebuild (Morton codes, sort, hierarchy, refit, restructuring passes, collapse, as
 * grt_build_bvh) into the existing BVH after the surfels moved; same n.  Sort scratch
 * comes from the stream-ordered pool. */
int grt_rebuild_bvh(grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                    void* stream);

/* Allocation-free rebuild (no counterpart in the paper; a library-integration need).
 * Some callers cannot let a library allocate device memory: a host application that
 * owns and pre-reserves the whole device budget (a renderer or engine with a fixed
 * memory plan, a process whose own allocator enforces a hard cap) sees any cudaMalloc or
 * pool allocation inside a call as a failure risk at an arbitrary moment and as memory
 * it cannot account for.  This call does what grt_rebuild_bvh does -- Morton codes,
 * sort, hierarchy, refit, into the existing BVH that the caller already owns -- without
 * allocating: its sort scratch is a fixed array compiled into the library (about 15 MB
 * for GRT_NOALLOC_MAX_SURFELS surfels), which every device that loads libgrt keeps until
 * the process exits.
 *   - n > GRT_NOALLOC_MAX_SURFELS is rejected with GRT_ERR_ARG before any device work.
 *   - The device that built `bvh` must be current; a call made while another device is
 *     current is rejected with GRT_ERR_ARG.
 *   - The first call on a device looks up the scratch array's device address (with that
 *     device current); make that first call before any stream capture.  The address is
 *     cached per device for the life of the process: after cudaDeviceReset the library
 *     (and every BVH built before the reset) is no longer usable on that device.
 *   - All calls share the one array: calls that may overlap on the GPU (other streams,
 *     other host threads) race on it and must be serialised by the caller.
 * Asynchronous on `stream`; results are identical to grt_rebuild_bvh. */
#define GRT_NOALLOC_MAX_SURFELS 524288
int grt_rebuild_bvh_noalloc(grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                            void* stream);

/* Synchronises the device, then frees the BVH.  NULL is ignored. */
void grt_bvh_destroy(grt_bvh* bvh);

int grt_bvh_info(const grt_bvh* bvh, grt_bvh_info_t* info);

/* Synchronises `stream`, returns the device status bits accumulated since the last call
 * in *status and clears them. */
int grt_bvh_status(grt_bvh* bvh, int32_t* status, void* stream);

/* Trace operator of Eq. 8 for R rays: ray_o[R][3], ray_d[R][3] (unit length) ->
 * out_rgb[R][3] = c_rt, out_opacity[R] = o_rt.  Optional (may be NULL): out_hits
 * [R][max_hits] ids of the composited surfels in order (-1 padded), out_nhits[R] number
 * composited.  Uses the surfels the BVH was built or refit from (mu, quat, scale,
 * opacity baked into the BVH; color read from `surfels` at composite time). */
int grt_trace_forward(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                      const float* ray_o, const float* ray_d, int32_t R, float* out_rgb,
                      float* out_opacity, int32_t* out_hits, int32_t max_hits, int32_t* out_nhits,
                      void* stream);

/* Gradient buffers, each accumulated (+=): mu[n][3], quat[n][4] (w.r.t. the
 * unnormalised quaternion), scale[n][2], opacity[n], color[n][color_dim].  Any pointer
 * may be NULL to skip that parameter. */
typedef struct {
    float* mu;
    float* quat;
    float* scale;
    float* opacity;
    float* color;
} grt_grads;

/* Adjoint of Eq. 8 for R rays given dL/dc_rt (dL_drgb[R][3]) and dL/do_rt
 * (dL_dopacity[R]; may be NULL).  Hit lists are recomputed, never stored. */
int grt_trace_backward(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                       const float* ray_o, const float* ray_d, int32_t R, const float* dL_drgb,
                       const float* dL_dopacity, const grt_grads* grads, void* stream);

/* Primary G-buffer (Eq. 9, traced along camera rays instead of rasterised): camera =
 * host array {eye xyz, target xyz, up xyz, tan(fovy/2)}, pinhole, pixel centres, row 0
 * at the top.  Per pixel p = y*W + x: pos[p][3] = eye + D d, normal[p][3] = normalised
 * blend of camera-facing surfel normals, albedo[p][3], rough[p], metal[p], alpha[p] =
 * o_rt, depth[p] = D, valid[p] = alpha >= 0.5.  Invalid pixels hold zeros.  Needs
 * albedo/rough/metal in `surfels`. */
int grt_gbuffer_primary(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                        const float camera[10], int32_t W, int32_t H, float* pos, float* normal,
                        float* albedo, float* rough, float* metal, float* alpha, float* depth,
                        int32_t* valid, void* stream);

/* Environment map (Eq. 10, L_dir): equirectangular rgb[H][W][3]; texel (row, col)
 * spans theta in [pi row/H, pi (row+1)/H] from +y and phi in [2 pi col/W, 2 pi (col+1)/W]
 * about +y, direction (sin t sin p, cos t, sin t cos p); nearest-texel lookup.
 * `tables` is a device buffer of grt_env_tables_bytes(W, H) bytes filled by
 * grt_env_prepare(): texel radiance with its selection probability and the FP32
 * marginal/conditional CDFs of the luminance distribution (environment proposal p_e of
 * Sec. III-D). */
typedef struct {
    int32_t W, H;
    const void* tables;
} grt_envmap;

size_t grt_env_tables_bytes(int32_t W, int32_t H);
int grt_env_prepare(const float* rgb, int32_t W, int32_t H, void* tables, void* stream);

/* G-buffer consumed by shading (Sec. III-C "Shading state"): device arrays over W*H
 * pixels as written by grt_gbuffer_primary(); eye = camera position (host values). */
typedef struct {
    const float* pos;
    const float* normal;
    const float* albedo;
    const float* rough;
    const float* metal;
    const int32_t* valid;
    float eye[3];
    int32_t W, H;
} grt_gbuffer;

/* MIS allocation (Sec. III-D, Eq. 13): sample j of a pixel is cosine for j < n_cos,
 * GGX visible-normal for j < n_cos + n_ggx, environment otherwise; N_r = n_cos + n_ggx +
 * n_env <= 1024.  brdf: 0 = Lambert a/pi, 1 = metallic microfacet (Eq. 4-5).  Random
 * numbers: Philox4x32-10 with key (seed lo, seed hi) and counter (pixel index, j, 0, 0). */
typedef struct {
    int32_t n_cos, n_ggx, n_env;
    int32_t brdf;
    uint64_t seed;
} grt_sampling;

/* Workspace convention of the shading calls (grt_shade_pixels, grt_shade_pixels_save,
 * grt_shade_backward, grt_shade_backward_saved, grt_shade_batch): the last two arguments
 * before `stream` are an optional device workspace and its size in bytes.  NULL: the call
 * takes its scratch from the device's stream-ordered pool (cudaMallocAsync) and returns it
 * on `stream` before it returns.  Non-NULL: a caller-owned device buffer, 256-byte aligned
 * and at least the size the matching *_workspace_size call reports (else GRT_ERR_ARG, no
 * device work), used instead of the pool; the call reads and writes it on `stream` only, so
 * the caller may reuse it for the next call on the same stream.  The contents need no
 * initialisation and are meaningless afterwards.  The other calls (G-buffer, relighting,
 * material adjoint, tree builds) take their scratch from the pool. */

/* Bytes of workspace of grt_shade_pixels and grt_shade_batch over n_rays ray slots (the
 * sum of n_pixels x N_r over the requests): direction and traced (c_rt, T) per slot (32
 * bytes), a ray counter, and the order in which the walk takes the rays (12 bytes per slot
 * and 4.2 MB of bucket counters).  grt_shade_pixels_save keeps directions and totals in its
 * `saved` buffer, so this size bounds its workspace too.  0 (with the error text) for
 * n_rays < 0. */
size_t grt_shade_workspace_size(int64_t n_rays);

/* Bytes of workspace of grt_shade_backward (saved = 0: the recomputing form, one or two
 * chunk buffers of at most 8M rays holding directions, totals, a transient record of 64
 * hits per ray, adjoints and the ray order) or grt_shade_backward_saved (saved = 1: the
 * adjoint per ray and the list of rays longer than the record, 24 bytes per ray slot).
 * 0 (with the error text) for invalid arguments. */
size_t grt_shade_backward_workspace_size(int32_t n_pixels, const grt_sampling* sampling, int32_t saved);

/* Shade pixels (Eq. 13): out_color[i][3] = (1/N_r) sum g/q, out_vis[i] = (1/N_r) sum V,
 * out_ind[i][3] = (1/N_r) sum L_ind for i < n_pixels, pixel index pixel_list[i]
 * (NULL = all W*H pixels in order).  Samples below the horizon count V = L_ind = 0.
 * out_vis / out_ind may be NULL.  Ray buffers (32 bytes per ray slot, pixels x N_r) and the
 * order in which the walk takes the rays (12 bytes per slot) live in `workspace`
 * (grt_shade_workspace_size(n_pixels x N_r) bytes) or, with workspace NULL, in the
 * stream-ordered pool. */
int grt_shade_pixels(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                     const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                     const int32_t* pixel_list, int32_t n_pixels, float* out_color, float* out_vis,
                     float* out_ind, void* workspace, size_t workspace_bytes, void* stream);

/* Adjoint of grt_shade_pixels with respect to the surfels, given dL_dcolor[n_pixels][3]
 * and optional dL_dvis[n_pixels], dL_dind[n_pixels][3] (NULL = 0).  Nothing is kept from
 * the forward pass: the same samples are drawn and traced again, in chunks of at most 8M
 * rays whose hit lists (first 64 hits per ray) live only during the call (two chunks in
 * flight on two library streams, ~14 GB of pool memory at most), then replayed; rays with
 * more hits are traversed again.  Gradients accumulate (+=) into grads. */
int grt_shade_backward(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                       const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                       const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                       const float* dL_dvis, const float* dL_dind, const grt_grads* grads,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Stored forward record for the backward pass (Sec. III-B: the loss gradient flows back
 * through the secondary trace into the surfels).  grt_shade_pixels_save does what
 * grt_shade_pixels does and also keeps, in the caller's device buffer `saved` (256-byte
 * aligned, at least grt_shade_saved_bytes() bytes), every secondary ray's sampled
 * direction, its traced (c_rt, T) and its first max_hits composited hits (surfel id,
 * tau, alpha) in compositing order: 36 + 12 max_hits bytes per ray.  Rays with more than
 * max_hits hits keep their next 192 hits in an overflow area of one slot per 256 rays (at
 * least 64 slots, 2,308 bytes each), so that the backward replays them without a traversal;
 * only rays longer than that, or beyond the slots, are traced again.
 * grt_shade_backward_saved is grt_shade_backward without the resampling and the forward
 * re-trace: rays with at most max_hits hits are replayed from the record, longer ones are
 * traced again.  Gradients equal grt_shade_backward's up to the order of the float atomic
 * additions.  The backward call must get the same bvh, surfels, params, gbuffer, env,
 * sampling, pixel_list, n_pixels and max_hits as the save call, with the surfels unchanged
 * in between (a replayed surfel id outside the scene is skipped and reported as
 * GRT_STATUS_BAD_INDEX).  grt_shade_saved_bytes returns 0 (and sets the error text) for
 * invalid arguments; max_hits is in [0, GRT_MAX_SAVED_HITS].  The save call's workspace
 * (or pool scratch) holds the walk's ray order, 12 bytes per ray slot. */
#define GRT_MAX_SAVED_HITS 64
size_t grt_shade_saved_bytes(int32_t n_pixels, const grt_sampling* sampling, int32_t max_hits);
int grt_shade_pixels_save(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                          const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                          const int32_t* pixel_list, int32_t n_pixels, float* out_color, float* out_vis,
                          float* out_ind, int32_t max_hits, void* saved, size_t saved_bytes, void* workspace,
                          size_t workspace_bytes, void* stream);
int grt_shade_backward_saved(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                             const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                             const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                             const float* dL_dvis, const float* dL_dind, int32_t max_hits, const void* saved,
                             size_t saved_bytes, const grt_grads* grads, void* workspace, size_t workspace_bytes,
                             void* stream);

/* grt_shade_pixels plus out_light[n_pixels][3] = (1/N_r) sum_j L_i(w_j), the mean incident
 * radiance of the lighting regulariser (Eq. 16), L_i = V L_env + L_ind (samples below the
 * horizon count 0). */
int grt_shade_pixels_light(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                           const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                           const int32_t* pixel_list, int32_t n_pixels, float* out_color, float* out_vis,
                           float* out_ind, float* out_light, void* stream);

/* Adjoint of the estimate (Eq. 13) and of the mean incident radiance (Eq. 16) with respect
 * to the environment map and the per-pixel materials of the G-buffer (the paper optimises
 * lighting and materials jointly, Sec. III-F), the sampled directions and the proposal
 * density q held fixed.  Given dL_dcolor[n_pixels][3] and optional dL_dlight[n_pixels][3]:
 *   grad_env[H][W][3]    += (1/N_r) sum_j (dL/dc g_j + dL/dlight) V_j at the texel of w_j,
 *   grad_albedo[n][3], grad_rough[n], grad_metal[n] += (1/N_r) sum_j dL/dc (df/dx) (cos/q)_j L_i,j
 * (per list entry; no roughness gradient where max(r^2, 1e-4) clamps).  Every gradient
 * pointer may be NULL; all accumulate.  The samples are drawn and traced again (44 bytes per
 * ray slot of pool scratch during the call); map gradients are float atomics. */
int grt_shade_backward_material(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                                const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                                const int32_t* pixel_list, int32_t n_pixels, const float* dL_dcolor,
                                const float* dL_dlight, float* grad_env, float* grad_albedo, float* grad_rough,
                                float* grad_metal, void* stream);

/* One shading request of a batch (same meaning as the grt_shade_pixels arguments).
 * With pixel_list NULL, output i shades pixel pixel_offset + i (a contiguous slice of
 * the image, so a long request can be split over several launches). */
typedef struct {
    const grt_bvh* bvh;
    const grt_surfels* surfels;
    grt_gbuffer gbuffer;
    grt_envmap env;
    grt_sampling sampling;
    const int32_t* pixel_list;
    int32_t n_pixels;
    int32_t pixel_offset;
    float* out_color;
    float* out_vis;
    float* out_ind;
} grt_shade_request;

#define GRT_MAX_BATCH 48

/* Shade up to GRT_MAX_BATCH requests (possibly on different scenes, environment maps,
 * resolutions and sample counts) in one wavefront pass: every request's samples go into
 * one ray list, one persistent trace launch serves them all, and each pixel is summed in
 * a fixed order.  Each request's outputs are bit-identical to shading it alone with
 * grt_shade_pixels.  Ray buffers (44 bytes per ray slot) live in `workspace`
 * (grt_shade_workspace_size of the requests' total ray slots) or, with workspace NULL, in the
 * stream-ordered pool. */
int grt_shade_batch(const grt_shade_request* requests, int32_t n_requests,
                    const grt_trace_params* params, void* workspace, size_t workspace_bytes, void* stream);

/* Relighting under a novel map (Sec. III-E).
 * Trace_attr (Eq. 14), Gaussian backend: the hits of Trace (Eq. 8), same order and
 * termination, blended with w_k = T_k a_k into out_albedo[R][3], out_rough[R], out_metal[R]
 * (weighted means) and out_normal[R][3] (normalised weighted sum of the surfel normals turned
 * towards the ray origin); out_vis[R] = V_r = final transmittance.  No hit: V_r = 1, zeros.
 * Surfels need quat, albedo, rough and metal. */
int grt_trace_attr(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                   const float* ray_o, const float* ray_d, int32_t R, float* out_vis, float* out_albedo,
                   float* out_rough, float* out_metal, float* out_normal, void* stream);

/* Prefiltered form E of a novel map rgb[H][W][3] (Eq. 15 leaves it open): E_diff(n) = (1/pi)
 * sum_t L_t max(0, n.w_t) dW_t on a 32 x 16 equirectangular grid; E_spec(R, r) = GGX-lobe
 * (n = v = R) normalised texel average for r = 0.2, 0.4, ..., 1 on 64 x 32 grids (r = 0 is
 * the map itself); the split-sum BRDF table A, B(n.v, r) of the specular lobe of Eq. 5 on 32 x
 * 32 cell centres (256 x 256 midpoint rule over GGX half vectors); the top and bottom row
 * means of each grid and of the map, towards which lookups fade inside the polar half-cell
 * caps (phi has no meaning at a pole).  out: caller-owned device
 * buffer of grt_env_prefilter_bytes() bytes, 16-byte aligned; a pool scratch of 16 bytes per
 * texel is used during the call. */
size_t grt_env_prefilter_bytes(void);
int grt_env_prefilter(const float* rgb, int32_t W, int32_t H, void* out, size_t out_bytes, void* stream);

/* MIS relighting (Eq. 15 substituted into Eq. 13): as grt_shade_pixels, with env the novel
 * map (its proposal tables drive the samples) and, per sample, L_i = V_r L_new(w) + (1 - V_r)
 * SplitSum(a_r, r_r, m_r, n_r, E) seen from v = -w, SplitSum = a (1 - m) E_diff(n) +
 * E_spec(R, r) (F0 A + B), R = 2 (n.v) n - v, F0 = 0.04 (1 - m) + a m.  out_ind = the mean of
 * (1 - V_r) SplitSum.  prefiltered: the output of grt_env_prefilter for the same map. */
int grt_shade_relight(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                      const grt_gbuffer* gbuffer, const grt_envmap* env, const void* prefiltered,
                      const grt_sampling* sampling, const int32_t* pixel_list, int32_t n_pixels, float* out_color,
                      float* out_vis, float* out_ind, void* stream);

/* Mesh backend of the relighting query (Sec. III-E): a triangle mesh with per-vertex
 * attributes (all device pointers, float32 / int32): pos[V][3], tri[T][3] (vertex indices),
 * normal[V][3], albedo[V][3], rough[V], metal[V]. */
typedef struct {
    int32_t n_vertices, n_triangles;
    const float* pos;
    const int32_t* tri;
    const float* normal;
    const float* albedo;
    const float* rough;
    const float* metal;
} grt_mesh;

/* Builds the 4-wide LBVH of a mesh's triangles (the same build as grt_build_bvh with one
 * triangle per leaf; the tree keeps its own copy of the geometry, the attributes are read
 * from the mesh at query time).  A vertex index outside [0, n_vertices) is reported as
 * GRT_STATUS_BAD_INDEX (grt_bvh_status) and read as vertex 0.  Free with grt_bvh_destroy. */
int grt_build_mesh_bvh(const grt_mesh* mesh, grt_bvh** out, void* stream);

/* Trace_attr (Eq. 14), mesh backend: the closest triangle hit with t in (t_min, t_max)
 * (Moeller-Trumbore; equal t by triangle index): a miss gives out_vis = 1 and zeros; a hit
 * gives out_vis = 0 and the barycentric interpolation of the triangle's per-vertex albedo,
 * roughness, metallic and normal (normalised, turned towards the ray origin).  Only
 * params->t_min / t_max are used. */
int grt_mesh_trace_attr(const grt_bvh* mesh_bvh, const grt_mesh* mesh, const grt_trace_params* params,
                        const float* ray_o, const float* ray_d, int32_t R, float* out_vis, float* out_albedo,
                        float* out_rough, float* out_metal, float* out_normal, void* stream);

/* grt_shade_relight with the mesh backend answering Eq. 14 (V_r in {0, 1}). */
int grt_shade_relight_mesh(const grt_bvh* mesh_bvh, const grt_mesh* mesh, const grt_trace_params* params,
                           const grt_gbuffer* gbuffer, const grt_envmap* env, const void* prefiltered,
                           const grt_sampling* sampling, const int32_t* pixel_list, int32_t n_pixels,
                           float* out_color, float* out_vis, float* out_ind, void* stream);

/* Cross-bilateral denoiser for low-sample shading (Sec. III-D, "Denoising"):
 *   out(p) = sum_{p' in Q(p)} B(p,p') color(p') / sum B(p,p'),
 *   B = exp(-|p-p'|^2 / (2 sigma_s^2)) * exp(-|D(p)-D(p')| / (sigma_d |grad D(p).(p-p')| + eps_d))
 *       * max(0, N(p).N(p'))^sigma_n,
 * over images of W x H pixels in raster order: color[P][3], depth[P] (e.g. the G-buffer
 * depth), normal[P][3] (normalised inside), valid[P] (0 = no surface), out[P][3].  Q(p) is
 * the valid pixels of the (2 radius + 1)^2 window inside the image; grad D is the central
 * difference of depth (one-sided next to an invalid or missing neighbour).  Invalid pixels,
 * and valid ones with a zero normal, keep their colour.  out must not alias color.
 * radius in [0, GRT_DENOISE_MAX_RADIUS]; sigma_s, sigma_d, sigma_n, eps_d > 0.  The paper
 * leaves the window and the parameter values open (defaults in the Python binding). */
#define GRT_DENOISE_MAX_RADIUS 8
typedef struct {
    int32_t radius;
    float sigma_s, sigma_d, sigma_n, eps_d;
} grt_denoise_params;
int grt_denoise(const float* color, const float* depth, const float* normal, const int32_t* valid, int32_t W,
                int32_t H, const grt_denoise_params* params, float* out, void* stream);

/* Performance counters of one grt_trace_forward-style pass (for roofline accounting):
 * counts of internal nodes visited, surfel records tested and hits composited, summed
 * over all rays, written to counters[3] (device, int64, accumulated). */
int grt_trace_count(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                    const float* ray_o, const float* ray_d, int32_t R, long long* counters,
                    void* stream);

/* Same counters for one grt_shade_pixels pass over the given pixels (no image output). */
int grt_shade_count(const grt_bvh* bvh, const grt_surfels* surfels, const grt_trace_params* params,
                    const grt_gbuffer* gbuffer, const grt_envmap* env, const grt_sampling* sampling,
                    const int32_t* pixel_list, int32_t n_pixels, long long* counters, void* stream);

/* Phase timing of grt_shade_pixels / grt_shade_batch (for roofline accounting).  With
 * enable = 1 the following shading calls of the calling thread record CUDA events on their
 * stream around the three kernels (ray sampling, trace, per-pixel accumulation); enable = 0
 * stops, enable = -1 leaves the setting unchanged.  With ms_out non-NULL the call waits for
 * the most recent timed shading call and writes its three durations in milliseconds. */
int grt_phase_timing(int32_t enable, float* ms_out);

/* Kernel timing of the adjoint (for roofline accounting; the same conventions as
 * grt_phase_timing): with enable = 1 the following grt_shade_backward /
 * grt_shade_backward_saved calls of the calling thread record CUDA events on their stream
 * around the adjoint weights, the replay of the recorded rays and the traced adjoint walk
 * of rays the record does not hold; with ms_out non-NULL the call waits for the most recent
 * timed adjoint pass (the last chunk of a recomputing backward) and writes the three
 * durations in milliseconds. */
int grt_adjoint_timing(int32_t enable, float* ms_out);

const char* grt_last_error(void);
const char* grt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GRT_H */
