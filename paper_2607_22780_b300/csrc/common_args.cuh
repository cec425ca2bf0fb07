// common_args.cuh -- argument checks and k-buffer size dispatch shared by entry points.
#pragma once

#include <type_traits>

#include "grt_internal.cuh"
#include "trace.cuh"

namespace grt {

inline int check_params(const grt_trace_params* p) {
    if (!p) return set_error(GRT_ERR_ARG, "params is NULL");
    if (!(p->alpha_min > 0.f && p->alpha_min < 1.f)) return set_error(GRT_ERR_ARG, "alpha_min must be in (0,1)");
    if (!(p->alpha_max >= p->alpha_min && p->alpha_max <= 1.f))
        return set_error(GRT_ERR_ARG, "alpha_max must be in [alpha_min, 1]");
    if (!(p->t_min >= 0.f) || !(p->t_max > p->t_min)) return set_error(GRT_ERR_ARG, "need 0 <= t_min < t_max");
    if (!(p->T_min >= 0.f && p->T_min < 1.f)) return set_error(GRT_ERR_ARG, "T_min must be in [0,1)");
    if (!(p->eps_nd >= 0.f)) return set_error(GRT_ERR_ARG, "eps_nd must be >= 0");
    if (p->k != 4 && p->k != 8 && p->k != 16 && p->k != 32)
        return set_error(GRT_ERR_UNSUPPORTED, "k = %d; built sizes are 4, 8, 16, 32", p->k);
    if (p->build_passes < 0 || p->build_passes > GRT_MAX_BUILD_PASSES)
        return set_error(GRT_ERR_ARG, "build_passes = %d outside [0, %d]", p->build_passes, GRT_MAX_BUILD_PASSES);
    if (p->gbuffer_k != 0 && p->gbuffer_k != 4 && p->gbuffer_k != 8 && p->gbuffer_k != 16 && p->gbuffer_k != 32)
        return set_error(GRT_ERR_UNSUPPORTED, "gbuffer_k = %d; 0 (by frame size) or a built size 4, 8, 16, 32",
                         p->gbuffer_k);
    return GRT_OK;
}

inline int check_trace_inputs(const grt_bvh* b, const grt_surfels* s, const grt_trace_params* p) {
    if (!b) return set_error(GRT_ERR_ARG, "bvh is NULL");
    if (!s) return set_error(GRT_ERR_ARG, "surfels is NULL");
    if (s->n != b->n) return set_error(GRT_ERR_ARG, "surfels->n = %d but the BVH holds %d", s->n, b->n);
    if (s->color_dim != 3 && s->color_dim != 48)
        return set_error(GRT_ERR_ARG, "color_dim = %d; must be 3 or 48", s->color_dim);
    if (s->n > 0 && !s->color) return set_error(GRT_ERR_ARG, "surfels->color is NULL");
    if (s->color_dim == 48 && ((uintptr_t)s->color & 15))
        return set_error(GRT_ERR_ARG, "SH colour array must be 16-byte aligned");
    return check_params(p);
}

inline int launch_error(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, what);
    return GRT_OK;
}

// Calls f(std::integral_constant<int, K>{}) for the runtime k-buffer size.
template <class F>
inline void dispatch_k(int k, F&& f) {
    switch (k) {
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}

}  // namespace grt
