// mesh.cu -- grt_mesh_trace_attr: Trace_attr (Eq. 14) with the mesh backend for a flat list
// of rays, one thread per ray (definitions in mesh.cuh).
#include "common_args.cuh"
#include "mesh.cuh"

namespace grt {
namespace {

struct MeshAttrOut {
    float *vis, *albedo, *rough, *metal, *normal;
};

__global__ void __launch_bounds__(128) k_mesh_trace_attr(DevBvh bvh, MeshDev M, float tmin, float tmax,
                                                         const float* __restrict__ ro, const float* __restrict__ rd,
                                                         int R, MeshAttrOut out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    const f3 o = mk3(ro[3 * (size_t)i], ro[3 * (size_t)i + 1], ro[3 * (size_t)i + 2]);
    const f3 d = mk3(rd[3 * (size_t)i], rd[3 * (size_t)i + 1], rd[3 * (size_t)i + 2]);
    const MeshHit h = mesh_closest(bvh, o, d, tmin, tmax);
    float a[3] = {0.f, 0.f, 0.f}, r = 0.f, m = 0.f;
    f3 n = mk3(0.f, 0.f, 0.f);
    if (h.id >= 0) mesh_attr(M, h, d, bvh.status, a, &r, &m, &n);
    out.vis[i] = h.id >= 0 ? 0.f : 1.f;
    out.rough[i] = r;
    out.metal[i] = m;
    out.albedo[3 * (size_t)i] = a[0];
    out.albedo[3 * (size_t)i + 1] = a[1];
    out.albedo[3 * (size_t)i + 2] = a[2];
    out.normal[3 * (size_t)i] = n.x;
    out.normal[3 * (size_t)i + 1] = n.y;
    out.normal[3 * (size_t)i + 2] = n.z;
}

}  // namespace
}  // namespace grt

using namespace grt;

extern "C" int grt_mesh_trace_attr(const grt_bvh* b, const grt_mesh* m, const grt_trace_params* p, const float* ray_o,
                                   const float* ray_d, int32_t R, float* out_vis, float* out_albedo, float* out_rough,
                                   float* out_metal, float* out_normal, void* stream) {
    if (!b || !m) return set_error(GRT_ERR_ARG, "mesh bvh or mesh is NULL");
    if (m->n_triangles != b->n) return set_error(GRT_ERR_ARG, "mesh has %d triangles, the tree %d", m->n_triangles, b->n);
    int rc = check_params(p);
    if (rc) return rc;
    if (R < 0) return set_error(GRT_ERR_ARG, "R < 0");
    if (R == 0) return GRT_OK;
    if (!ray_o || !ray_d || !out_vis || !out_albedo || !out_rough || !out_metal || !out_normal)
        return set_error(GRT_ERR_ARG, "rays and every output must be non-NULL");
    if (m->n_triangles > 0 && (!m->tri || !m->normal || !m->albedo || !m->rough || !m->metal))
        return set_error(GRT_ERR_ARG, "mesh attributes must be non-NULL");
    MeshDev M{m->tri, m->normal, m->albedo, m->rough, m->metal, m->n_vertices};
    MeshAttrOut out{out_vis, out_albedo, out_rough, out_metal, out_normal};
    k_mesh_trace_attr<<<(R + 127) / 128, 128, 0, (cudaStream_t)stream>>>(dev_bvh(b), M, p->t_min, p->t_max, ray_o,
                                                                         ray_d, R, out);
    return launch_error("k_mesh_trace_attr");
}
