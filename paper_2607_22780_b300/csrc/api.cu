// api.cu -- error plumbing shared by the entry points of libgrt.
#include <cstdarg>
#include <cstdio>

#include "grt_internal.cuh"

namespace grt {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return set_error(GRT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(GRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

DevBvh dev_bvh(const grt_bvh* b) {
    DevBvh d;
    d.nodes = b->wnodes;
    d.records = b->records;
    d.normals = b->normals;
    d.n = b->n;
    d.cap = b->n_int;
    d.root = b->n == 0 ? kRefEmpty : (b->n == 1 ? leaf_ref(0, 1) : 0);
    d.status = b->status;
    return d;
}

}  // namespace grt

extern "C" const char* grt_last_error(void) { return grt::g_err; }

extern "C" const char* grt_version(void) { return "grt 0.1.0 (sm_103a)"; }
