// svlf_render_rays_static: the render call for callers that cannot allocate
// device memory. Its scratch (sample records, network outputs, per-ray spans,
// counters, packed weights) lives in one file-scope device array of fixed size
// instead of a caller-provided workspace.
//
// Who needs it: hosts that hand a renderer a fixed device-memory budget at
// start-up and forbid allocations afterwards (plugin hosts, engines with their
// own pooled allocator), and frame loops that must not call cudaMalloc because
// it can synchronise the device and stall the frame. Such a caller passes only
// its inputs and outputs.
//
// Costs and limits:
//  * every GPU that loads the library holds kStaticScratchBytes for the life
//    of the process;
//  * a call is limited to what fits in that array (see svlf.h); larger calls
//    are rejected with SVLF_ERR_WORKSPACE before any work is queued;
//  * all calls share the one array: two calls that overlap on the GPU (other
//    streams, other host threads) race on it. The array keeps the previous
//    call's contents; the sample counter is cleared at the start of each call;
//  * the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) and caches it with the id of the device's current
//    context; make that first call before any stream capture. A later call in
//    a new context (after cudaDeviceReset) looks the address up again.
#include <mutex>

#include "svlf_internal.cuh"
#include "mlp_common.cuh"

namespace svlf {
const OctreeView &octree_view(svlf_octree t);
}  // namespace svlf

using namespace svlf;

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // id of the context the address belongs to

// Driver calls reached through the runtime's entry-point table (no link-time
// dependency on libcuda): the current context and its process-unique id.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

int current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return SVLF_ERR_CUDA;
        get_current = reinterpret_cast<CtxGetCurrentFn>(a);
        get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0) return SVLF_ERR_CUDA;
    *id = 0;
    if (ctx && get_id(ctx, id) != 0) return SVLF_ERR_CUDA;
    return SVLF_OK;
}

// Device address of the scratch array in the current device's context (host
// code only sees a stand-in for the symbol). Looked up once per device and
// context: a cudaDeviceReset gives the device a new context, in which the
// library's module (and the array) may sit at another address.
int scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SVLF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc) return rc;
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        // also makes the device's primary context current if none was
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SVLF_ERR_CUDA;
        rc = current_context_id(&ctx);
        if (rc) return rc;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return SVLF_OK;
}

}  // namespace

extern "C" int svlf_render_rays_static(svlf_octree tree, const void *features,
                                       const float *mlp_params, const svlf_mlp_desc *mlp,
                                       const float *rays, int64_t n_rays,
                                       const svlf_render_opts *opts, float *rgb, float *depth,
                                       void *stream) {
    if (!tree || !mlp || !opts || n_rays < 0) return SVLF_ERR_ARG;
    if (opts->K < 1 || opts->K > kMaxK) return SVLF_ERR_UNSUPPORTED;
    if (workspace_bytes(*mlp, n_rays, opts->K) > kStaticScratchBytes) return SVLF_ERR_WORKSPACE;
    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    return svlf_render_rays(tree, features, mlp_params, mlp, rays, n_rays, opts, rgb, depth,
                            nullptr, nullptr, scratch, kStaticScratchBytes, stream);
}
