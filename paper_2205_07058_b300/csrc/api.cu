// C-ABI entry points for rendering, its backward pass and device status.
// Argument checking happens here, before any work is queued.
#include <cstring>

#include "svlf_internal.cuh"
#include "mlp_common.cuh"

namespace svlf {

const OctreeView &octree_view(svlf_octree t);

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

MlpDims make_dims(const svlf_mlp_desc &d) {
    MlpDims md;
    std::memset(&md, 0, sizeof(md));
    md.F = d.feat_dim;
    md.in0 = d.feat_dim + 9;
    md.H = d.hidden;
    md.nh = d.n_hidden;
    int woff = 0, poff = 0;
    for (int l = 0; l <= md.nh; ++l) {
        md.in_l[l] = l == 0 ? md.in0 : md.H;
        md.out_l[l] = l == md.nh ? 4 : md.H;
        md.w_off[l] = woff;
        woff += md.out_l[l] * md.in_l[l] + md.out_l[l];
        md.wt_off[l] = poff;
        poff += md.out_l[l] * md.in_l[l];
        md.b_off[l] = poff;
        poff += (md.out_l[l] + 3) & ~3;
        poff = (poff + 3) & ~3;
    }
    return md;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t packed_weight_bytes(const svlf_mlp_desc &mlp) {
    const MlpDims md = make_dims(mlp);
    size_t a = sizeof(float) * packed_f32_floats(md);
    size_t b = packed_tc_bytes(md);
    return align256(a > b ? a : b);
}

size_t workspace_bytes(const svlf_mlp_desc &mlp, int64_t n_rays, int K) {
    const size_t S = (size_t)n_rays * (size_t)K;
    size_t b = 0;
    b += align256(sizeof(Sample) * S);
    b += align256(sizeof(float4) * S);
    b += align256(sizeof(float4) * S);
    b += align256(sizeof(int2) * (size_t)n_rays);
    b += 256;  // counters
    b += packed_weight_bytes(mlp);
    return b;
}

Workspace carve_workspace(void *base, const svlf_mlp_desc &mlp, int64_t n_rays, int K) {
    Workspace w;
    const size_t S = (size_t)n_rays * (size_t)K;
    char *p = static_cast<char *>(base);
    w.samples = reinterpret_cast<Sample *>(p);
    p += align256(sizeof(Sample) * S);
    w.outputs = reinterpret_cast<float4 *>(p);
    p += align256(sizeof(float4) * S);
    w.dout = reinterpret_cast<float4 *>(p);
    p += align256(sizeof(float4) * S);
    w.ray_span = reinterpret_cast<int2 *>(p);
    p += align256(sizeof(int2) * (size_t)n_rays);
    w.counter = reinterpret_cast<unsigned int *>(p);
    p += 256;
    w.packed_w = p;
    p += packed_weight_bytes(mlp);
    w.bytes = (size_t)(p - static_cast<char *>(base));
    return w;
}

static int check_mlp(const svlf_mlp_desc *m) {
    if (!m) return SVLF_ERR_ARG;
    if (m->out_dim != 4) return SVLF_ERR_UNSUPPORTED;
    if (m->feat_dim < 8 || m->feat_dim > 64 || m->feat_dim % 8) return SVLF_ERR_UNSUPPORTED;
    if (m->hidden < 32 || m->hidden > 256 || m->hidden % 16) return SVLF_ERR_UNSUPPORTED;
    if (m->n_hidden < 1 || m->n_hidden > 6) return SVLF_ERR_UNSUPPORTED;
    if (m->precision != SVLF_FP32 && m->precision != SVLF_BF16 && m->precision != SVLF_FP16)
        return SVLF_ERR_ARG;
    if (m->feat_dtype != SVLF_FEAT_F32 && m->feat_dtype != SVLF_FEAT_BF16) return SVLF_ERR_ARG;
    if (m->precision == SVLF_FP32 && m->hidden != 32 && m->hidden != 64 && m->hidden != 128 &&
        m->hidden != 256)
        return SVLF_ERR_UNSUPPORTED;
    if (m->precision != SVLF_FP32 && !tc_supported(make_dims(*m))) return SVLF_ERR_UNSUPPORTED;
    return SVLF_OK;
}

static int check_common(svlf_octree tree, const void *features, const float *params,
                        const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                        const svlf_render_opts *opts, void *workspace, size_t ws_bytes) {
    if (!tree || !opts || n_rays < 0) return SVLF_ERR_ARG;
    int rc = check_mlp(mlp);
    if (rc) return rc;
    const int K = opts->K;
    if (K < 1 || K > kMaxK) return SVLF_ERR_UNSUPPORTED;
    if (n_rays == 0) return SVLF_OK;  // nothing to read or write
    if (!params || !rays) return SVLF_ERR_ARG;
    if (!features && octree_view(tree).n_leaves > 0) return SVLF_ERR_ARG;
    if ((int64_t)n_rays * K >= ((int64_t)1 << 31)) return SVLF_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(features) % 16 || reinterpret_cast<uintptr_t>(rays) % 8)
        return SVLF_ERR_ARG;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes(*mlp, n_rays, K)) return SVLF_ERR_WORKSPACE;
    return SVLF_OK;
}

int launch_pack_weights(const svlf_mlp_desc &mlp, const float *params, void *packed,
                        cudaStream_t s) {
    const MlpDims md = make_dims(mlp);
    if (mlp.precision == SVLF_FP32) return launch_pack_f32(md, params, (float *)packed, s);
    return launch_pack_tc(md, mlp.precision, params, packed, s);
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_workspace_size(const svlf_mlp_desc *mlp, int64_t n_rays, int K,
                                   size_t *bytes) {
    if (!mlp || !bytes || n_rays < 0 || K < 1 || K > kMaxK) return SVLF_ERR_ARG;
    *bytes = workspace_bytes(*mlp, n_rays, K);
    return SVLF_OK;
}

extern "C" int svlf_render_rays(svlf_octree tree, const void *features, const float *mlp_params,
                                const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                                const svlf_render_opts *opts, float *rgb, float *depth,
                                int32_t *hits, float *t_io, void *workspace, size_t ws_bytes,
                                void *stream) {
    int rc = check_common(tree, features, mlp_params, mlp, rays, n_rays, opts, workspace, ws_bytes);
    if (rc) return rc;
    if (n_rays == 0) return SVLF_OK;
    if (!rgb || !depth) return SVLF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = opts->K;
    Workspace ws = carve_workspace(workspace, *mlp, n_rays, K);
    const MlpDims md = make_dims(*mlp);
    if (cudaMemsetAsync(ws.counter, 0, 256, s) != cudaSuccess) return SVLF_ERR_CUDA;
    if ((rc = launch_pack_weights(*mlp, mlp_params, ws.packed_w, s))) return rc;
    const OctreeView &T = octree_view(tree);
    if ((rc = launch_trace(T, rays, n_rays, K, ws, hits, t_io, s))) return rc;
    const int64_t max_samples = n_rays * (int64_t)K;
    const int fb = mlp->feat_dtype == SVLF_FEAT_BF16;
    if (mlp->precision == SVLF_FP32)
        rc = launch_mlp_forward_f32(md, T.depth, features, fb, (const float *)ws.packed_w, rays, ws,
                                    max_samples, s);
    else
        rc = launch_mlp_forward_tc(md, mlp->precision, T.depth, features, fb, ws.packed_w, rays,
                                   ws, max_samples, s);
    if (rc) return rc;
    return launch_composite(ws, n_rays, opts->bg, rgb, depth, s);
}

extern "C" int svlf_render_rays_backward(svlf_octree tree, const void *features,
                                         const float *mlp_params, const svlf_mlp_desc *mlp,
                                         const float *rays, int64_t n_rays,
                                         const svlf_render_opts *opts, const float *d_rgb,
                                         const float *d_depth, float *d_features,
                                         float *d_mlp_params, void *workspace, size_t ws_bytes,
                                         void *stream) {
    int rc = check_common(tree, features, mlp_params, mlp, rays, n_rays, opts, workspace, ws_bytes);
    if (rc) return rc;
    if (n_rays == 0 || (!d_features && !d_mlp_params)) return SVLF_OK;
    if (!d_rgb || !d_depth) return SVLF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = opts->K;
    Workspace ws = carve_workspace(workspace, *mlp, n_rays, K);
    const MlpDims md = make_dims(*mlp);
    const OctreeView &T = octree_view(tree);
    if (cudaMemsetAsync(ws.counter + 3, 0, sizeof(unsigned int), s) != cudaSuccess) return SVLF_ERR_CUDA;
    if ((rc = launch_composite_backward(ws, n_rays, opts->bg, d_rgb, d_depth, s))) return rc;
    const int64_t max_samples = n_rays * (int64_t)K;
    const int fb = mlp->feat_dtype == SVLF_FEAT_BF16;
    if (mlp->precision == SVLF_FP32)
        return launch_mlp_backward_f32(md, T.depth, features, fb, mlp_params,
                                       (const float *)ws.packed_w, rays, ws, max_samples,
                                       d_features, d_mlp_params, s);
    return launch_mlp_backward_tc(md, mlp->precision, T.depth, features, fb, ws.packed_w, rays, ws,
                                  max_samples, d_features, d_mlp_params, s);
}

extern "C" int svlf_workspace_samples(const void *workspace, const svlf_mlp_desc *mlp,
                                      int64_t n_rays, int K, int64_t *n_samples, void *stream) {
    if (!workspace || !mlp || !n_samples || n_rays < 0 || K < 1) return SVLF_ERR_ARG;
    if (n_rays == 0) {
        *n_samples = 0;
        return SVLF_OK;
    }
    Workspace ws = carve_workspace(const_cast<void *>(workspace), *mlp, n_rays, K);
    unsigned int c = 0;
    if (cudaMemcpyAsync(&c, ws.counter, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return SVLF_ERR_CUDA;
    const int64_t cap = n_rays * (int64_t)K;
    *n_samples = (int64_t)c < cap ? (int64_t)c : cap;
    return SVLF_OK;
}

extern "C" int svlf_get_device_status(int *status) {
    if (!status) return SVLF_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return SVLF_ERR_CUDA;
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof(v)) != cudaSuccess) return SVLF_ERR_CUDA;
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_device_status, &zero, sizeof(zero)) != cudaSuccess)
        return SVLF_ERR_CUDA;
    *status = (int)v;
    return SVLF_OK;
}

extern "C" const char *svlf_status_string(int status) {
    switch (status) {
        case SVLF_OK: return "ok";
        case SVLF_ERR_ARG: return "invalid argument";
        case SVLF_ERR_CUDA: return "CUDA runtime error";
        case SVLF_ERR_DEVICE: return "device-side error latched";
        case SVLF_ERR_UNSUPPORTED: return "unsupported shape or mode";
        case SVLF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}
