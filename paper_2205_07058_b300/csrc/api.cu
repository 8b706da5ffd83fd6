// C-ABI entry points for rendering, its backward pass and device status.
// Argument checking happens here, before any work is queued.
#include <cstring>

#include "svlf_internal.cuh"
#include "mlp_common.cuh"
#include "mlp_simt.h"

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

static svlf_tuning g_tuning = {0, 1, 16, 256, 0};

const svlf_tuning &tuning() { return g_tuning; }

// traversal step bound per ray (svlf_set_step_limit); 0 = 3 * 2^L + 64
int g_step_limit = 0;

MlpDims make_dims(const svlf_mlp_desc &d) {
    return make_dims_io(d.feat_dim, d.feat_dim + 9, d.hidden, d.n_hidden, 4);
}

MlpDims make_dims_io(int F, int in0, int H, int nh, int out) {
    MlpDims md;
    std::memset(&md, 0, sizeof(md));
    md.F = F;
    md.in0 = in0;
    md.H = H;
    md.nh = nh;
    md.out = out;
    int woff = 0, poff = 0;
    for (int l = 0; l <= md.nh; ++l) {
        md.in_l[l] = l == 0 ? md.in0 : md.H;
        md.out_l[l] = l == md.nh ? md.out : md.H;
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

// Workspace of n_rays rays with n_scenes packed weight images of `stride` bytes.
static size_t workspace_bytes_raw(int64_t n_rays, int K, size_t stride, int n_scenes) {
    const size_t S = (size_t)n_rays * (size_t)K;
    size_t b = 0;
    b += align256(sizeof(Sample) * S);
    b += align256(sizeof(float4) * S);
    b += align256(sizeof(float4) * S);
    b += align256(sizeof(int2) * (size_t)n_rays);
    b += kCounterBytes;
    b += (size_t)n_scenes * stride;
    return b;
}

size_t workspace_bytes(const svlf_mlp_desc &mlp, int64_t n_rays, int K, int n_scenes) {
    return workspace_bytes_raw(n_rays, K, packed_weight_bytes(mlp), n_scenes);
}

static Workspace carve_workspace_raw(void *base, int64_t n_rays, int K, size_t stride, int n_scenes);

Workspace carve_workspace(void *base, const svlf_mlp_desc &mlp, int64_t n_rays, int K,
                          int n_scenes) {
    return carve_workspace_raw(base, n_rays, K, packed_weight_bytes(mlp), n_scenes);
}

static Workspace carve_workspace_raw(void *base, int64_t n_rays, int K, size_t stride, int n_scenes) {
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
    p += kCounterBytes;
    w.packed_w = p;
    w.packed_stride = stride;
    p += (size_t)n_scenes * w.packed_stride;
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
    if (m->precision == SVLF_FP32 && !f32_forward_fits(make_dims(*m))) return SVLF_ERR_UNSUPPORTED;
    if (m->precision != SVLF_FP32 && !tc_supported(make_dims(*m))) return SVLF_ERR_UNSUPPORTED;
    return SVLF_OK;
}

static int check_scene(const svlf_scene &sc, bool need_outputs) {
    if (!sc.tree || sc.n_rays < 0) return SVLF_ERR_ARG;
    if (sc.n_rays == 0) return SVLF_OK;  // nothing to read or write
    if (!sc.mlp_params || !sc.rays) return SVLF_ERR_ARG;
    if (!sc.features && octree_view(sc.tree).n_leaves > 0) return SVLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(sc.features) % 16 || reinterpret_cast<uintptr_t>(sc.rays) % 8)
        return SVLF_ERR_ARG;
    if (need_outputs && (!sc.rgb || !sc.depth)) return SVLF_ERR_ARG;
    return SVLF_OK;
}

// Validate a call and build its scene table (device-side view of the scenes).
static int make_table_core(const svlf_scene *scenes, int n_scenes, const svlf_render_opts *opts,
                           bool backward, SceneTable &T, bool per_ray_io = true);

static int make_table(const svlf_scene *scenes, int n_scenes, const svlf_mlp_desc *mlp,
                      const svlf_render_opts *opts, void *workspace, size_t ws_bytes,
                      bool backward, SceneTable &T) {
    if (!scenes || n_scenes < 1 || !opts) return SVLF_ERR_ARG;
    if (n_scenes > kMaxScenes) return SVLF_ERR_UNSUPPORTED;
    int rc = check_mlp(mlp);
    if (rc) return rc;
    if ((rc = make_table_core(scenes, n_scenes, opts, backward, T))) return rc;
    if (T.total_rays == 0) return SVLF_OK;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes(*mlp, T.total_rays, T.K, n_scenes)) return SVLF_ERR_WORKSPACE;
    return SVLF_OK;
}

// Scene table of a call (device-side view of the scenes), without the
// network or workspace checks.
// per_ray_io = false: the call reads and writes no per-ray images or image
// gradients (the surface loss of the staged training)
static int make_table_core(const svlf_scene *scenes, int n_scenes, const svlf_render_opts *opts,
                           bool backward, SceneTable &T, bool per_ray_io) {
    if (!scenes || n_scenes < 1 || !opts) return SVLF_ERR_ARG;
    if (n_scenes > kMaxScenes) return SVLF_ERR_UNSUPPORTED;
    int rc = SVLF_OK;
    const int K = opts->K;
    if (K < 1 || K > kMaxK) return SVLF_ERR_UNSUPPORTED;
    if (opts->rparam_mode != SVLF_RPARAM_SPHERE && opts->rparam_mode != SVLF_RPARAM_AABB) return SVLF_ERR_ARG;
    if (opts->image_width < 0) return SVLF_ERR_ARG;
    std::memset(&T, 0, sizeof(T));
    T.n = n_scenes;
    T.K = K;
    T.rparam = opts->rparam_mode;
    // traversal work items: kTraceChunk rays each (a warp walks neighbouring
    // rays together, which keeps their walks coherent)
    int64_t rays = 0, chunks = 0;
    for (int i = 0; i < n_scenes; ++i) {
        const svlf_scene &sc = scenes[i];
        if ((rc = check_scene(sc, per_ray_io && !backward))) return rc;
        // backward: a scene without output gradients (both NULL) takes no part
        if (per_ray_io && backward && sc.n_rays > 0 && (!sc.d_rgb != !sc.d_depth)) return SVLF_ERR_ARG;
        SceneDev &d = T.s[i];
        d.grad = !(per_ray_io && backward && !sc.d_rgb);
        // image rows walked in 8 x 4 tiles of 32 rays (kTraceChunk), where the scene's
        // rays are whole bands of four rows of a width that is a multiple of 8
        const int64_t iw = opts->image_width;
        d.tile_w = (iw > 0 && iw % 8 == 0 && sc.n_rays % (4 * iw) == 0) ? (int)iw : 0;
        d.grad_begin = T.grad_rays;
        if (d.grad) T.grad_rays += sc.n_rays;
        d.tree = octree_view(sc.tree);
        d.feats = sc.features;
        d.params = sc.mlp_params;
        d.rays = sc.rays;
        d.rgb = sc.rgb;
        d.depth = sc.depth;
        d.d_rgb = sc.d_rgb;
        d.d_depth = sc.d_depth;
        d.d_feat = sc.d_features;
        d.d_params = sc.d_mlp_params;
        d.ray_begin = rays;
        d.n_rays = sc.n_rays;
        d.chunk_begin = chunks;
        rays += sc.n_rays;
        chunks += (sc.n_rays + kTraceChunk - 1) / kTraceChunk;
    }
    T.total_rays = rays;
    T.total_chunks = chunks;
    if (rays * K >= ((int64_t)1 << 31)) return SVLF_ERR_UNSUPPORTED;
    return SVLF_OK;
}

int launch_pack_weights(const svlf_mlp_desc &mlp, const SceneTable &T, const Workspace &ws,
                        cudaStream_t s) {
    const MlpDims md = make_dims(mlp);
    if (mlp.precision == SVLF_FP32) {
        int rc = SVLF_OK;
        for (int i = 0; i < T.n && !rc; ++i)
            if (T.s[i].params)  // a scene without rays may come without parameters
                rc = launch_pack_f32(md, T.s[i].params, (float *)((char *)ws.packed_w + i * ws.packed_stride), s);
        return rc;
    }
    return launch_pack_tc(md, mlp.precision, T, ws.packed_w, ws.packed_stride, s);
}

static int render_table(const SceneTable &T, const svlf_mlp_desc &mlp, const svlf_render_opts &opts,
                        void *workspace, int32_t *hits, float *t_io, cudaStream_t s) {
    if (T.total_rays == 0) return SVLF_OK;
    Workspace ws = carve_workspace(workspace, mlp, T.total_rays, T.K, T.n);
    int rc;
    if (cudaMemsetAsync(ws.counter, 0, kCounterBytes, s) != cudaSuccess) return SVLF_ERR_CUDA;
    if ((rc = launch_pack_weights(mlp, T, ws, s))) return rc;
    if ((rc = launch_trace(T, ws, hits, t_io, s))) return rc;
    const MlpDims md = make_dims(mlp);
    const int fb = mlp.feat_dtype == SVLF_FEAT_BF16;
    if (mlp.precision == SVLF_FP32) {
        if (T.n != 1) return SVLF_ERR_UNSUPPORTED;
        rc = launch_mlp_forward_f32(md, T.s[0].tree.depth, T.rparam, T.s[0].feats, fb, (const float *)ws.packed_w,
                                    T.s[0].rays, ws, T.total_rays * (int64_t)T.K, s);
    } else {
        rc = launch_mlp_forward_tc(md, mlp.precision, fb, T, ws, s);
    }
    if (rc) return rc;
    return launch_composite(T, ws, opts.bg, s);
}

static int backward_table(const SceneTable &T, const svlf_mlp_desc &mlp, const svlf_render_opts &opts,
                          void *workspace, bool want_feat, bool want_params, cudaStream_t s) {
    if (T.grad_rays == 0 || (!want_feat && !want_params)) return SVLF_OK;
    if (mlp.precision == SVLF_FP32 && (T.n != 1 || !f32_backward_fits(make_dims(mlp)))) return SVLF_ERR_UNSUPPORTED;
    Workspace ws = carve_workspace(workspace, mlp, T.total_rays, T.K, T.n);
    int rc;
    if (cudaMemsetAsync(ws.counter + kCtrMaxAbsDout, 0, sizeof(unsigned int), s) != cudaSuccess)
        return SVLF_ERR_CUDA;
    if ((rc = launch_composite_backward(T, ws, opts.bg, s))) return rc;
    const MlpDims md = make_dims(mlp);
    const int fb = mlp.feat_dtype == SVLF_FEAT_BF16;
    if (mlp.precision == SVLF_FP32) {
        if (T.n != 1) return SVLF_ERR_UNSUPPORTED;
        const SceneDev &d = T.s[0];
        return launch_mlp_backward_f32(md, d.tree.depth, T.rparam, d.feats, fb, d.params, (const float *)ws.packed_w,
                                       d.rays, ws, T.total_rays * (int64_t)T.K,
                                       want_feat ? d.d_feat : nullptr, want_params ? d.d_params : nullptr, s);
    }
    return launch_mlp_backward_tc(md, mlp.precision, fb, T, ws, want_feat, want_params, s);
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_workspace_size(const svlf_mlp_desc *mlp, int64_t n_rays, int K,
                                   size_t *bytes) {
    if (!mlp || !bytes || n_rays < 0 || K < 1 || K > kMaxK) return SVLF_ERR_ARG;
    *bytes = workspace_bytes(*mlp, n_rays, K, 1);
    return SVLF_OK;
}

extern "C" int svlf_workspace_size_batched(const svlf_mlp_desc *mlp, int64_t total_rays,
                                           int n_scenes, int K, size_t *bytes) {
    if (!mlp || !bytes || total_rays < 0 || K < 1 || K > kMaxK || n_scenes < 1 ||
        n_scenes > kMaxScenes)
        return SVLF_ERR_ARG;
    *bytes = workspace_bytes(*mlp, total_rays, K, n_scenes);
    return SVLF_OK;
}

static svlf_scene one_scene(svlf_octree tree, const void *features, const float *mlp_params,
                            const float *rays, int64_t n_rays) {
    svlf_scene sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.tree = tree;
    sc.features = features;
    sc.mlp_params = mlp_params;
    sc.rays = rays;
    sc.n_rays = n_rays;
    return sc;
}

extern "C" int svlf_render_rays(svlf_octree tree, const void *features, const float *mlp_params,
                                const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                                const svlf_render_opts *opts, float *rgb, float *depth,
                                int32_t *hits, float *t_io, void *workspace, size_t ws_bytes,
                                void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    svlf_scene sc = one_scene(tree, features, mlp_params, rays, n_rays);
    sc.rgb = rgb;
    sc.depth = depth;
    SceneTable T;
    int rc = make_table(&sc, 1, mlp, opts, workspace, ws_bytes, false, T);
    if (rc) return rc;
    return render_table(T, *mlp, *opts, workspace, hits, t_io, (cudaStream_t)stream);
}

extern "C" int svlf_render_rays_backward(svlf_octree tree, const void *features,
                                         const float *mlp_params, const svlf_mlp_desc *mlp,
                                         const float *rays, int64_t n_rays,
                                         const svlf_render_opts *opts, const float *d_rgb,
                                         const float *d_depth, float *d_features,
                                         float *d_mlp_params, void *workspace, size_t ws_bytes,
                                         void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    if (n_rays > 0 && (!d_rgb || !d_depth)) return SVLF_ERR_ARG;
    svlf_scene sc = one_scene(tree, features, mlp_params, rays, n_rays);
    sc.d_rgb = d_rgb;
    sc.d_depth = d_depth;
    sc.d_features = d_features;
    sc.d_mlp_params = d_mlp_params;
    SceneTable T;
    int rc = make_table(&sc, 1, mlp, opts, workspace, ws_bytes, true, T);
    if (rc) return rc;
    return backward_table(T, *mlp, *opts, workspace, d_features != nullptr, d_mlp_params != nullptr,
                          (cudaStream_t)stream);
}

extern "C" int svlf_render_rays_batched(const svlf_scene *scenes, int n_scenes,
                                        const svlf_mlp_desc *mlp, const svlf_render_opts *opts,
                                        void *workspace, size_t ws_bytes, void *stream) {
    SceneTable T;
    int rc = make_table(scenes, n_scenes, mlp, opts, workspace, ws_bytes, false, T);
    if (rc) return rc;
    if (mlp->precision == SVLF_FP32 && n_scenes > 1) return SVLF_ERR_UNSUPPORTED;
    return render_table(T, *mlp, *opts, workspace, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int svlf_render_rays_backward_batched(const svlf_scene *scenes, int n_scenes,
                                                 const svlf_mlp_desc *mlp,
                                                 const svlf_render_opts *opts, void *workspace,
                                                 size_t ws_bytes, void *stream) {
    SceneTable T;
    int rc = make_table(scenes, n_scenes, mlp, opts, workspace, ws_bytes, true, T);
    if (rc) return rc;
    if (mlp->precision == SVLF_FP32 && n_scenes > 1) return SVLF_ERR_UNSUPPORTED;
    bool want_feat = false, want_params = false;
    for (int i = 0; i < n_scenes; ++i) {
        if (!T.s[i].grad) continue;
        want_feat |= scenes[i].d_features != nullptr;
        want_params |= scenes[i].d_mlp_params != nullptr;
    }
    for (int i = 0; i < n_scenes; ++i) {  // each gradient for all scenes that take part, or none
        if (!T.s[i].grad) continue;
        if ((want_feat && !scenes[i].d_features) || (want_params && !scenes[i].d_mlp_params))
            if (scenes[i].n_rays > 0) return SVLF_ERR_ARG;
    }
    return backward_table(T, *mlp, *opts, workspace, want_feat, want_params, (cudaStream_t)stream);
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
    if (cudaMemcpyAsync(&c, ws.counter + kCtrScene, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return SVLF_ERR_CUDA;
    const int64_t cap = n_rays * (int64_t)K;
    *n_samples = (int64_t)c < cap ? (int64_t)c : cap;
    return SVLF_OK;
}

extern "C" int svlf_workspace_scene_samples(const void *workspace, const svlf_mlp_desc *mlp,
                                            const int64_t *n_rays, int n_scenes, int K, int64_t *per_scene,
                                            void *stream) {
    if (!workspace || !mlp || !n_rays || !per_scene || n_scenes < 1 || n_scenes > kMaxScenes || K < 1)
        return SVLF_ERR_ARG;
    int64_t total = 0;
    for (int i = 0; i < n_scenes; ++i) {
        if (n_rays[i] < 0) return SVLF_ERR_ARG;
        total += n_rays[i];
        per_scene[i] = 0;
    }
    if (total == 0) return SVLF_OK;
    Workspace ws = carve_workspace(const_cast<void *>(workspace), *mlp, total, K, n_scenes);
    unsigned int c[kMaxScenes];
    if (cudaMemcpyAsync(c, ws.counter + kCtrScene, sizeof(unsigned int) * n_scenes, cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return SVLF_ERR_CUDA;
    for (int i = 0; i < n_scenes; ++i) {
        const int64_t cap = n_rays[i] * (int64_t)K;
        per_scene[i] = (int64_t)c[i] < cap ? (int64_t)c[i] : cap;
    }
    return SVLF_OK;
}

extern "C" int svlf_workspace_samples_batched(const void *workspace, const svlf_mlp_desc *mlp,
                                              const int64_t *n_rays, int n_scenes, int K, int64_t *n_samples,
                                              void *stream) {
    if (!n_samples) return SVLF_ERR_ARG;
    int64_t per[kMaxScenes];
    if (n_scenes < 1 || n_scenes > kMaxScenes) return SVLF_ERR_ARG;
    const int rc = svlf_workspace_scene_samples(workspace, mlp, n_rays, n_scenes, K, per, stream);
    if (rc) return rc;
    *n_samples = 0;
    for (int i = 0; i < n_scenes; ++i) *n_samples += per[i];
    return SVLF_OK;
}

extern "C" int svlf_set_tuning(const svlf_tuning *t) {
    if (!t) return SVLF_ERR_ARG;
    svlf_tuning v = *t;
    if (v.mlp_warpgroups < 0 || v.mlp_warpgroups > 4) return SVLF_ERR_ARG;
    if (v.mlp_epilogue_batch == 0) v.mlp_epilogue_batch = 1;
    if (v.mlp_epilogue_batch < 1 || v.mlp_epilogue_batch > 3) return SVLF_ERR_ARG;
    if (v.trace_budget == 0) v.trace_budget = 64;
    if (v.trace_budget < 1 || v.trace_budget > 256) return SVLF_ERR_ARG;
    if (v.trace_block == 0) v.trace_block = 256;
    if (v.trace_block != 128 && v.trace_block != 256) return SVLF_ERR_ARG;
    if (v.trace_refill < 0 || v.trace_refill > 32) return SVLF_ERR_ARG;
    if (v.mlp_bwd_warpgroups < 0 || v.mlp_bwd_warpgroups > 2) return SVLF_ERR_ARG;
    g_tuning = v;
    return SVLF_OK;
}

extern "C" int svlf_get_tuning(svlf_tuning *t) {
    if (!t) return SVLF_ERR_ARG;
    *t = g_tuning;
    return SVLF_OK;
}

namespace svlf {
// the value the last status read took out of the status word
__device__ unsigned int g_status_taken = 0;

__global__ void take_status_kernel() { g_status_taken = atomicExch(&g_device_status, 0u); }
}  // namespace svlf

extern "C" int svlf_get_device_status(void *stream, int *status) {
    if (!status) return SVLF_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // read-and-clear in one atomic, ordered after the work queued on `stream`
    take_status_kernel<<<1, 1, 0, s>>>();
    if (cudaGetLastError() != cudaSuccess) return SVLF_ERR_CUDA;
    unsigned int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_status_taken, sizeof(v), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SVLF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SVLF_ERR_CUDA;
    *status = (int)v;
    return SVLF_OK;
}

extern "C" int svlf_set_step_limit(int64_t max_steps) {
    if (max_steps < 0 || max_steps > (int64_t)1 << 30) return SVLF_ERR_ARG;
    g_step_limit = (int)max_steps;
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

// ---------------------------------------------------------------- two-decoder form
namespace svlf {

static int check_two_decoder(const svlf_two_decoder_desc *d) {
    if (!d) return SVLF_ERR_ARG;
    if (d->feat_t < 8 || d->feat_t > 64 || d->feat_t % 8 || d->feat_c < 8 || d->feat_c > 64 || d->feat_c % 8)
        return SVLF_ERR_UNSUPPORTED;
    if (d->hidden_t < 32 || d->hidden_t > 128 || d->hidden_t % 16 || d->hidden_c < 32 || d->hidden_c > 128 ||
        d->hidden_c % 16)
        return SVLF_ERR_UNSUPPORTED;
    if (d->n_hidden_t < 1 || d->n_hidden_t > 4 || d->n_hidden_c < 1 || d->n_hidden_c > 4)
        return SVLF_ERR_UNSUPPORTED;
    if (d->precision != SVLF_BF16 && d->precision != SVLF_FP16) {
        return d->precision == SVLF_FP32 ? SVLF_ERR_UNSUPPORTED : SVLF_ERR_ARG;
    }
    if (d->feat_dtype != SVLF_FEAT_F32 && d->feat_dtype != SVLF_FEAT_BF16) return SVLF_ERR_ARG;
    return SVLF_OK;
}

static MlpDims dims_t(const svlf_two_decoder_desc &d) {
    return make_dims_io(d.feat_t, 2 * d.feat_t + 6, d.hidden_t, d.n_hidden_t, 2);
}
static MlpDims dims_c(const svlf_two_decoder_desc &d) {
    return make_dims_io(d.feat_c, d.feat_c + 6, d.hidden_c, d.n_hidden_c, 3);
}
// packed images: F^T at offset 0, F^C at image_c_offset
static size_t image_c_offset(const svlf_two_decoder_desc &d) { return align256(packed_tc_bytes(dims_t(d))); }
static size_t images_bytes(const svlf_two_decoder_desc &d) {
    return image_c_offset(d) + align256(packed_tc_bytes(dims_c(d)));
}
// after the images: aux (tau, eta, t_in, t_out per sample), w dL/dD per sample and
// a direct dL/d(eta) per sample (a loss term on eta; zero unless one is added)
static size_t two_decoder_stride(const svlf_two_decoder_desc &d, int64_t n_rays, int K) {
    const size_t S = (size_t)n_rays * (size_t)K;
    return images_bytes(d) + align256(sizeof(float4) * S) + 2 * align256(sizeof(float) * S);
}
static float4 *aux_of(const Workspace &ws, const svlf_two_decoder_desc &d) {
    return reinterpret_cast<float4 *>(static_cast<char *>(ws.packed_w) + images_bytes(d));
}
static float *w_dD_of(const Workspace &ws, const svlf_two_decoder_desc &d, int64_t n_rays, int K) {
    return reinterpret_cast<float *>(reinterpret_cast<char *>(aux_of(ws, d)) +
                                     align256(sizeof(float4) * (size_t)n_rays * (size_t)K));
}
static float *deta_of(const Workspace &ws, const svlf_two_decoder_desc &d, int64_t n_rays, int K) {
    return reinterpret_cast<float *>(reinterpret_cast<char *>(w_dD_of(ws, d, n_rays, K)) +
                                     align256(sizeof(float) * (size_t)n_rays * (size_t)K));
}

}  // namespace svlf

extern "C" int svlf_workspace_size_two_decoder(const svlf_two_decoder_desc *desc, int64_t n_rays, int K,
                                               size_t *bytes) {
    if (!bytes || n_rays < 0 || K < 1 || K > kMaxK) return SVLF_ERR_ARG;
    int rc = check_two_decoder(desc);
    if (rc) return rc;
    *bytes = workspace_bytes_raw(n_rays, K, two_decoder_stride(*desc, n_rays, K), 1);
    return SVLF_OK;
}

extern "C" int svlf_render_rays_two_decoder(svlf_octree tree, const void *z_t, const void *z_c,
                                            const float *params_t, const float *params_c,
                                            const svlf_two_decoder_desc *desc, const float *rays,
                                            int64_t n_rays, const svlf_render_opts *opts, float *rgb,
                                            float *depth, int32_t *hits, float *t_io, void *workspace,
                                            size_t ws_bytes, void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    int rc = check_two_decoder(desc);
    if (rc) return rc;
    const OctreeView &view = octree_view(tree);
    if (!view.leaf_vertices && view.n_leaves > 0) return SVLF_ERR_ARG;  // svlf_octree_build_vertices first
    if (n_rays > 0 && view.n_leaves > 0 && (!z_t || !z_c || !params_t || !params_c)) return SVLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(z_c) % 16) return SVLF_ERR_ARG;
    if (opts && opts->rparam_mode != SVLF_RPARAM_SPHERE) return SVLF_ERR_UNSUPPORTED;
    svlf_scene sc = one_scene(tree, z_t, params_t, rays, n_rays);
    sc.rgb = rgb;
    sc.depth = depth;
    SceneTable T;
    if ((rc = make_table_core(&sc, 1, opts, false, T))) return rc;
    if (T.total_rays == 0) return SVLF_OK;
    const size_t stride = two_decoder_stride(*desc, T.total_rays, T.K);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes_raw(T.total_rays, T.K, stride, 1)) return SVLF_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws = carve_workspace_raw(workspace, T.total_rays, T.K, stride, 1);
    const MlpDims mt = dims_t(*desc), mc = dims_c(*desc);
    const int fb = desc->feat_dtype == SVLF_FEAT_BF16;
    SceneTable Tc = T;  // the colour pass: Z^C and F^C
    Tc.s[0].feats = z_c;
    Tc.s[0].params = params_c;
    Workspace wc = ws;
    wc.packed_w = static_cast<char *>(ws.packed_w) + image_c_offset(*desc);
    if (cudaMemsetAsync(ws.counter, 0, kCounterBytes, s) != cudaSuccess) return SVLF_ERR_CUDA;
    if (cudaMemsetAsync(deta_of(ws, *desc, T.total_rays, T.K), 0, sizeof(float) * (size_t)T.total_rays * T.K, s) !=
        cudaSuccess)
        return SVLF_ERR_CUDA;
    if ((rc = launch_pack_tc(mt, desc->precision, T, ws.packed_w, stride, s))) return rc;
    if ((rc = launch_pack_tc(mc, desc->precision, Tc, wc.packed_w, stride, s))) return rc;
    if ((rc = launch_trace(T, ws, hits, t_io, s))) return rc;
    float4 *aux = aux_of(ws, *desc);
    if ((rc = launch_mlp_forward_tc(mt, desc->precision, fb, T, ws, s, 1, aux))) return rc;
    if ((rc = launch_mlp_forward_tc(mc, desc->precision, fb, Tc, wc, s, 2, aux))) return rc;
    return launch_composite(T, ws, opts->bg, s);
}

extern "C" int svlf_render_rays_backward_two_decoder(
    svlf_octree tree, const void *z_t, const void *z_c, const float *params_t, const float *params_c,
    const svlf_two_decoder_desc *desc, const float *rays, int64_t n_rays, const svlf_render_opts *opts,
    const float *d_rgb, const float *d_depth, float *d_z_t, float *d_z_c, float *d_params_t, float *d_params_c,
    void *workspace, size_t ws_bytes, void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    int rc = check_two_decoder(desc);
    if (rc) return rc;
    const OctreeView &view = octree_view(tree);
    if (!view.leaf_vertices && view.n_leaves > 0) return SVLF_ERR_ARG;
    if (n_rays > 0 && view.n_leaves > 0 && (!z_t || !z_c || !params_t || !params_c)) return SVLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(z_c) % 16) return SVLF_ERR_ARG;
    if (n_rays > 0 && (!d_rgb || !d_depth)) return SVLF_ERR_ARG;
    svlf_scene sc = one_scene(tree, z_t, params_t, rays, n_rays);
    sc.d_rgb = d_rgb;
    sc.d_depth = d_depth;
    sc.d_features = d_z_t;
    sc.d_mlp_params = d_params_t;
    SceneTable T;
    if (opts && opts->rparam_mode != SVLF_RPARAM_SPHERE) return SVLF_ERR_UNSUPPORTED;
    if ((rc = make_table_core(&sc, 1, opts, true, T))) return rc;
    if (T.total_rays == 0 || (!d_z_t && !d_z_c && !d_params_t && !d_params_c)) return SVLF_OK;
    const size_t stride = two_decoder_stride(*desc, T.total_rays, T.K);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes_raw(T.total_rays, T.K, stride, 1)) return SVLF_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws = carve_workspace_raw(workspace, T.total_rays, T.K, stride, 1);
    const MlpDims mt = dims_t(*desc), mc = dims_c(*desc);
    const int fb = desc->feat_dtype == SVLF_FEAT_BF16;
    SceneTable Tc = T;
    Tc.s[0].feats = z_c;
    Tc.s[0].params = params_c;
    Tc.s[0].d_feat = d_z_c;
    Tc.s[0].d_params = d_params_c;
    Workspace wc = ws;
    wc.packed_w = static_cast<char *>(ws.packed_w) + image_c_offset(*desc);
    float4 *aux = aux_of(ws, *desc);
    float *w_dD = w_dD_of(ws, *desc, T.total_rays, T.K);
    if (cudaMemsetAsync(ws.counter + kCtrMaxAbsDout, 0, sizeof(unsigned int), s) != cudaSuccess)
        return SVLF_ERR_CUDA;
    if ((rc = launch_composite_backward(T, ws, opts->bg, s, w_dD))) return rc;
    // the colour pass runs whenever anything is wanted: it forms dL/d(eta) for the
    // optical-thickness pass
    if ((rc = launch_mlp_backward_tc(mc, desc->precision, fb, Tc, wc, d_z_c != nullptr, d_params_c != nullptr, s,
                                     2, aux, w_dD, deta_of(ws, *desc, T.total_rays, T.K))))
        return rc;
    if (!d_z_t && !d_params_t) return SVLF_OK;
    return launch_mlp_backward_tc(mt, desc->precision, fb, T, ws, d_z_t != nullptr, d_params_t != nullptr, s, 1,
                                  aux, w_dD);
}

// ---------------------------------------------------------------- staged training (Sec. 4.4)
namespace svlf {
int launch_surface_samples(const SceneTable &T, const float *depth_t, const float *mask, Sample *samples,
                           float *eta_gt, unsigned int *counter, cudaStream_t s);
int launch_surface_loss(const Sample *samples, const unsigned int *counter, const float4 *outputs,
                        const float4 *aux, const float *rgb_t, int64_t n_rays, float lam_eta, float lam_tau,
                        float4 *dout, float *deta, float *w_dD, unsigned int *max_abs_bits, double *loss_accum,
                        cudaStream_t s);
int launch_eta_term(const SceneTable &T, const int2 *ray_span, const float4 *aux, const float *depth_t,
                    const float *mask, float lam_eta, float *deta, double *loss_accum, cudaStream_t s);
}  // namespace svlf

extern "C" int svlf_surface_loss_two_decoder(
    svlf_octree tree, const void *z_t, const void *z_c, const float *params_t, const float *params_c,
    const svlf_two_decoder_desc *desc, const float *rays, int64_t n_rays, const float *rgb_target,
    const float *depth_target, const float *mask, float lambda_eta, float lambda_tau, double *loss_accum,
    float *d_z_t, float *d_z_c, float *d_params_t, float *d_params_c, void *workspace, size_t ws_bytes,
    void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    int rc = check_two_decoder(desc);
    if (rc) return rc;
    const OctreeView &view = octree_view(tree);
    if (!view.leaf_vertices && view.n_leaves > 0) return SVLF_ERR_ARG;
    if (n_rays > 0 && (!rgb_target || !depth_target || !loss_accum)) return SVLF_ERR_ARG;
    if (n_rays > 0 && view.n_leaves > 0 && (!z_t || !z_c || !params_t || !params_c)) return SVLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(z_c) % 16) return SVLF_ERR_ARG;
    svlf_render_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.K = 1;  // one sample (the surface voxel) per ray
    svlf_scene sc = one_scene(tree, z_t, params_t, rays, n_rays);
    SceneTable T;
    if ((rc = make_table_core(&sc, 1, &opts, false, T, false))) return rc;
    if (T.total_rays == 0 || view.n_leaves == 0) return SVLF_OK;
    const size_t stride = two_decoder_stride(*desc, T.total_rays, 1);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes_raw(T.total_rays, 1, stride, 1)) return SVLF_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws = carve_workspace_raw(workspace, T.total_rays, 1, stride, 1);
    const MlpDims mt = dims_t(*desc), mc = dims_c(*desc);
    const int fb = desc->feat_dtype == SVLF_FEAT_BF16;
    SceneTable Tc = T;
    Tc.s[0].feats = z_c;
    Tc.s[0].params = params_c;
    Tc.s[0].d_feat = d_z_c;
    Tc.s[0].d_params = d_params_c;
    T.s[0].d_feat = d_z_t;
    T.s[0].d_params = d_params_t;
    Workspace wc = ws;
    wc.packed_w = static_cast<char *>(ws.packed_w) + image_c_offset(*desc);
    float4 *aux = aux_of(ws, *desc);
    float *w_dD = w_dD_of(ws, *desc, T.total_rays, 1);
    float *deta = deta_of(ws, *desc, T.total_rays, 1);
    if (cudaMemsetAsync(ws.counter, 0, kCounterBytes, s) != cudaSuccess) return SVLF_ERR_CUDA;
    if ((rc = launch_pack_tc(mt, desc->precision, T, ws.packed_w, stride, s))) return rc;
    if ((rc = launch_pack_tc(mc, desc->precision, Tc, wc.packed_w, stride, s))) return rc;
    if ((rc = launch_surface_samples(T, depth_target, mask, ws.samples, deta, ws.counter, s))) return rc;
    if ((rc = launch_mlp_forward_tc(mt, desc->precision, fb, T, ws, s, 1, aux))) return rc;
    if ((rc = launch_mlp_forward_tc(mc, desc->precision, fb, Tc, wc, s, 2, aux))) return rc;
    if ((rc = launch_surface_loss(ws.samples, ws.counter, ws.outputs, aux, rgb_target, T.total_rays, lambda_eta,
                                  lambda_tau, ws.dout, deta, w_dD, ws.counter + kCtrMaxAbsDout, loss_accum, s)))
        return rc;
    if (!d_z_t && !d_z_c && !d_params_t && !d_params_c) return SVLF_OK;
    if ((rc = launch_mlp_backward_tc(mc, desc->precision, fb, Tc, wc, d_z_c != nullptr, d_params_c != nullptr, s,
                                     2, aux, w_dD, deta)))
        return rc;
    if (!d_z_t && !d_params_t) return SVLF_OK;
    return launch_mlp_backward_tc(mt, desc->precision, fb, T, ws, d_z_t != nullptr, d_params_t != nullptr, s, 1,
                                  aux, w_dD, nullptr);
}

extern "C" int svlf_eta_loss_two_decoder(svlf_octree tree, const svlf_two_decoder_desc *desc, const float *rays,
                                         int64_t n_rays, const svlf_render_opts *opts, const float *depth_target,
                                         const float *mask, float lambda_eta, double *loss_accum, void *workspace,
                                         size_t ws_bytes, void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    int rc = check_two_decoder(desc);
    if (rc) return rc;
    if (n_rays > 0 && (!depth_target || !loss_accum)) return SVLF_ERR_ARG;
    SceneTable T;
    std::memset(&T, 0, sizeof(T));
    if (!opts || opts->K < 1 || opts->K > kMaxK) return opts ? SVLF_ERR_UNSUPPORTED : SVLF_ERR_ARG;
    if (n_rays < 0) return SVLF_ERR_ARG;
    if (n_rays == 0) return SVLF_OK;
    T.n = 1;
    T.K = opts->K;
    T.s[0].tree = octree_view(tree);
    T.s[0].rays = rays;
    T.s[0].n_rays = n_rays;
    T.s[0].grad = 1;
    T.total_rays = T.grad_rays = n_rays;
    const size_t stride = two_decoder_stride(*desc, n_rays, T.K);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return SVLF_ERR_WORKSPACE;
    if (ws_bytes < workspace_bytes_raw(n_rays, T.K, stride, 1)) return SVLF_ERR_WORKSPACE;
    Workspace ws = carve_workspace_raw(workspace, n_rays, T.K, stride, 1);
    return launch_eta_term(T, ws.ray_span, aux_of(ws, *desc), depth_target, mask, lambda_eta,
                           deta_of(ws, *desc, n_rays, T.K), loss_accum, (cudaStream_t)stream);
}
