/*
 * svlf.h - C ABI of the SVLF hot path (sparse voxel light field rendering and
 * training) for NVIDIA B300 (sm_103a).
 *
 * The operations follow the method of "RTMV: A Ray-Traced Multi-View
 * Synthetic Dataset for Novel View Synthesis" (Sec. 4, Sparse Voxel Light
 * Field): a ray is mapped, voxel by voxel, to an optical thickness tau and a
 * colour c (Sec. 4, opening paragraph), and a pixel is the alpha composite of
 * the voxels the ray meets, in order (Sec. 4.3, Eq. 3).
 *
 * Conventions shared by every call:
 *  - Return value: SVLF_OK (0) or a negative SVLF_ERR_* code. Nothing aborts
 *    or throws across this boundary. Argument errors are reported before any
 *    work is queued. Device-side errors (a traversal step limit, an index out
 *    of range) are latched in a device status word read by
 *    svlf_get_device_status().
 *  - Pointers named "device" are CUDA device memory owned by the caller; the
 *    library never frees them. Pointers named "host" are host memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Gradients ACCUMULATE (+=) into caller-zeroed buffers.
 *  - A leaf (occupied finest-level voxel) is identified by its rank in
 *    ascending Morton order of its integer coordinates (i, j, k), with bit
 *    3b = bit b of i, 3b+1 = bit b of j, 3b+2 = bit b of k. The rank is the
 *    leaf's row in the feature table and the value reported in hit lists
 *    (-1 = empty slot).
 *  - Voxel (i, j, k) at depth L is the box [i, i+1] x [j, j+1] x [k, k+1] *
 *    2^-L inside the unit cube (Sec. 3.1 normalises every scene to a unit
 *    cube). Supported depths: 2 <= L <= 10.
 */
#ifndef SVLF_H
#define SVLF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SVLF_OK 0
#define SVLF_ERR_ARG (-1)          /* invalid argument (null pointer, size, range) */
#define SVLF_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define SVLF_ERR_DEVICE (-3)       /* a kernel latched an error (see device status) */
#define SVLF_ERR_UNSUPPORTED (-4)  /* shape or mode the library does not handle */
#define SVLF_ERR_WORKSPACE (-5)    /* workspace missing, misaligned or too small */

/* device status bits (svlf_get_device_status) */
#define SVLF_DEV_STEP_LIMIT 1      /* a traversal exceeded its step bound */
#define SVLF_DEV_BAD_INDEX 2       /* a node, brick or leaf index was out of range */
#define SVLF_DEV_SAMPLE_OVERFLOW 4 /* more samples than the workspace holds */
#define SVLF_DEV_WAIT_TIMEOUT 8    /* a bounded wait on an mbarrier gave up */

/* network arithmetic */
#define SVLF_FP32 0  /* SIMT float32 throughout */
#define SVLF_BF16 1  /* tcgen05 tensor cores, bfloat16 operands, float32 accumulate */
#define SVLF_FP16 2  /* tcgen05 tensor cores, float16 operands, float32 accumulate */

/* feature table storage */
#define SVLF_FEAT_F32 0
#define SVLF_FEAT_BF16 1

/* ------------------------------------------------------------------ types */
typedef struct svlf_octree_s *svlf_octree; /* opaque, library-owned */

/* The per-sample network. Input h0 = [z (feat_dim) | ray direction (3) |
 * p~1 (3) | p~2 (3)], in_dim = feat_dim + 9; n_hidden ReLU layers of width
 * `hidden`; a linear output layer of out_dim = 4 values [r, g, b, tau_pre].
 * Colour = sigmoid(r, g, b), optical thickness tau = max(tau_pre, 0)
 * (Sec. 4.5 "Architecture": ReLU decoders, sigmoid colour, ReLU thickness).
 * Parameters are one flat float32 array: for each layer, W (out x in,
 * row-major) followed by b (out). */
typedef struct {
    int feat_dim;   /* F: 8..64, multiple of 8 */
    int hidden;     /* H: 32..256, multiple of 16. Tensor-core precisions: H <= 128
                       (padded to 128 inside). SVLF_FP32: H in {32, 64, 128, 256}; its
                       forward needs two 128-sample activation tiles in shared memory
                       and its backward every layer's activations for 64 samples
                       (H <= 128, up to 4 x 128 or 6 x 64); calls outside these
                       return SVLF_ERR_UNSUPPORTED */
    int n_hidden;   /* 1..6 */
    int out_dim;    /* must be 4 */
    int precision;  /* SVLF_FP32 | SVLF_BF16 | SVLF_FP16 */
    int feat_dtype; /* SVLF_FEAT_F32 | SVLF_FEAT_BF16 */
} svlf_mlp_desc;

/* Ray parameterisation r of the network input (Sec. 4.1 "Ray
 * parameterization"; the text takes the bounding-sphere points relative to
 * the "voxel origin", which it does not define further):
 *   SVLF_RPARAM_SPHERE (default): r = [p~1 | p~2], the ray's entry and exit
 *     points on the voxel's minimum bounding sphere (centre c = the voxel
 *     centre (ijk + 1/2) 2^-L, radius (sqrt(3)/2) 2^-L), taken from c and
 *     scaled to unit norm;
 *   SVLF_RPARAM_AABB: r = [x~1 | x~2], the ray's entry and exit points of the
 *     voxel box itself (its slab segment, entry clipped at t = 0), in
 *     voxel-local coordinates (x - c) / (2^-L / 2), each component in
 *     [-1, 1] (the "local entry/exit points" reading, with the voxel's own
 *     frame as the origin). */
#define SVLF_RPARAM_SPHERE 0
#define SVLF_RPARAM_AABB 1

typedef struct {
    int K;        /* hits evaluated per ray (the first K leaves): 1..32 */
    float bg[3];  /* colour multiplied by the transmittance left after the K-th hit */
    int rparam_mode; /* SVLF_RPARAM_SPHERE or SVLF_RPARAM_AABB (the single-network
                      * calls; the two-decoder calls take SVLF_RPARAM_SPHERE only) */
    int image_width; /* traversal order only (results do not depend on it): 0 =
                      * the rays' own order; W > 0 = the rays are the pixels of
                      * images W wide, row-major, one image after another, and
                      * are walked in tiles of 8 x 4 pixels, so that the 32 rays
                      * a warp walks together are neighbours in both directions.
                      * Applies to each scene whose ray count is a multiple of
                      * 4 W with W a multiple of 8; other scenes keep their
                      * order. Negative: SVLF_ERR_ARG. */
} svlf_render_opts;

/* ------------------------------------------------------------ octree */
/* Build the sparse octree over the given leaves (Sec. 4.1 "Scene volume":
 * only voxels that contain a surface are stored), on the GPU: each leaf sets
 * one bit of a Morton-indexed occupancy bitmap (duplicates merge), prefix
 * scans give the brick and leaf ranks and the node levels, and the parent
 * index with its grown empty boxes is built from them.
 *   leaf_ijk: device, n x 3 int32 (i, j, k); duplicates are merged.
 *   depth: L, 2..10. Coordinates must lie in [0, 2^L), else SVLF_ERR_ARG
 *     (counted on the device and checked before the build goes on).
 *   out: receives the handle. n_leaves_out (host, may be NULL): unique leaves.
 * Synchronises `stream`; allocates 2^(3 depth) bits of temporary device
 * memory (128 MB at depth 10). Not on the per-frame path. */
int svlf_build_octree(const int32_t *leaf_ijk, int64_t n, int depth, void *stream,
                      svlf_octree *out, int64_t *n_leaves_out);

/* The same octree built on the host (the leaf list is copied to the host,
 * sorted and de-duplicated there, and the arrays uploaded): an independent
 * construction of the arrays svlf_build_octree builds, kept for checking one
 * against the other. Same arguments and errors; synchronises `stream`. */
int svlf_build_octree_host(const int32_t *leaf_ijk, int64_t n, int depth, void *stream,
                           svlf_octree *out, int64_t *n_leaves_out);

/* Builds the octree on the GPU from depth maps (Sec. 4.1: the voxel grid
 * comes from the dataset's depth maps; Sec. 4.5: 128^3, i.e. depth 7). Pixel
 * p (rays: device n x 6 float32, origin and unit direction; depth: device n
 * float32) marks the leaf floor((o + D d) 2^depth_levels) (clamped to the
 * grid; the point is formed as the product D d rounded, then the sum rounded);
 * pixels with a non-finite or non-positive depth are skipped. The result is
 * the same octree svlf_build_octree gives for those leaves. Synchronises
 * `stream`; allocates 2^(3 depth_levels) bits of temporary device memory
 * (128 MB at depth 10). */
int svlf_build_octree_from_depth(const float *rays, const float *depth, int64_t n, int depth_levels,
                                 void *stream, svlf_octree *out, int64_t *n_leaves_out);

/* Leaf coordinates in rank order. out_ijk: device, n_leaves x 3 int32. */
int svlf_octree_leaf_ijk(svlf_octree tree, int32_t *out_ijk, void *stream);

/* The dense parent index the traversal reads (inspection and tests): one
 * entry of two uint32 per level L-3 cell, (2^(L-3))^3 entries, x fastest.
 * Entry = (node word, 0) where the cell's node exists (bits 24..31 = child
 * mask, bits 0..23 = index of its first child brick); else (lo, hi), an
 * empty box of level L-3 cells around the cell, lo = x | y << 8 | z << 16
 * inclusive, hi exclusive, with bits 24..31 zero. The box is the largest
 * empty octree block holding the cell, grown face by face (x, y, z; low face
 * then high) by slabs that hold no leaf, each face's slab doubling after a
 * success and halving after a failure, until no face can grow by one layer.
 * out: device, 2 x *n_entries uint32, or NULL to query *n_entries (host; 0
 * for depths below 3 or an empty tree). */
int svlf_octree_parent_index(svlf_octree tree, uint32_t *out, int64_t *n_entries, void *stream);

/* Sizes: depth, leaves, internal node words, leaf bricks (host outputs, any
 * may be NULL). */
int svlf_octree_info(svlf_octree tree, int *depth, int64_t *n_leaves, int64_t *n_nodes,
                     int64_t *n_bricks);

int svlf_free_octree(svlf_octree tree);

/* ------------------------------------------------------------ rendering */
/* Pinhole cameras: rays generated on the device (row a1's optional in-kernel
 * ray generation; the rays of svlf_render_rays are otherwise the caller's).
 * eye: the centre of projection; fwd, right, up: an orthonormal basis (the
 * viewing direction, the image's +x and +y); tan_half_fov: tan of half the
 * (square) field of view. */
typedef struct {
    float eye[3];
    float fwd[3];
    float right[3];
    float up[3];
    float tan_half_fov;
} svlf_camera;

/* rays_out (device, n_views x height x width x 6 float32; view-major, then
 * row-major over pixels) receives, for pixel (r, c) of view v, origin eye
 * and the unit direction of fwd + x right + y up with x = (2 (c + 1/2) /
 * width - 1) tan_half_fov, y = (1 - 2 (r + 1/2) / height) tan_half_fov,
 * normalised in float32 (within a few ulp of the same formula in FP64).
 * cams: host, n_views cameras (copied into the launch). Errors: SVLF_ERR_ARG
 * for a null pointer, n_views < 1 or a non-positive size. */
int svlf_pinhole_rays(const svlf_camera *cams, int n_views, int width, int height, float *rays_out,
                      void *stream);

/* Bytes of workspace a render (and the matching backward) needs. */
int svlf_workspace_size(const svlf_mlp_desc *mlp, int64_t n_rays, int K, size_t *bytes);

/* Render rays (Sec. 4.3): for each ray, the first K leaves it meets in
 * ascending t (slab test, Sec. 4.2), each evaluated once by the network on
 * [z | d | r] with r = [p~1 | p~2] the ray's entry and exit points on the
 * leaf's minimum bounding sphere, relative to the leaf centre and scaled to
 * unit norm (Sec. 4.1 "Ray parameterization"), then composited by Eq. 3:
 *   C = sum_i T_i (1 - exp(-tau_i)) c_i + T_{n+1} bg,  T_i = prod_{j<i} exp(-tau_j)
 *   D = sum_i T_i (1 - exp(-tau_i)) (t_in,i + t_out,i) / 2      (0 if no hit)
 * Arguments (all device unless noted):
 *   features: n_leaves x feat_dim, float32 or bfloat16 (mlp->feat_dtype),
 *             row-major, 16-byte aligned rows.
 *   mlp_params: flat float32 parameters (layout in svlf_mlp_desc).
 *   rays: n_rays x 6 float32 (ox, oy, oz, dx, dy, dz), |d| = 1.
 *   rgb: n_rays x 3 float32 out; depth: n_rays float32 out.
 *   hits: n_rays x K int32 out (leaf ranks, -1 = none) or NULL.
 *   t_io: n_rays x K x 2 float32 out (t_in, t_out) or NULL.
 *   workspace: >= svlf_workspace_size() bytes, 256-byte aligned. The samples
 *             and network outputs it holds afterwards are what
 *             svlf_render_rays_backward() reads: pass it unchanged.
 * Errors: SVLF_ERR_ARG / _UNSUPPORTED / _WORKSPACE before launch. */
int svlf_render_rays(svlf_octree tree, const void *features, const float *mlp_params,
                     const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                     const svlf_render_opts *opts, float *rgb, float *depth, int32_t *hits,
                     float *t_io, void *workspace, size_t ws_bytes, void *stream);

/* Backward of svlf_render_rays with respect to the features and the network
 * parameters, given d_rgb (n_rays x 3) and d_depth (n_rays) (device). Reads
 * the samples and outputs the forward call left in `workspace` (same tree,
 * features, parameters, rays and options), recomputes the network
 * activations, and accumulates into d_features (n_leaves x feat_dim float32)
 * and d_mlp_params (flat float32, same layout as mlp_params). Either output
 * may be NULL to skip it. */
int svlf_render_rays_backward(svlf_octree tree, const void *features, const float *mlp_params,
                              const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                              const svlf_render_opts *opts, const float *d_rgb,
                              const float *d_depth, float *d_features, float *d_mlp_params,
                              void *workspace, size_t ws_bytes, void *stream);

/* Training loss over n rays (device buffers):
 *   L = (1/n) sum_r [ |C_r - C*_r|^2 + depth_weight * m_r |D_r - D*_r| ]
 * Writes dL/dC (n x 3) into d_rgb and dL/dD (n) into d_depth (overwritten,
 * sign(0) = 0) and adds L to *loss_accum (device double). */
int svlf_loss(const float *rgb, const float *depth, const float *rgb_target,
              const float *depth_target, const float *mask, int64_t n, float depth_weight,
              float *d_rgb, float *d_depth, double *loss_accum, void *stream);

/* The loss of one shard of a training batch of n_total rays split across
 * ranks (data-parallel training over the ray batch): the same per-ray terms
 * over this shard's n rays, divided by n_total instead of n,
 *   L_shard = (1/n_total) sum_{r in shard} [ |C_r - C*_r|^2 + w m_r |D_r - D*_r| ],
 * with d_rgb, d_depth scaled alike. The shards' losses, and therefore their
 * gradients after the backward, sum exactly to the whole batch's mean loss
 * and its gradient, so one all-reduce (sum) of the gradient buffers completes
 * the batch's gradient on every rank. svlf_loss is the case n_total = n.
 * Errors: SVLF_ERR_ARG also for n_total < n. */
int svlf_loss_shard(const float *rgb, const float *depth, const float *rgb_target,
                    const float *depth_target, const float *mask, int64_t n, int64_t n_total,
                    float depth_weight, float *d_rgb, float *d_depth, double *loss_accum, void *stream);

/* ------------------------------------------------------------ batched form */
/* Many scenes of uneven octree size in one call (one launch per kernel for
 * all of them; the calls queue no host-device copy and can be captured in a
 * CUDA graph). Each scene has its own octree, features, network parameters
 * (same network shape for all, given by `mlp`), rays and outputs. All device
 * pointers as in svlf_render_rays; the d_* members are only read or written
 * by the backward call. Up to 64 scenes per call; the tensor-core precisions
 * (SVLF_BF16, SVLF_FP16) handle any number, SVLF_FP32 a single scene. */
typedef struct {
    svlf_octree tree;
    const void *features;       /* n_leaves x feat_dim, fp32 or bf16 */
    const float *mlp_params;    /* flat float32 network parameters */
    const float *rays;          /* n_rays x 6 */
    int64_t n_rays;
    float *rgb, *depth;         /* render outputs: n_rays x 3, n_rays */
    const float *d_rgb, *d_depth;      /* backward inputs */
    float *d_features, *d_mlp_params;  /* backward outputs (accumulate), or NULL */
} svlf_scene;

/* Workspace for a batched call over n_scenes scenes and total_rays rays. */
int svlf_workspace_size_batched(const svlf_mlp_desc *mlp, int64_t total_rays, int n_scenes, int K,
                                size_t *bytes);

/* Render every scene (Sec. 4.3; see svlf_render_rays). The workspace keeps
 * what the matching batched backward reads. */
int svlf_render_rays_batched(const svlf_scene *scenes, int n_scenes, const svlf_mlp_desc *mlp,
                             const svlf_render_opts *opts, void *workspace, size_t ws_bytes,
                             void *stream);

/* Backward of svlf_render_rays_batched for every scene (see
 * svlf_render_rays_backward). Either gradient may be skipped by passing NULL
 * for it in every scene. A scene whose d_rgb and d_depth are both NULL takes
 * no part: its samples are not differentiated and its d_features and
 * d_mlp_params are not touched (so rays that are only rendered, e.g. the views
 * of a training step, can share the render call with the rays that are
 * trained on). Errors: SVLF_ERR_ARG when exactly one of a scene's d_rgb,
 * d_depth is NULL. */
int svlf_render_rays_backward_batched(const svlf_scene *scenes, int n_scenes,
                                      const svlf_mlp_desc *mlp, const svlf_render_opts *opts,
                                      void *workspace, size_t ws_bytes, void *stream);

/* Samples (hits evaluated) that the last batched render or backward wrote
 * into `workspace`, summed over the scenes (host result; synchronises
 * `stream`). n_rays: host, n_scenes ray counts, as in the call. */
int svlf_workspace_samples_batched(const void *workspace, const svlf_mlp_desc *mlp, const int64_t *n_rays,
                                   int n_scenes, int K, int64_t *n_samples, void *stream);

/* The same per scene: per_scene (host, n_scenes entries) receives each
 * scene's samples. */
int svlf_workspace_scene_samples(const void *workspace, const svlf_mlp_desc *mlp, const int64_t *n_rays,
                                 int n_scenes, int K, int64_t *per_scene, void *stream);

/* ------------------------------------------------ two-decoder form (Sec. 4.1-4.2) */
/* The paper's full SVLF: features live on octree vertices (Sec. 4.1 "Scene
 * volume": one vector per leaf corner, shared by the voxels meeting there)
 * and are trilinearly interpolated, psi(p; Z). For each hit voxel with
 * entry / exit points x1, x2 (Sec. 4.2):
 *   tau, eta = F^T([psi(x1; Z^T) | psi(x2; Z^T) | p~1 | p~2])      (Eq. 1)
 *   x_s = eta x1 + (1 - eta) x2
 *   c = F^C([psi(x_s; Z^C) | p~1 | p~2])                            (Eq. 2)
 * with ReLU hidden layers, ReLU on tau, sigmoid on eta and c (Sec. 4.5), then
 * Eq. 3 compositing; a hit's depth is the ray parameter of x_s. */

/* Builds (once; later calls only report) the octree's vertex table: the
 * corners of every leaf, de-duplicated, ids = ranks of the corner lattice
 * points (depth + 1 bits per axis) in Morton order. Synchronises `stream`;
 * allocates n_leaves x 8 int32 on the device, freed with the octree. */
int svlf_octree_build_vertices(svlf_octree tree, int64_t *n_vertices, void *stream);
/* Copies the table to out (device, n_leaves x 8 int32, rank order): entry
 * 8 q + a + 2b + 4c is the vertex id of corner (a, b, c) of leaf q.
 * SVLF_ERR_ARG if the table was not built. */
int svlf_octree_leaf_vertices(svlf_octree tree, int32_t *out, void *stream);

typedef struct {
    int feat_t, feat_c;          /* Z^T and Z^C widths, 8..64, multiples of 8 (paper: 64, 32) */
    int hidden_t, n_hidden_t;    /* F^T: hidden width 32..128 (multiple of 16), 1..4 layers (paper: 128, 1) */
    int hidden_c, n_hidden_c;    /* F^C: the same (paper: 128, 3) */
    int precision;               /* SVLF_BF16 or SVLF_FP16 (tensor cores); SVLF_FP32: unsupported */
    int feat_dtype;              /* storage of Z^T and Z^C: SVLF_FEAT_F32 or SVLF_FEAT_BF16 */
} svlf_two_decoder_desc;

int svlf_workspace_size_two_decoder(const svlf_two_decoder_desc *desc, int64_t n_rays, int K,
                                    size_t *bytes);

/* Render n_rays rays with the two-decoder form. z_t: device, n_vertices x
 * feat_t, z_c: n_vertices x feat_c (16-byte aligned rows, vertex ids of the
 * table above). params_t / params_c: device float32, per layer W (out x in,
 * row-major) then b; F^T maps 2 feat_t + 6 inputs to (tau_pre, eta_pre), F^C
 * maps feat_c + 6 inputs to colour pre-activations. rays, opts, rgb, depth,
 * hits, t_io, workspace as in svlf_render_rays. The vertex table must have
 * been built (SVLF_ERR_ARG otherwise). */
int svlf_render_rays_two_decoder(svlf_octree tree, const void *z_t, const void *z_c,
                                 const float *params_t, const float *params_c,
                                 const svlf_two_decoder_desc *desc, const float *rays, int64_t n_rays,
                                 const svlf_render_opts *opts, float *rgb, float *depth,
                                 int32_t *hits, float *t_io, void *workspace, size_t ws_bytes,
                                 void *stream);

/* Backward of svlf_render_rays_two_decoder with the workspace of that render
 * (same inputs; it reuses the render's samples, outputs and per-sample
 * (tau, eta, t_in, t_out)). Accumulates (+=) into d_z_t (n_vertices x feat_t
 * float32), d_z_c (n_vertices x feat_c), d_params_t, d_params_c (layouts of
 * z_t, z_c, params_t, params_c); any of them may be NULL. The adjoint runs
 * through Eq. 3, F^C, the trilinear scatter to the corners, the surface point
 * (x_s depends on eta: dL/deta = (dL/dx_s . d + w dL/dD)(t_in - t_out)) and
 * F^T. Float16 operands scale the deltas by a power of two as in
 * svlf_render_rays_backward. */
int svlf_render_rays_backward_two_decoder(svlf_octree tree, const void *z_t, const void *z_c,
                                          const float *params_t, const float *params_c,
                                          const svlf_two_decoder_desc *desc, const float *rays,
                                          int64_t n_rays, const svlf_render_opts *opts,
                                          const float *d_rgb, const float *d_depth, float *d_z_t,
                                          float *d_z_c, float *d_params_t, float *d_params_c,
                                          void *workspace, size_t ws_bytes, void *stream);

/* Staged training of the two-decoder form (Sec. 4.4, Eq. 4).
 * Stage 1 (voxel training): every ray with mask > 0 (mask may be NULL = all)
 * and a finite surface depth D* (depth_target, device, n_rays float32) is
 * evaluated at one voxel, the leaf containing o + D* d (skipped if that cell
 * is empty or the ray's segment through it is empty); with
 * eta* = (t_out - D*) / (t_out - t_in) clamped to [0, 1] (the within-voxel
 * depth of the surface point), it adds to *loss_accum (device double)
 *   (1/n_rays) sum_v |c_v - c*|^2 + lambda_eta (eta_v - eta*)^2
 *                    + lambda_tau exp(-tau_v)^2
 * (rgb_target: device, n_rays x 3 float32) and accumulates the gradients
 * (any may be NULL). Workspace: svlf_workspace_size_two_decoder(desc, n_rays,
 * 1). The paper gives no values for lambda_eta, lambda_tau. */
int svlf_surface_loss_two_decoder(svlf_octree tree, const void *z_t, const void *z_c,
                                  const float *params_t, const float *params_c,
                                  const svlf_two_decoder_desc *desc, const float *rays, int64_t n_rays,
                                  const float *rgb_target, const float *depth_target, const float *mask,
                                  float lambda_eta, float lambda_tau, double *loss_accum, float *d_z_t,
                                  float *d_z_c, float *d_params_t, float *d_params_c, void *workspace,
                                  size_t ws_bytes, void *stream);
/* Stages 2-3 (volumetric training): after svlf_render_rays_two_decoder and
 * before its backward, on the same workspace and rays: adds
 * lambda_eta (eta_v - eta*)^2 / n_rays over each ray's surface voxel among
 * its hits (the first hit whose segment contains D*) to *loss_accum and
 * records the term's gradient for the backward. (Stage 2 freezes Z^C and F^C:
 * pass NULL for their gradients to the backward.) */
int svlf_eta_loss_two_decoder(svlf_octree tree, const svlf_two_decoder_desc *desc, const float *rays,
                              int64_t n_rays, const svlf_render_opts *opts, const float *depth_target,
                              const float *mask, float lambda_eta, double *loss_accum, void *workspace,
                              size_t ws_bytes, void *stream);

/* ------------------------------------------------------------ optimiser */
/* One bias-corrected Adam step (Sec. 4.5 trains with Adam; Kingma & Ba) over
 * n float32 parameters (device): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
 * p <- p - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * step >= 1. If bf16_shadow (device, n bfloat16) is not NULL, the updated
 * parameters are also written there rounded to bfloat16. */
int svlf_adam_step(float *params, const float *grads, float *m, float *v, int64_t n, float lr,
                   float beta1, float beta2, float eps, int64_t step, void *bf16_shadow,
                   void *stream);

/* svlf_adam_step with the step count read from device memory when the
 * kernels run (step: device, one int64_t, values < 1 act as 1), so that a
 * captured CUDA graph that replays a whole training step, Adam included,
 * needs no host argument that changes from step to step. The bias
 * corrections 1 / (1 - beta^t) are formed in float64 by the same sequence of
 * multiplications as in svlf_adam_step, so both give identical results for
 * the same step. */
int svlf_adam_step_device(float *params, const float *grads, float *m, float *v, int64_t n, float lr,
                          float beta1, float beta2, float eps, const int64_t *step, void *bf16_shadow,
                          void *stream);

/* Adds one to the device step counter of svlf_adam_step_device (device, one
 * int64_t), queued on `stream`: one launch at the start of each training
 * step's optimiser phase. */
int svlf_step_advance(int64_t *step, void *stream);

/* ------------------------------------------------------------ status */
/* Reads and clears the device status word (bitwise OR of SVLF_DEV_*) in one
 * atomic exchange queued on `stream`, after the work already queued there,
 * then synchronises `stream` only and writes the value to *status (host).
 * Bits latched by work on other streams that has not finished yet are left
 * for a later read. Two reads that overlap on different streams share one
 * device-side result slot: issue reads from one host thread at a time.
 * Errors: SVLF_ERR_ARG for a null `status`, SVLF_ERR_CUDA if the launch or
 * copy fails. */
int svlf_get_device_status(void *stream, int *status);

/* Safety bound of the traversal (process-wide): a ray that has taken more
 * than max_steps walk steps (cells or empty boxes visited; the bound is
 * checked between rounds of trace_budget steps, so a ray may overrun it by
 * one round) stops with the hits found so far and latches
 * SVLF_DEV_STEP_LIMIT. A walk over the finest grid of depth L never needs
 * more than 3 * 2^L steps, so the default (max_steps = 0) of 3 * 2^L + 64
 * trips only on a corrupted octree. Lower values truncate real walks: they
 * serve to exercise the error path. Errors: SVLF_ERR_ARG outside
 * [0, 2^30]. */
int svlf_set_step_limit(int64_t max_steps);

const char *svlf_status_string(int status);

/* ------------------------------------------------------------ no allocation */
/* svlf_render_rays for callers that cannot allocate device memory: hosts that
 * give a renderer a fixed device-memory budget at start-up and forbid later
 * allocations, and frame loops that must not call cudaMalloc because it can
 * synchronise the device. The paper has no counterpart; this is a deployment
 * variant of svlf_render_rays with the same arguments minus the workspace and
 * the optional hit outputs.
 * Its scratch is a fixed 32 MiB array inside the library (every GPU that
 * loads the library holds it until exit). A call fits when
 * svlf_workspace_size(mlp, n_rays, K) <= 32 MiB, e.g. about 85 000 rays at
 * K = 8 for a 41 -> 3 x 128 -> 4 network; larger calls return
 * SVLF_ERR_WORKSPACE before any work is queued. The call allocates nothing.
 * All calls share the array and it keeps the previous call's contents (the
 * sample counter is cleared by each call): calls that overlap on the GPU
 * race. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for that device's current context;
 * make that first call before any stream capture. After cudaDeviceReset the
 * library is loaded into a new context at a possibly different address: the
 * next call sees the new context and looks the address up again. */
int svlf_render_rays_static(svlf_octree tree, const void *features, const float *mlp_params,
                            const svlf_mlp_desc *mlp, const float *rays, int64_t n_rays,
                            const svlf_render_opts *opts, float *rgb, float *depth, void *stream);

/* ------------------------------------------------------------ tuning */
/* Launch-shape knobs (process-wide; 0 = the library's default). The
 * autotuner (paper_2205_07058_b300/autotune.py) times candidates on the
 * caller's workload and sets the best. They change speed, never results.
 *   mlp_warpgroups      tensor-core forward: tiles in flight per CTA, 1..4
 *                       (the two-decoder F^T pass runs at most 3)
 *   mlp_epilogue_batch  tensor-core forward, hidden-layer epilogue: 1 = 32
 *                       TMEM columns per load and wait, 2 = 64 (limits the
 *                       CTA to 3 warpgroups), 3 = 16 with the next load in
 *                       flight while a chunk is packed
 *   trace_budget        traversal steps between lane refills, 1..256
 *                       (default 64)
 *   trace_block         traversal threads per block, 128 or 256
 *   trace_refill        traversal: idle lanes a warp needs before it claims
 *                       a new work item of 32 neighbouring rays while rays
 *                       of its earlier ones still walk, 1..32 (32: only once
 *                       all lanes are idle; default 32 for large launches,
 *                       with at least two work items per resident warp, 16
 *                       for smaller ones)
 *   mlp_bwd_warpgroups  tensor-core backward: warpgroups per tile, 1 or 2
 *                       (2 adds a second warpgroup that takes half of every
 *                       epilogue; used for the plain form with resident
 *                       weights in one pass; default 2 there) */
typedef struct {
    int mlp_warpgroups;
    int mlp_epilogue_batch;
    int trace_budget;
    int trace_block;
    int trace_refill;
    int mlp_bwd_warpgroups;
} svlf_tuning;

int svlf_set_tuning(const svlf_tuning *t);
int svlf_get_tuning(svlf_tuning *t);

/* ------------------------------------------------------------ measurement */
/* Per-kernel timing (measurement aid, not part of the method). When enabled,
 * every kernel the library launches is bracketed by CUDA events on its own
 * launch stream. svlf_profile_report() synchronises the device, writes up to
 * max_entries per-kernel sums into `out` (host), the number of distinct
 * kernels into *n_entries, and clears the record. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} svlf_kernel_stat;

int svlf_profile_enable(int on);
int svlf_profile_report(svlf_kernel_stat *out, int max_entries, int *n_entries);

/* Number of (ray, hit) samples the last render left in `workspace` (device
 * counter copied to *n_samples on the host; synchronises `stream`). */
int svlf_workspace_samples(const void *workspace, const svlf_mlp_desc *mlp, int64_t n_rays, int K,
                           int64_t *n_samples, void *stream);

/* ------------------------------------------------------------ self-test */
/* Test aid, not part of the rendering method: D = A B^T for one tile through
 * the tensor cores, with the operands staged in the shared-memory layouts the
 * network kernels use (K-major, or MN-major when the flag is set).
 * A: device, 128 x K 16-bit values (bf16 if bf16 != 0, else f16), row-major.
 * B: device, N x K, row-major. D: device, 128 x N float32.
 * N in {16, 32, ..., 256}, K in {16, 32, ..., 256}. flags (layout diagnosis,
 * 0 for the kernels' convention): bit 0 exchanges the two descriptor byte
 * offsets, bit 1 stages B before A, bits 2 / 3 start the B / A descriptor
 * 16 bytes later; bit 5 reads A from tensor memory instead (row m in lane m,
 * element pairs packed per 32-bit column; requires a_mn_major = 0). */
int svlf_selftest_mma(const uint16_t *A, const uint16_t *B, float *D, int N, int K,
                      int a_mn_major, int b_mn_major, int bf16, int flags, void *stream);

/* Measurement aid, not part of the rendering method: a float32 FMA
 * throughput kernel, the denominator of the FP32 SIMT network's roofline.
 * Launches one grid of `blocks` x 256 threads; each thread runs `iters`
 * rounds of 16 independent fmaf chains (32 flop per round), so the launch
 * does blocks x 256 x iters x 32 flop; the caller times it on `stream`.
 * out: device, `blocks` floats (written only to keep the work live).
 * Errors: SVLF_ERR_ARG for blocks < 1 or iters < 1. */
int svlf_selftest_ffma(float *out, int blocks, int64_t iters, void *stream);

/* Test aid, not part of the rendering method: the bounded mbarrier wait that
 * every kernel uses. One thread waits for a barrier phase that completes only
 * if `arrive` != 0, giving up after `limit_cycles` SM clocks (1 .. 4e9). When
 * it gives up it latches SVLF_DEV_WAIT_TIMEOUT in the device status, as a
 * kernel does when a copy or MMA it waits for never completes, and returns, so
 * the context stays usable.
 * out: device, 2 int64: [0] = 1 if the phase completed, 0 if the wait gave
 * up; [1] = SM clocks spent waiting.
 * Errors: SVLF_ERR_ARG for a null `out` or a limit out of range. */
int svlf_selftest_wait(int64_t limit_cycles, int arrive, int64_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SVLF_H */
