// Internal declarations shared by the CUDA translation units of libsvlf.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/svlf.h"

namespace svlf {

constexpr int kMaxDepth = 10;
constexpr int kMaxK = 32;

// ---------------------------------------------------------------- octree
// Device layout of the sparse octree (built in octree.cu):
//  * node words for levels 0 .. L-3, level-major, Morton order inside a level:
//      bits 31..24 child mask (bit o set = child octant o occupied,
//      octant bit 0 = x, 1 = y, 2 = z), bits 23..0 index of the first child
//      (into the node words for levels < L-3, into the bricks for level L-3).
//  * bricks = the occupied nodes of level L-2, each covering 4^3 leaves:
//      x, y = 64-bit leaf mask (bit = Morton code of the leaf inside the brick),
//      z = rank of the brick's first leaf, w = 0.
//  Leaf rank = brick.z + popcount(mask & ((1 << bit) - 1)).
struct OctreeView {
    int depth;
    int n_node_levels;  // L - 2
    int64_t n_leaves;
    int n_nodes, n_bricks;
    const uint32_t *nodes;
    const uint4 *bricks;
    // (2^(L-3))^3 entries, x fastest, one per level L-3 cell (a parent of
    // bricks). .x: the cell's node word where that node exists. Else .x has a
    // zero mask byte and the low corner of an empty box around the cell, in
    // level L-3 cells (x | y << 8 | z << 16), and .y its exclusive high
    // corner: the largest empty octree block holding the cell, grown face by
    // face while it stays empty (grow_empty_box)
    const uint2 *pgrid;
    int pgrid_shift;    // L - 3 (0 when L = 2)
    int root_is_brick;  // depth 2: the root itself is the only brick
    int empty;          // no leaves
    // vertex table (two-decoder form, built on request): vertex id of corner
    // (a, b, c) of leaf q at leaf_vertices[8 q + a + 2b + 4c]; null until built
    const int32_t *leaf_vertices;
    int64_t n_vertices;
};

struct OctreeHost {
    OctreeView view;
    int32_t *leaf_ijk_dev;  // n_leaves x 3, rank order
    uint32_t *nodes_dev;
    uint4 *bricks_dev;
    uint2 *pgrid_dev;
    int32_t *vtx_dev;       // n_leaves x 8 vertex ids, or null
};

// ---------------------------------------------------------------- samples
// One record per (ray, hit): leaf rank, ray index, packed voxel coordinates
// (i | j << 10 | k << 20), segment midpoint (t_in + t_out)/2 as float bits.
struct __align__(16) Sample {
    int32_t leaf;
    int32_t ray;
    uint32_t cell;
    float tmid;
};

// ---------------------------------------------------------------- scenes
// One render / backward call covers up to kMaxScenes scenes, each with its
// own octree, features, network parameters, rays and outputs (the batched
// form; a single-scene call is a table of one). The table travels by value
// as a kernel parameter, so a call needs no host-to-device copy and can be
// captured in a CUDA graph.
constexpr int kMaxScenes = 64;
constexpr int kTraceChunk = 32;  // rays per traversal work item (one warp: one ray per lane)

struct SceneDev {
    OctreeView tree;
    const void *feats;
    const float *params;  // flat float32 network parameters
    const float *rays;
    float *rgb, *depth;
    const float *d_rgb, *d_depth;
    float *d_feat, *d_params;
    int64_t ray_begin;    // first global ray index of the scene
    int64_t n_rays;
    int64_t chunk_begin;  // first traversal chunk of the scene
    // backward: the scene takes part (it has output gradients), and the index of
    // its first ray among the rays of the scenes that take part
    int grad;
    // traversal order: 0 = the given order; W = the rays are rows of images W
    // pixels wide, walked in tiles of 8 x 4 pixels (one work item each)
    int tile_w;
    int64_t grad_begin;
};

struct SceneTable {
    int n;
    int K;
    int64_t total_rays;
    int64_t total_chunks;
    int rparam;      // ray parameterisation of the network input (SVLF_RPARAM_*)
    int64_t grad_rays;  // backward: rays of the scenes that take part
    SceneDev s[kMaxScenes];
};

// Backward: index of the scene holding the `i`-th ray among the rays of the
// scenes that take part (grad_begin is non-decreasing; scenes that take no
// part, or have no rays, hold none and tie with the next, so the last scene
// whose grad_begin <= i is the one).
__host__ __device__ __forceinline__ int scene_of_grad_ray(const SceneTable &T, int64_t i) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.s[mid].grad_begin <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Index of the scene holding global ray g (the table is sorted by ray_begin).
__host__ __device__ __forceinline__ int scene_of_ray(const SceneTable &T, int64_t g) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.s[mid].ray_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ __forceinline__ int scene_of_chunk(const SceneTable &T, int64_t c) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.s[mid].chunk_begin <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Counters at the start of the workspace's counter block.
constexpr int kCtrMaxAbsDout = 3;    // float bits of max |dL/d(network output)|
constexpr int kCtrTraceChunks = 4;   // traversal work items claimed
constexpr int kCtrScene = 16;        // + s: samples written for scene s
constexpr size_t kCounterBytes = 4096;

// Workspace layout (byte offsets from a 256-aligned base). Scene s owns the
// sample slots [K * ray_begin_s, K * (ray_begin_s + n_rays_s)).
struct Workspace {
    Sample *samples;       // total_rays*K
    float4 *outputs;       // total_rays*K: sigmoid colour (xyz), tau (w)
    float4 *dout;          // total_rays*K: dL/d(network output)
    int2 *ray_span;        // total_rays: first sample, count
    unsigned int *counter; // see kCtr*
    void *packed_w;        // network weights packed for the kernels, per scene
    size_t packed_stride;  // bytes between the packed weights of consecutive scenes
    size_t bytes;
};

Workspace carve_workspace(void *base, const svlf_mlp_desc &mlp, int64_t n_rays, int K,
                          int n_scenes = 1);
size_t workspace_bytes(const svlf_mlp_desc &mlp, int64_t n_rays, int K, int n_scenes = 1);
size_t packed_weight_bytes(const svlf_mlp_desc &mlp);

// ---------------------------------------------------------------- device status
extern __device__ unsigned int g_device_status;

__device__ __forceinline__ void raise_status(unsigned int bit) {
    atomicOr(&g_device_status, bit);
}

// ---------------------------------------------------------------- launches
int launch_trace(const SceneTable &T, const Workspace &ws, int32_t *hits, float *t_io,
                 cudaStream_t s);
int launch_composite(const SceneTable &T, const Workspace &ws, const float bg[3], cudaStream_t s);
int launch_composite_backward(const SceneTable &T, const Workspace &ws, const float bg[3],
                              cudaStream_t s, float *w_dD = nullptr);
int launch_pack_weights(const svlf_mlp_desc &mlp, const SceneTable &T, const Workspace &ws,
                        cudaStream_t s);

int num_sms();

// process-wide launch-shape settings (svlf_set_tuning), with defaults filled in
const svlf_tuning &tuning();

// traversal step bound per ray set by svlf_set_step_limit (0: 3 * 2^L + 64)
extern int g_step_limit;

// per-kernel timing (profile.cu); no-ops unless svlf_profile_enable(1)
void prof_begin(const char *name, cudaStream_t s);
void prof_end(cudaStream_t s);

// ---------------------------------------------------------------- geometry
// Ray parameterisation r = [p~1 | p~2] (Sec. 4.1): the ray's entry and exit
// points on the minimum bounding sphere of voxel `cell`, relative to the voxel
// centre c = (ijk + 1/2) 2^-L, scaled to unit norm.
//
// The perpendicular offset q of the ray from c is tiny (at most the sphere
// radius, ~1e-3) next to |o - c| (~2.5), so it is formed in double-float
// arithmetic (Dekker 1971: exact TwoSum / TwoProduct with FMA): o - c exactly,
// t_f = -(d.(o-c)) / |d|^2 and q = (o - c) + t_f d to about 1e-12 absolute.
// The half chord and the normalisation are then plain float32.
// Every product and sum is written with an explicit rounding (fmaf, __fmul_rn,
// __fadd_rn), which the compiler never fuses or reassociates: each inlined
// copy computes the same bits (TwoProduct also needs its product rounded on
// its own, not fused into a following sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void sphere_param(const float o[3], const float d[3], uint32_t cell,
                                             int depth, float p1[3], float p2[3]) {
    const float h = ldexpf(1.0f, -depth);
    const float R = __fmul_rn(0.8660254037844386f, h);
    float oc_hi[3], oc_lo[3];
    {
        int ijk[3] = {(int)(cell & 1023u), (int)((cell >> 10) & 1023u), (int)((cell >> 20) & 1023u)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float c = __fmul_rn(__fadd_rn((float)ijk[a], 0.5f), h);  // exact
            two_sum(o[a], -c, oc_hi[a], oc_lo[a]);
        }
    }
    // b = d . (o - c) and dd = d . d in double-float
    float b_hi = 0.f, b_lo = 0.f, dd_hi = 0.f, dd_lo = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p, pe, s, se;
        two_prod(d[a], oc_hi[a], p, pe);
        two_sum(b_hi, p, s, se);
        b_hi = s;
        b_lo = __fadd_rn(b_lo, fmaf(d[a], oc_lo[a], __fadd_rn(se, pe)));
        two_prod(d[a], d[a], p, pe);
        two_sum(dd_hi, p, s, se);
        dd_hi = s;
        dd_lo = __fadd_rn(dd_lo, __fadd_rn(se, pe));
    }
    {
        float s, se;
        two_sum(b_hi, b_lo, s, se);
        b_hi = s;
        b_lo = se;
    }
    // 1/dd = 1 + e + O(e^2) with e = 1 - dd (|e| ~ 1e-7 for a float32 unit vector)
    const float e = __fsub_rn(__fsub_rn(1.0f, dd_hi), dd_lo);
    // t_f = -b (1 + e) as (tf_hi, tf_lo)
    const float tf_hi = -b_hi;
    const float tf_lo = fmaf(-b_hi, e, -b_lo);
    float q[3];
    float qq = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p, pe;
        two_prod(tf_hi, d[a], p, pe);
        q[a] = __fadd_rn(__fadd_rn(oc_hi[a], p), fmaf(tf_lo, d[a], __fadd_rn(oc_lo[a], pe)));
        qq = fmaf(q[a], q[a], qq);
    }
    const float half = sqrtf(__fmul_rn(fmaxf(fmaf(R, R, -qq), 0.0f), __fadd_rn(1.0f, e)));
    float n1 = 0.f, n2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p1[a] = fmaf(-half, d[a], q[a]);
        p2[a] = fmaf(half, d[a], q[a]);
        n1 = fmaf(p1[a], p1[a], n1);
        n2 = fmaf(p2[a], p2[a], n2);
    }
    const float i1 = rsqrtf(n1), i2 = rsqrtf(n2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p1[a] = __fmul_rn(p1[a], i1);
        p2[a] = __fmul_rn(p2[a], i2);
    }
}

// The same parameterisation from a point of the ray inside the voxel, x = o +
// t d with t in the voxel's segment (the sample's midpoint t). x is formed
// exactly as a double-float (TwoProduct, TwoSum), so delta = x - c is small
// (within a few voxel radii) and accurate to about 2^-24 of the radius; the
// perpendicular offset q = delta - (delta . d) d then needs no double-float
// (d is unit to float32 precision: the 1 - |d|^2 term is ~1e-7 of |delta|).
// Fewer, shorter dependent chains than sphere_param, same accuracy; any t on
// the segment gives the same q up to rounding.
__device__ __forceinline__ void sphere_param_at(const float o[3], const float d[3], float t, uint32_t cell,
                                                int depth, float p1[3], float p2[3]) {
    const float h = ldexpf(1.0f, -depth);
    const float R = __fmul_rn(0.8660254037844386f, h);
    float del[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float pr, pe, sx, se;
        two_prod(t, d[a], pr, pe);
        two_sum(o[a], pr, sx, se);
        const float c = __fmul_rn(__fadd_rn((float)((cell >> (10 * a)) & 1023u), 0.5f), h);  // exact
        del[a] = __fadd_rn(__fsub_rn(sx, c), __fadd_rn(se, pe));
    }
    const float b = fmaf(del[2], d[2], fmaf(del[1], d[1], __fmul_rn(del[0], d[0])));
    float q[3];
    float qq = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q[a] = fmaf(-b, d[a], del[a]);
        qq = fmaf(q[a], q[a], qq);
    }
    const float half = sqrtf(fmaxf(fmaf(R, R, -qq), 0.0f));
    float n1 = 0.f, n2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p1[a] = fmaf(-half, d[a], q[a]);
        p2[a] = fmaf(half, d[a], q[a]);
        n1 = fmaf(p1[a], p1[a], n1);
        n2 = fmaf(p2[a], p2[a], n2);
    }
    const float i1 = rsqrtf(n1), i2 = rsqrtf(n2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p1[a] = __fmul_rn(p1[a], i1);
        p2[a] = __fmul_rn(p2[a], i2);
    }
}

// The alternative reading of "voxel origin" (svlf_render_opts.rparam_mode =
// SVLF_RPARAM_AABB): r = [x~1 | x~2], the ray's entry and exit points of the
// voxel itself (its slab segment, entry clipped at t = 0) in voxel-local
// coordinates x~ = (x - c) / (h / 2), each component in [-1, 1]. Formed
// around the exactly formed point x_t = o + t d of the segment (t = its
// midpoint), like sphere_param_at: delta = x_t - c, then the segment's ends
// delta + u d with u found by the slab test in the voxel's own frame, so the
// result carries no rounding of the distance from the ray origin.
__device__ __forceinline__ void aabb_param_at(const float o[3], const float d[3], float t, uint32_t cell,
                                              int depth, float p1[3], float p2[3]) {
    const float h = ldexpf(1.0f, -depth);
    const float half = __fmul_rn(0.5f, h);
    float del[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float pr, pe, sx, se;
        two_prod(t, d[a], pr, pe);
        two_sum(o[a], pr, sx, se);
        const float c = __fmul_rn(__fadd_rn((float)((cell >> (10 * a)) & 1023u), 0.5f), h);  // exact
        del[a] = __fadd_rn(__fsub_rn(sx, c), __fadd_rn(se, pe));
    }
    float u_in = -t, u_out = INFINITY;  // the entry never precedes the ray origin
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.f) continue;  // parallel to this slab: it never bounds the segment
        const float lo = __fdiv_rn(__fsub_rn(-half, del[a]), d[a]);
        const float hi = __fdiv_rn(__fsub_rn(half, del[a]), d[a]);
        u_in = fmaxf(u_in, fminf(lo, hi));
        u_out = fminf(u_out, fmaxf(lo, hi));
    }
    const float inv = __fdiv_rn(1.0f, half);  // a power of two: exact
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p1[a] = __fmul_rn(fmaf(u_in, d[a], del[a]), inv);
        p2[a] = __fmul_rn(fmaf(u_out, d[a], del[a]), inv);
    }
}

// r = [p~1 | p~2] of a sample under the chosen reading (SVLF_RPARAM_*).
__device__ __forceinline__ void voxel_param_at(int rparam, const float o[3], const float d[3], float t,
                                               uint32_t cell, int depth, float p1[3], float p2[3]) {
    if (rparam == SVLF_RPARAM_AABB)
        aabb_param_at(o, d, t, cell, depth, p1, p2);
    else
        sphere_param_at(o, d, t, cell, depth, p1, p2);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// Four float32 adds to 16 aligned bytes of global memory as one reduction
// (no value returned, so the thread never waits for it).
__device__ __forceinline__ void red_add_f4(float4 *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

}  // namespace svlf
