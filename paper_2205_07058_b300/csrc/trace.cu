// Per-ray sparse-octree traversal: the first K occupied leaves along each ray,
// in ascending t, with their segments [t_in, t_out] (Sec. 4.3 "Evaluating
// intersected voxels"; slab test of Sec. 4.2).
//
// Design (one ray per thread, stackless):
//  * The ray is walked voxel-block by voxel-block. At every position the
//    octree is descended from the root to find either the largest empty
//    block containing the current finest cell, or the cell's brick (the 4^3
//    leaves under a level L-2 node, held as a 64-bit mask). The brick of the
//    current cell stays cached in registers, so consecutive cells inside it
//    cost no memory access.
//  * The node words of the top levels (up to kSmemNodeWords) are staged in
//    shared memory; deeper levels and bricks come through the read-only path.
//  * Plane crossings t = (k 2^-L - o) / d are evaluated without a division:
//    k 2^-L - o is split exactly into hi + lo (TwoSum) and multiplied by 1/d
//    held as a double-float (r_hi + r_lo, formed once per ray with an FMA
//    residual), so each crossing carries about half an ulp of error. The cell
//    after a crossing is found by counting the planes whose crossing is <= the
//    current t. A voxel is therefore entered at the t its slab test gives as
//    t_in and left at its t_out, every visited voxel has t_out > t_in, and no
//    voxel with a positive segment is skipped.
//  * Hits go straight to the ray's K slots in a scratch area (the network
//    output buffer, not yet in use), keeping registers free for occupancy; at
//    the end each warp reserves space for its rays' samples with one atomic
//    and copies them contiguously per ray from the (cache-hot) slots.
//  * Many scenes can be traced in one launch (see SceneTable).
#include "svlf_internal.cuh"

namespace svlf {

__device__ unsigned int g_device_status = 0;

struct RayState {
    float o[3], d[3];
    float rhi[3], rlo[3];  // 1/d as a double-float
    float h;
    int n;  // 2^L
};

__device__ __forceinline__ float cross_t(const RayState &R, int a, int k) {
    float xh, xl;
    two_sum((float)k * R.h, -R.o[a], xh, xl);  // k 2^-L exact; difference split exactly
    return fmaf(xh, R.rhi[a], fmaf(xh, R.rlo[a], xl * R.rhi[a]));
}

// Cell index along axis a occupied just after time t, searched in [lo, hi].
__device__ __forceinline__ int cell_after(const RayState &R, int a, float t, int lo, int hi) {
    float pos = (R.o[a] + t * R.d[a]) * (float)R.n;
    int k = (int)floorf(fminf(fmaxf(pos, -1.0f), (float)R.n));
    k = min(max(k, lo), hi);
    if (R.d[a] > 0.f) {
        for (int it = 0; it < 64 && k > lo && cross_t(R, a, k) > t; ++it) --k;
        for (int it = 0; it < 64 && k < hi && cross_t(R, a, k + 1) <= t; ++it) ++k;
    } else {
        for (int it = 0; it < 64 && k < hi && cross_t(R, a, k + 1) > t; ++it) ++k;
        for (int it = 0; it < 64 && k > lo && cross_t(R, a, k) <= t; ++it) --k;
    }
    return k;
}

// Hits are written to slot[0 .. K-1] (16 bytes each: rank, packed cell,
// t_in, t_out); returns their number.
__device__ int traverse(const OctreeView &T, const uint32_t *s_nodes, int n_smem, RayState &R,
                        int K, int4 *__restrict__ slot) {
    if (T.empty) return 0;
    const int L = T.depth;
    const int n = R.n;
    float t0 = 0.f, t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] == 0.f) {
            if (R.o[a] < 0.f || R.o[a] > 1.f) return 0;
            continue;
        }
        float ta = cross_t(R, a, 0), tb = cross_t(R, a, n);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (!(t1 - t0 > 0.f)) return 0;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] == 0.f) {
            c[a] = min(max((int)floorf(R.o[a] * (float)n), 0), n - 1);
        } else {
            c[a] = cell_after(R, a, t0, 0, n - 1);
        }
    }
    float t = t0;
    int nh = 0;
    uint32_t cached = 0xFFFFFFFFu;
    uint64_t bmask = 0;
    int bbase = 0;
    const int max_steps = 3 * n + 64;
    for (int step = 0;; ++step) {
        if (step >= max_steps) {
            raise_status(SVLF_DEV_STEP_LIMIT);
            break;
        }
        const uint32_t key = (uint32_t)(c[0] >> 2) | ((uint32_t)(c[1] >> 2) << 10) |
                             ((uint32_t)(c[2] >> 2) << 20);
        int sz_log = 0;
        bool leaf = false;
        int rank = -1;
        if (key != cached) {
            int node = 0;
            bool found = true;
            for (int l = 0; l < T.n_node_levels; ++l) {
                const int s = L - 1 - l;
                const int oct = ((c[0] >> s) & 1) | (((c[1] >> s) & 1) << 1) | (((c[2] >> s) & 1) << 2);
                uint32_t w;
                if (node < n_smem) {
                    w = s_nodes[node];
                } else if (node < T.n_nodes) {
                    w = __ldg(T.nodes + node);
                } else {
                    raise_status(SVLF_DEV_BAD_INDEX);
                    return nh;
                }
                const uint32_t m = w >> 24;
                if (!((m >> oct) & 1u)) {
                    sz_log = s;
                    found = false;
                    break;
                }
                node = (int)(w & 0xFFFFFFu) + __popc(m & ((1u << oct) - 1u));
            }
            if (found) {
                if (node >= T.n_bricks) {
                    raise_status(SVLF_DEV_BAD_INDEX);
                    return nh;
                }
                const uint4 b = __ldg(T.bricks + node);
                bmask = (uint64_t)b.x | ((uint64_t)b.y << 32);
                bbase = (int)b.z;
                cached = key;
            } else {
                cached = 0xFFFFFFFFu;
            }
        }
        if (cached == key) {
            const int bit = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2) |
                            (((c[0] >> 1) & 1) << 3) | (((c[1] >> 1) & 1) << 4) |
                            (((c[2] >> 1) & 1) << 5);
            if (((bmask >> (bit & 56)) & 0xFFull) == 0) {
                sz_log = 1;
            } else if (!((bmask >> bit) & 1ull)) {
                sz_log = 0;
            } else {
                leaf = true;
                rank = bbase + __popcll(bmask & ((1ull << bit) - 1ull));
            }
        }
        const int sz = 1 << sz_log;
        int B[3];
        float ta[3];
        float tx = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            B[a] = c[a] & ~(sz - 1);
            ta[a] = R.d[a] > 0.f ? cross_t(R, a, B[a] + sz)
                  : R.d[a] < 0.f ? cross_t(R, a, B[a]) : INFINITY;
            tx = fminf(tx, ta[a]);
        }
        if (leaf) {
            const uint32_t packed = (uint32_t)c[0] | ((uint32_t)c[1] << 10) | ((uint32_t)c[2] << 20);
            slot[nh] = make_int4(rank, (int)packed, __float_as_int(t), __float_as_int(tx));
            if (++nh == K) break;
        }
        bool out = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (R.d[a] == 0.f) continue;
            if (ta[a] <= tx) {
                c[a] = R.d[a] > 0.f ? B[a] + sz : B[a] - 1;
            } else if (sz > 1) {
                const int lo = R.d[a] > 0.f ? c[a] : B[a];
                const int hi = R.d[a] > 0.f ? B[a] + sz - 1 : c[a];
                c[a] = cell_after(R, a, tx, lo, hi);
            }
            out |= (c[a] < 0) | (c[a] >= n);
        }
        if (out) break;
        t = tx;
    }
    return nh;
}

// Work items are chunks of kTraceChunk rays of one scene, claimed in order
// from a global counter (dynamic balancing; a block's consecutive chunks are
// usually of the same scene, so its staged top levels stay valid).
__global__ void __launch_bounds__(kTraceChunk) trace_kernel(const __grid_constant__ SceneTable T,
                                                            Sample *__restrict__ samples,
                                                            int4 *__restrict__ slots,
                                                            int2 *__restrict__ ray_span,
                                                            unsigned int *__restrict__ counter,
                                                            int32_t *__restrict__ hits,
                                                            float *__restrict__ t_io) {
    extern __shared__ uint32_t s_nodes[];
    __shared__ long long s_chunk;
    const int lane = threadIdx.x & 31;
    const int K = T.K;
    int staged = -1;
    int n_smem = 0;
    for (;;) {
        if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(counter + kCtrTraceChunks, 1u);
        __syncthreads();
        const int64_t chunk = s_chunk;
        if (chunk >= T.total_chunks) break;
        const int sc = scene_of_chunk(T, chunk);
        const SceneDev &S = T.s[sc];
        const OctreeView &tree = S.tree;
        if (sc != staged) {  // stage this scene's top octree levels
            n_smem = min(tree.n_nodes, kSmemNodeWords);
            for (int i = threadIdx.x; i < n_smem; i += blockDim.x) s_nodes[i] = tree.nodes[i];
            staged = sc;
        }
        __syncthreads();
        const int64_t r_local = (chunk - S.chunk_begin) * kTraceChunk + threadIdx.x;
        const bool valid = r_local < S.n_rays;
        const int64_t g = S.ray_begin + r_local;  // global ray index
        int nh = 0;
        int4 *slot = slots + g * K;
        if (valid) {
            RayState R;
            const float2 *rp = reinterpret_cast<const float2 *>(S.rays + 6 * r_local);
            const float2 a = __ldg(rp), b = __ldg(rp + 1), cc = __ldg(rp + 2);
            R.o[0] = a.x; R.o[1] = a.y; R.o[2] = b.x;
            R.d[0] = b.y; R.d[1] = cc.x; R.d[2] = cc.y;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float rh = 1.0f / R.d[q];  // inf for d = 0 (that axis is never crossed)
                R.rhi[q] = rh;
                R.rlo[q] = R.d[q] != 0.f ? fmaf(-R.d[q], rh, 1.0f) * rh : 0.f;
            }
            R.n = 1 << tree.depth;
            R.h = ldexpf(1.0f, -tree.depth);
            nh = traverse(tree, s_nodes, n_smem, R, K, slot);
        }
        // warp-aggregated reservation of nh samples per lane in the scene's region
        int incl = nh;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned int wbase = 0;
        if (lane == 31 && total > 0) wbase = atomicAdd(counter + kCtrScene + sc, (unsigned int)total);
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
        const int64_t cap = S.n_rays * (int64_t)K;  // the scene's slot region
        const int64_t first = (int64_t)wbase + (incl - nh);
        if (valid) {
            int keep = nh;
            if (first + nh > cap) {
                raise_status(SVLF_DEV_SAMPLE_OVERFLOW);
                keep = (int)max((int64_t)0, cap - first);
            }
            const int64_t base = S.ray_begin * K + first;  // global sample index
            ray_span[g] = make_int2((int)base, keep);
            for (int j = 0; j < keep; ++j) {
                const int4 h = slot[j];
                const float tm = 0.5f * (__int_as_float(h.z) + __int_as_float(h.w));
                reinterpret_cast<int4 *>(samples)[base + j] = make_int4(h.x, (int)g, h.y, __float_as_int(tm));
            }
            if (hits || t_io) {
                for (int j = 0; j < K; ++j) {
                    const int4 h = j < nh ? slot[j] : make_int4(-1, 0, 0, 0);
                    if (hits) hits[g * K + j] = h.x;
                    if (t_io)
                        reinterpret_cast<float2 *>(t_io)[g * K + j] =
                            j < nh ? make_float2(__int_as_float(h.z), __int_as_float(h.w))
                                   : make_float2(0.f, 0.f);
                }
            }
        }
        __syncthreads();  // s_chunk / s_nodes are rewritten next iteration
    }
}

int launch_trace(const SceneTable &T, const Workspace &ws, int32_t *hits, float *t_io,
                 cudaStream_t s) {
    if (T.K < 1 || T.K > kMaxK) return SVLF_ERR_UNSUPPORTED;
    int max_nodes = 0;
    for (int i = 0; i < T.n; ++i) max_nodes = max(max_nodes, T.s[i].tree.n_nodes);
    const size_t smem = sizeof(uint32_t) * (size_t)min(max_nodes, kSmemNodeWords);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trace_kernel, kTraceChunk, smem) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = T.total_chunks;
    const int64_t cap = (int64_t)num_sms() * per_sm;  // persistent: one wave of resident blocks
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // the per-ray hit slots live in the network-output buffer (total_rays*K x 16 B),
    // which the network kernels only write after this kernel is done
    prof_begin("trace", s);
    trace_kernel<<<(unsigned)blocks, kTraceChunk, smem, s>>>(T, ws.samples,
                                                             reinterpret_cast<int4 *>(ws.outputs),
                                                             ws.ray_span, ws.counter, hits, t_io);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

}  // namespace svlf
