// Per-ray sparse-octree traversal: the first K occupied leaves along each ray,
// in ascending t, with their segments [t_in, t_out] (Sec. 4.3 "Evaluating
// intersected voxels"; slab test of Sec. 4.2).
//
// Design (one ray per thread, stackless):
//  * The ray is walked region by region. At every position the octree
//    answers either an empty region containing the current finest cell, or
//    the cell's brick (the 4^3 leaves under a level L-2 node, held as a 64-bit
//    mask). A dense index over the level L-3 nodes (the parents of the
//    bricks) gives that answer in one load instead of a descent from the
//    root: the parent's node word, or an empty box around it (the largest
//    empty octree block holding it, grown face by face while it stays empty,
//    which takes about a third fewer steps than the octree blocks alone). The
//    brick of the current cell stays cached in registers, so consecutive
//    cells inside a brick cost no memory access.
//  * Plane crossings t = (k 2^-L - o) / d are evaluated without a division:
//    k 2^-L - o is split exactly into hi + lo (TwoSum) and multiplied by 1/d
//    held as a double-float (r_hi + r_lo, formed once per ray with an FMA
//    residual), so each crossing carries about half an ulp of error. The cell
//    after a crossing is the one whose planes' crossings bracket the current
//    t: floor of the position where that is provably exact (an error bound
//    per ray), else found by counting the planes whose crossing is <= t. A
//    voxel is therefore entered at the t its slab test gives as t_in and left
//    at its t_out, every visited voxel has t_out > t_in, and no voxel with a
//    positive segment is skipped.
//  * Hits go to the lane's K slots, in shared memory (interleaved by thread)
//    for K <= 16, else in a global scratch area (the network output buffer,
//    not yet in use), keeping registers free for occupancy; at the end each
//    warp reserves space for its rays' samples with one atomic and copies them
//    contiguously per ray from the slots.
//  * Many scenes can be traced in one launch (see SceneTable).
//  * Persistent warps fetch their own work items of 32 neighbouring rays
//    (one per lane) from a global counter, and claim the next one when
//    enough lanes are idle: all of them on large launches, so that a warp's
//    rays stay neighbours and walk through the same bricks together (32-ray
//    items run the render traversal about 11 % faster than 128-ray items
//    whose lanes refill from the rest of the item), half on small ones; no
//    warp waits for the rest of its block.
#include "svlf_internal.cuh"

namespace svlf {

__device__ unsigned int g_device_status = 0;

#ifdef SVLF_TRACE_STATS
// [0] walk steps, [1] parent-index loads, [2], [3] unused, [4] brick loads,
// [5] rays entering the cube, [6] steps inside a cached brick, [7] rays
__device__ unsigned long long g_trace_stats[8];
#define TRACE_STAT(i, v) atomicAdd(&g_trace_stats[i], (unsigned long long)(v))
#else
#define TRACE_STAT(i, v) ((void)0)
#endif

struct RayState {
    float o[3], d[3];
    float rhi[3], rlo[3];  // 1/d as a double-float
    float h;
    int n;  // 2^L
};

__device__ __forceinline__ float cross_t1(int k, float h, float o, float rhi, float rlo) {
    float xh, xl;
    two_sum((float)k * h, -o, xh, xl);  // k 2^-L exact; difference split exactly
    return fmaf(xh, rhi, fmaf(xh, rlo, xl * rhi));
}

__device__ __forceinline__ float cross_t(const RayState &R, int a, int k) {
    return cross_t1(k, R.h, R.o[a], R.rhi[a], R.rlo[a]);
}

// Cell index along axis a occupied just after time t, searched in [lo, hi],
// by counting the planes whose crossing is <= t. (Kept inline: a call would
// make the walk state spill around it.)
__device__ __forceinline__ int cell_after_exact(float h, float o, float d, float rhi, float rlo, float t, int k,
                                             int lo, int hi) {
    k = min(max(k, lo), hi);
    if (d > 0.f) {
        for (int it = 0; it < 64 && k > lo && cross_t1(k, h, o, rhi, rlo) > t; ++it) --k;
        for (int it = 0; it < 64 && k < hi && cross_t1(k + 1, h, o, rhi, rlo) <= t; ++it) ++k;
    } else {
        for (int it = 0; it < 64 && k < hi && cross_t1(k + 1, h, o, rhi, rlo) > t; ++it) ++k;
        for (int it = 0; it < 64 && k > lo && cross_t1(k, h, o, rhi, rlo) <= t; ++it) --k;
    }
    return k;
}

// The same, with a fast path: pos = (o + t d) n is rounded once (FMA; n is a
// power of two), so it is within 2^-24 (|o| + |t d|) n cells of the exact
// position at t, and a crossing from cross_t is within 2^-23 |t| of the exact
// one, i.e. 2^-23 |t d| n cells. `eps` (per ray, see walk_init) is at least
// 16x the sum for every t of the walk; when pos is farther than that from
// every cell boundary, the plane counts cannot change floor(pos).
__device__ __forceinline__ int cell_after(const RayState &R, int a, float t, int lo, int hi, float eps) {
    const float pos = fmaf(t, R.d[a], R.o[a]) * (float)R.n;
    const float fl = floorf(fminf(fmaxf(pos, -1.0f), (float)R.n));
    const int k = (int)fl;
    const float fr = pos - fl;
    if (k >= lo && k <= hi && fr > eps && fr < 1.0f - eps) return k;
    return cell_after_exact(R.h, R.o[a], R.d[a], R.rhi[a], R.rlo[a], t, k, lo, hi);
}

// Traversal state of one ray, kept in registers across the rounds of the
// warp loop below.
struct Walk {
    RayState R;
    int c[3];        // current finest cell
    float t;         // entry t of the current cell
    float eps;       // fast-path margin of cell_after, in cells (valid for t up to the cube exit)
    int nh;          // hits so far
    int steps;
    uint32_t cached;  // brick (level L-2) of the current cell
    uint64_t bmask;
    int bbase;
};

// Root clip (slab test against the unit cube) and the first cell. Returns
// false when the ray does not enter the cube with a positive segment.
__device__ __forceinline__ bool walk_init(const OctreeView &T, Walk &w) {
    if (T.empty) return false;
    RayState &R = w.R;
    const int n = R.n;
    float t0 = 0.f, t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] == 0.f) {
            if (R.o[a] < 0.f || R.o[a] > 1.f) return false;
            continue;
        }
        float ta = cross_t(R, a, 0), tb = cross_t(R, a, n);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (!(t1 - t0 > 0.f)) return false;
    // margin for every t <= t1: (|o_a| + t |d_a| + 2^-10) n 2^-19 over the axes
    const float om = fmaxf(fabsf(R.o[0]), fmaxf(fabsf(R.o[1]), fabsf(R.o[2])));
    const float dm = fmaxf(fabsf(R.d[0]), fmaxf(fabsf(R.d[1]), fabsf(R.d[2])));
    w.eps = (om + t1 * dm + 0x1p-10f) * (float)n * 0x1p-19f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        w.c[a] = R.d[a] == 0.f ? min(max((int)floorf(R.o[a] * (float)n), 0), n - 1)
                               : cell_after(R, a, t0, 0, n - 1, w.eps);
    w.t = t0;
    w.nh = 0;
    w.steps = 0;
    w.cached = 0xFFFFFFFFu;
    w.bmask = 0;
    w.bbase = 0;
    return true;
}

// Up to `budget` steps of the walk; hit j goes to slot[j * stride] (16 bytes:
// rank, packed cell, t_in, t_out). Returns true when the ray is finished (K
// hits, left the cube, or an error was latched).
__device__ bool walk_steps(const OctreeView &T, Walk &w, int K, int4 *__restrict__ slot, int stride, int budget,
                           int step_limit) {
    const RayState &R = w.R;
    const int n = R.n;
    const int max_steps = step_limit > 0 ? step_limit : 3 * n + 64;
    const int ps = T.pgrid_shift;
    // the step bound is checked once per call (it may overrun by one budget)
    if (w.steps > max_steps) {
        raise_status(SVLF_DEV_STEP_LIMIT);
        return true;
    }
    w.steps += budget;
    for (int it = 0; it < budget; ++it) {
        int *c = w.c;
        TRACE_STAT(0, 1);
        const uint32_t key = (uint32_t)(c[0] >> 2) | ((uint32_t)(c[1] >> 2) << 10) |
                             ((uint32_t)(c[2] >> 2) << 20);
        int sz_log = 0;
        bool leaf = false;
        int rank = -1;
        uint32_t box_lo = 0, box_hi = 0;  // nonzero box_hi: an empty box around the parent (level L-3 cells)
        if (key == w.cached) TRACE_STAT(6, 1);
        if (key != w.cached) {
            int node = 0;  // depth 2: the root is the only brick
            bool found = true;
            if (T.n_node_levels > 0) {
                TRACE_STAT(1, 1);
                // 0 <= c < 2^L here, so the index stays inside the (2^(L-3))^3 words
                const uint32_t pidx = (uint32_t)(c[0] >> 3) | ((uint32_t)(c[1] >> 3) << ps) |
                                      ((uint32_t)(c[2] >> 3) << (2 * ps));
                const uint2 pe = __ldg(T.pgrid + pidx);
                const uint32_t pw = pe.x;
                const uint32_t m = pw >> 24;
                const int oct = ((c[0] >> 2) & 1) | (((c[1] >> 2) & 1) << 1) | (((c[2] >> 2) & 1) << 2);
                if (!((m >> oct) & 1u)) {
                    sz_log = 2;  // empty brick (unless the whole parent is empty: its box below)
                    box_lo = pw;
                    box_hi = m ? 0u : pe.y;
                    found = false;
                } else {
                    node = (int)(pw & 0xFFFFFFu) + __popc(m & ((1u << oct) - 1u));
                }
            }
            if (found) {
                if (node >= T.n_bricks) {
                    raise_status(SVLF_DEV_BAD_INDEX);
                    return true;
                }
                TRACE_STAT(4, 1);
                const uint4 b = __ldg(T.bricks + node);
                w.bmask = (uint64_t)b.x | ((uint64_t)b.y << 32);
                w.bbase = (int)b.z;
                w.cached = key;
            } else {
                w.cached = 0xFFFFFFFFu;
            }
        }
        if (w.cached == key) {
            const int bit = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2) |
                            (((c[0] >> 1) & 1) << 3) | (((c[1] >> 1) & 1) << 4) |
                            (((c[2] >> 1) & 1) << 5);
            if (((w.bmask >> (bit & 56)) & 0xFFull) == 0) {
                sz_log = 1;
            } else if (!((w.bmask >> bit) & 1ull)) {
                sz_log = 0;
            } else {
                leaf = true;
                rank = w.bbase + __popcll(w.bmask & ((1ull << bit) - 1ull));
            }
        }
        // the empty (or leaf) region the ray is in: [blo, bhi) per axis, finest cells
        const int sz = 1 << sz_log;
        int blo[3], bhi[3];
        float ta[3];
        float tx = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (box_hi) {
                blo[a] = (int)((box_lo >> (8 * a)) & 0xFFu) << 3;
                bhi[a] = (int)((box_hi >> (8 * a)) & 0xFFu) << 3;
            } else {
                blo[a] = c[a] & ~(sz - 1);
                bhi[a] = blo[a] + sz;
            }
            ta[a] = R.d[a] > 0.f ? cross_t(R, a, bhi[a])
                  : R.d[a] < 0.f ? cross_t(R, a, blo[a]) : INFINITY;
            tx = fminf(tx, ta[a]);
        }
        if (leaf) {
            const uint32_t packed = (uint32_t)c[0] | ((uint32_t)c[1] << 10) | ((uint32_t)c[2] << 20);
            slot[w.nh * stride] = make_int4(rank, (int)packed, __float_as_int(w.t), __float_as_int(tx));
            if (++w.nh == K) return true;
        }
        // the cell after tx on every axis, without a branch per axis: exit axes
        // step into the neighbouring block, the others stay inside the block at
        // floor(pos) where that is provably exact (cell_after's fast path), else
        // by plane counting (rare: one branch for the warp)
        int slow = 0;
        const float fn = (float)n;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool up = R.d[a] > 0.f;
            // floor(pos) by one saturating conversion: a position outside the block
            // (even one far outside int range) gives k outside [lo, hi] and takes the
            // exact search, which clamps its start itself
            const float p = fmaf(tx, R.d[a], R.o[a]) * fn;
            const int k = __float2int_rd(p);
            const float fr = p - (float)k;
            const int lo = up ? c[a] : blo[a];
            const int hi = up ? bhi[a] - 1 : c[a];
            // fr in (eps, 1 - eps), as one comparison (its rounding is far inside eps's 16x margin)
            const bool ok = k >= lo && k <= hi && fabsf(fr - 0.5f) < 0.5f - w.eps;
            const bool ex = ta[a] <= tx;
            const bool stay = !ex && bhi[a] - blo[a] > 1 && R.d[a] != 0.f;
            slow |= (stay && !ok) ? (1 << a) : 0;
            c[a] = ex ? (up ? bhi[a] : blo[a] - 1) : stay ? k : c[a];
        }
        if (slow) {
            // searched over the whole block: the plane counts cannot move below the
            // (exact) cell held before the step, whose entry crossing is <= tx
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if ((slow >> a) & 1)
                    c[a] = cell_after_exact(R.h, R.o[a], R.d[a], R.rhi[a], R.rlo[a], tx, c[a], blo[a], bhi[a] - 1);
        }
        if (((unsigned)c[0] >= (unsigned)n) | ((unsigned)c[1] >= (unsigned)n) | ((unsigned)c[2] >= (unsigned)n))
            return true;
        w.t = tx;
    }
    return false;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Each warp claims work items of kTraceChunk rays from a global counter (in
// order, so neighbouring warps walk neighbouring pixels; a scene's item is a
// run of 32 rays, or a tile of 8 x 4 pixels when its rays are image rows). A lane whose ray is
// finished takes the next ray of the warp's current chunk; once that chunk is
// handed out, the warp claims another one when at least `refill` lanes are
// idle (32: only when all are), so lanes may hold rays of different chunks
// and scenes. Rays that miss the unit cube never enter the walk. Finished rays
// write their samples to their scene's region, with one atomic per warp,
// scene and round.
#ifndef SVLF_TRACE_MIN_BLOCKS
#define SVLF_TRACE_MIN_BLOCKS 4  // resident blocks of 256 per SM the register budget is sized for
#endif

// MULTI = false: a single-scene table (scene 0 is then addressed statically).
template <bool MULTI>
__global__ void __launch_bounds__(256, SVLF_TRACE_MIN_BLOCKS) trace_kernel(const __grid_constant__ SceneTable T,
                                                    Sample *__restrict__ samples,
                                                    int4 *__restrict__ slots,
                                                    int2 *__restrict__ ray_span,
                                                    unsigned int *__restrict__ counter,
                                                    int32_t *__restrict__ hits,
                                                    float *__restrict__ t_io, int budget, int smem_slots,
                                                    int refill, int step_limit) {
    // a lane's hit slots: in shared memory, interleaved [hit][thread] (conflict-free
    // warp stores), when they fit; else its ray's K slots in the global scratch
    extern __shared__ int4 s_slots[];
    const int lane = threadIdx.x & 31;
    const int K = T.K;
    const int ss = smem_slots ? (int)blockDim.x : 1;
    // warp-uniform: the chunk being handed out
    // ray k of the work item (k < chunk_n) is r_begin + (k / 8) * row + k % 8,
    // row = 8 for rays in their own order, the image width for 8 x 4 pixel tiles
    int64_t r_begin = 0;
    int chunk_n = 0, next = 0, csc = 0;
    bool exhausted = false;  // the launch has no chunk left
    // per lane: the ray it walks
    bool have = false;
    int64_t g = 0;
    int sc = 0;
    Walk w;
    for (;;) {
        // ---- refill idle lanes (warp-uniform loop); rays that miss finish here
        for (int round = 0; round < 64; ++round) {
            const unsigned idle = __ballot_sync(0xFFFFFFFFu, !have);
            if (!idle || exhausted) break;
            if (next >= chunk_n) {
                if (__popc(idle) < refill) break;  // keep walking the rays in hand
                long long chunk = 0;
                if (lane == 0) chunk = (long long)atomicAdd(counter + kCtrTraceChunks, 1u);
                chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
                if (chunk >= T.total_chunks) {
                    exhausted = true;
                    break;
                }
                csc = MULTI ? scene_of_chunk(T, chunk) : 0;
                const int64_t q = chunk - T.s[csc].chunk_begin;  // work item within the scene
                const int tw = T.s[csc].tile_w;
                if (tw) {  // tile (q mod W/8, q div W/8) of 8 x 4 pixels; the scene holds whole tiles
                    const int64_t tpb = tw >> 3;
                    const int64_t band = q / tpb;
                    r_begin = band * 4 * tw + (q - band * tpb) * 8;
                    chunk_n = kTraceChunk;
                } else {
                    r_begin = q * kTraceChunk;
                    chunk_n = (int)min((int64_t)kTraceChunk, T.s[csc].n_rays - r_begin);
                }
                next = 0;
            }
            if (!have) {
                const int my = next + __popc(idle & lanemask_lt());
                if (my < chunk_n) {
                    const SceneDev &S = T.s[csc];
                    const int row = S.tile_w ? S.tile_w : 8;
                    const int64_t rl = r_begin + (int64_t)(my >> 3) * row + (my & 7);
                    g = S.ray_begin + rl;
                    sc = csc;
                    const float2 *rp = reinterpret_cast<const float2 *>(S.rays + 6 * rl);
                    const float2 a = __ldg(rp), b = __ldg(rp + 1), cc = __ldg(rp + 2);
                    RayState &R = w.R;
                    R.o[0] = a.x; R.o[1] = a.y; R.o[2] = b.x;
                    R.d[0] = b.y; R.d[1] = cc.x; R.d[2] = cc.y;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float rh = 1.0f / R.d[q];  // inf for d = 0 (that axis is never crossed)
                        R.rhi[q] = rh;
                        R.rlo[q] = R.d[q] != 0.f ? fmaf(-R.d[q], rh, 1.0f) * rh : 0.f;
                    }
                    R.n = 1 << S.tree.depth;
                    R.h = ldexpf(1.0f, -S.tree.depth);
                    w.nh = 0;
                    have = walk_init(S.tree, w);
                    TRACE_STAT(7, 1);
                    if (have) {
                        TRACE_STAT(5, 1);
                    } else {  // a miss: zero samples
                        ray_span[g] = make_int2((int)(S.ray_begin * K), 0);
                        for (int j = 0; hits && j < K; ++j) hits[g * K + j] = -1;
                        for (int j = 0; t_io && j < K; ++j)
                            reinterpret_cast<float2 *>(t_io)[g * K + j] = make_float2(0.f, 0.f);
                    }
                }
            }
            next = min(next + __popc(idle), chunk_n);
        }
        if (exhausted && !__any_sync(0xFFFFFFFFu, have)) break;
        // ---- walk
        bool done = false;
        if (have) {
            int4 *slot = smem_slots ? s_slots + threadIdx.x : slots + g * K;
            if (walk_steps(T.s[MULTI ? sc : 0].tree, w, K, slot, ss, budget, step_limit)) {
                have = false;
                done = true;
            }
        }
        // ---- finished rays: reserve their samples (one atomic per scene present) and copy them
        unsigned pending = __ballot_sync(0xFFFFFFFFu, done);
        while (pending) {
            const int lsc = MULTI ? __shfl_sync(0xFFFFFFFFu, sc, __ffs(pending) - 1) : 0;
            const bool mine = done && (!MULTI || sc == lsc);
            pending &= ~__ballot_sync(0xFFFFFFFFu, mine);
            const int nh = mine ? w.nh : 0;
            int incl = nh;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                if (lane >= off) incl += v;
            }
            const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            unsigned int wbase = 0;
            if (lane == 31 && total > 0) wbase = atomicAdd(counter + kCtrScene + lsc, (unsigned int)total);
            wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
            if (mine) {
                const SceneDev &S = T.s[lsc];
                const int64_t cap = S.n_rays * (int64_t)K;  // the scene's slot region
                const int64_t first = (int64_t)wbase + (incl - nh);
                int keep = nh;
                if (first + nh > cap) {
                    raise_status(SVLF_DEV_SAMPLE_OVERFLOW);
                    keep = (int)max((int64_t)0, cap - first);
                }
                const int64_t base = S.ray_begin * K + first;  // global sample index
                ray_span[g] = make_int2((int)base, keep);
                const int4 *slot = smem_slots ? s_slots + threadIdx.x : slots + g * K;
                for (int j = 0; j < keep; ++j) {
                    const int4 h = slot[j * ss];
                    const float tm = 0.5f * (__int_as_float(h.z) + __int_as_float(h.w));
                    reinterpret_cast<int4 *>(samples)[base + j] = make_int4(h.x, (int)g, h.y, __float_as_int(tm));
                }
                if (hits || t_io) {
                    for (int j = 0; j < K; ++j) {
                        const int4 h = j < nh ? slot[j * ss] : make_int4(-1, 0, 0, 0);
                        if (hits) hits[g * K + j] = h.x;
                        if (t_io)
                            reinterpret_cast<float2 *>(t_io)[g * K + j] =
                                j < nh ? make_float2(__int_as_float(h.z), __int_as_float(h.w))
                                       : make_float2(0.f, 0.f);
                    }
                }
            }
        }
    }
}

int launch_trace(const SceneTable &T, const Workspace &ws, int32_t *hits, float *t_io,
                 cudaStream_t s) {
    if (T.K < 1 || T.K > kMaxK) return SVLF_ERR_UNSUPPORTED;
    const int threads = tuning().trace_block;
    // hit slots in shared memory up to K = 16 (32-64 KB per block of 256)
    const int smem_slots = T.K <= 16 ? 1 : 0;
    const size_t smem = smem_slots ? sizeof(int4) * (size_t)threads * T.K : 0;
    const auto kernel = T.n > 1 ? trace_kernel<true> : trace_kernel<false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (T.total_chunks + threads / 32 - 1) / (threads / 32);
    const int64_t cap = (int64_t)num_sms() * per_sm;  // persistent: one wave of resident blocks
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // the per-ray hit slots live in the network-output buffer (total_rays*K x 16 B),
    // which the network kernels only write after this kernel is done
    // lanes wait for the whole warp before a new chunk on large launches (the
    // warp's rays stay neighbours), and refill at half a warp on small ones
    // (fewer than two rounds of work items for the resident warps)
    const int64_t large = (int64_t)2 * num_sms() * 32;
    const int refill = tuning().trace_refill ? tuning().trace_refill : T.total_chunks >= large ? 32 : 16;
    prof_begin("trace", s);
    kernel<<<(unsigned)blocks, threads, smem, s>>>(T, ws.samples, reinterpret_cast<int4 *>(ws.outputs),
                                                   ws.ray_span, ws.counter, hits, t_io, tuning().trace_budget,
                                                   smem_slots, refill, g_step_limit);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

}  // namespace svlf

#ifdef SVLF_TRACE_STATS
// statistics build only: copy (and optionally reset) the traversal counters
extern "C" int svlf_trace_stats(unsigned long long *out, int reset) {
    if (cudaDeviceSynchronize() != cudaSuccess) return SVLF_ERR_CUDA;
    if (cudaMemcpyFromSymbol(out, svlf::g_trace_stats, sizeof(unsigned long long) * 8) != cudaSuccess)
        return SVLF_ERR_CUDA;
    if (reset) {
        unsigned long long z[8] = {0};
        if (cudaMemcpyToSymbol(svlf::g_trace_stats, z, sizeof(z)) != cudaSuccess) return SVLF_ERR_CUDA;
    }
    return SVLF_OK;
}
#endif
