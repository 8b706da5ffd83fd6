// Sparse voxel octree construction (Sec. 4.1 "Scene volume": the octree keeps
// only the voxels that contain a surface) and the C-ABI calls that manage it.
//
// The build runs once per scene on the host: Morton-encode the leaves, sort,
// de-duplicate, then derive the 4^3-leaf bricks (level L-2) and every node
// level above them bottom-up, and a dense index over the parents of the
// bricks. The resulting arrays are uploaded once; the traversal kernel
// (trace.cu) reads them.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "svlf_internal.cuh"

namespace svlf {

static uint64_t spread3(uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

static uint64_t morton3(uint32_t i, uint32_t j, uint32_t k) {
    return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2);
}

static void unmorton3(uint64_t c, uint32_t &i, uint32_t &j, uint32_t &k) {
    i = j = k = 0;
    for (int b = 0; b < 21; ++b) {
        i |= (uint32_t)((c >> (3 * b)) & 1ull) << b;
        j |= (uint32_t)((c >> (3 * b + 1)) & 1ull) << b;
        k |= (uint32_t)((c >> (3 * b + 2)) & 1ull) << b;
    }
}

// Occupied cells in the box [l, h) of a G^3 grid, from its summed-volume
// table S ((G+1)^3 entries, x fastest): S(x, y, z) counts the occupied cells
// whose coordinates are all below (x, y, z).
__host__ __device__ inline int64_t svt_at(const int32_t *S, int64_t W, int x, int y, int z) {
    return S[((int64_t)z * W + y) * W + x];
}

__host__ __device__ inline int64_t svt_count(const int32_t *S, int G, const int l[3], const int h[3]) {
    const int64_t W = G + 1;
    return svt_at(S, W, h[0], h[1], h[2]) - svt_at(S, W, l[0], h[1], h[2]) - svt_at(S, W, h[0], l[1], h[2]) -
           svt_at(S, W, h[0], h[1], l[2]) + svt_at(S, W, l[0], l[1], h[2]) + svt_at(S, W, l[0], h[1], l[2]) +
           svt_at(S, W, h[0], l[1], l[2]) - svt_at(S, W, l[0], l[1], l[2]);
}

// Grows the empty box [lo, hi) of a G^3 grid face by face (axes x, y, z in
// turn, low face then high face) while the slab it would add is empty, until
// no face can grow by one layer. Each face tries a slab of `step` layers:
// on success the face moves and its step doubles, on failure the step halves,
// and a face that cannot take one layer is finished for good (growing the
// other faces only enlarges its slab). So the faces grow at similar rates and
// a long empty run costs a logarithmic number of tests, not one per layer.
// Deterministic, so the host and the GPU builds agree. A ray inside the box
// can jump to where it leaves the box: it meets no occupied cell on the way.
__host__ __device__ inline void grow_empty_box(const int32_t *S, int G, int lo[3], int hi[3]) {
    int step[6] = {1, 1, 1, 1, 1, 1};
    for (int round = 0; round <= 6 * G; ++round) {
        bool active = false;
        for (int f = 0; f < 6; ++f) {
            if (step[f] == 0) continue;  // finished
            const int a = f >> 1, side = f & 1;
            const int room = side == 0 ? lo[a] : G - hi[a];
            if (room == 0) {
                step[f] = 0;
                continue;
            }
            const int s = step[f] < room ? step[f] : room;
            int l[3] = {lo[0], lo[1], lo[2]}, h[3] = {hi[0], hi[1], hi[2]};
            if (side == 0) {
                l[a] = lo[a] - s;
                h[a] = lo[a];
            } else {
                l[a] = hi[a];
                h[a] = hi[a] + s;
            }
            if (svt_count(S, G, l, h) == 0) {
                if (side == 0) lo[a] -= s; else hi[a] += s;
                step[f] = 2 * s;
            } else {
                step[f] = s > 1 ? s / 2 : 0;
            }
            active |= step[f] != 0;
        }
        if (!active) break;
    }
}

__host__ __device__ inline uint32_t pack_corner(const int v[3]) {
    return (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16);
}

}  // namespace svlf

using namespace svlf;

struct svlf_octree_s {
    OctreeHost h;
};

extern "C" int svlf_build_octree_host(const int32_t *leaf_ijk, int64_t n, int depth, void *stream,
                                      svlf_octree *out, int64_t *n_leaves_out) {
    if (!out || n < 0 || (n > 0 && !leaf_ijk)) return SVLF_ERR_ARG;
    if (depth < 2 || depth > kMaxDepth) return SVLF_ERR_UNSUPPORTED;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> ijk((size_t)n * 3);
    if (n > 0) {
        if (cudaMemcpyAsync(ijk.data(), leaf_ijk, sizeof(int32_t) * 3 * (size_t)n,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SVLF_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SVLF_ERR_CUDA;
    }
    const int64_t side = (int64_t)1 << depth;
    std::vector<uint64_t> codes((size_t)n);
    for (int64_t q = 0; q < n; ++q) {
        for (int a = 0; a < 3; ++a)
            if (ijk[3 * q + a] < 0 || ijk[3 * q + a] >= side) return SVLF_ERR_ARG;
        codes[q] = morton3(ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2]);
    }
    std::sort(codes.begin(), codes.end());
    codes.erase(std::unique(codes.begin(), codes.end()), codes.end());
    const int64_t n_leaves = (int64_t)codes.size();
    if (n_leaves >= (int64_t)1 << 31) return SVLF_ERR_UNSUPPORTED;

    // bricks: occupied level L-2 cells, 64 leaves each
    std::vector<uint64_t> brick_code;
    std::vector<uint4> bricks;
    for (int64_t q = 0; q < n_leaves; ++q) {
        uint64_t bc = codes[q] >> 6;
        if (brick_code.empty() || brick_code.back() != bc) {
            brick_code.push_back(bc);
            bricks.push_back(make_uint4(0u, 0u, (uint32_t)q, 0u));
        }
        uint64_t bit = codes[q] & 63ull;
        uint4 &b = bricks.back();
        if (bit < 32) b.x |= 1u << bit; else b.y |= 1u << (bit - 32);
    }
    if (bricks.size() >= (1u << 24)) return SVLF_ERR_UNSUPPORTED;

    // node levels L-3 .. 0, built bottom-up; level l holds (code, word)
    const int n_levels = depth - 2;
    std::vector<std::vector<uint64_t>> lvl_code(n_levels);
    std::vector<std::vector<uint32_t>> lvl_word(n_levels);
    {
        const std::vector<uint64_t> *child_codes = &brick_code;
        for (int l = n_levels - 1; l >= 0; --l) {
            auto &cc = lvl_code[l];
            auto &ww = lvl_word[l];
            for (size_t q = 0; q < child_codes->size(); ++q) {
                uint64_t pc = (*child_codes)[q] >> 3;
                if (cc.empty() || cc.back() != pc) {
                    cc.push_back(pc);
                    ww.push_back((uint32_t)q);  // first child (relative to the child level)
                }
                ww.back() |= 1u << (24 + ((*child_codes)[q] & 7ull));
            }
            child_codes = &cc;
        }
    }
    // concatenate levels and make child indices absolute
    std::vector<uint32_t> nodes;
    std::vector<size_t> lvl_off(n_levels + 1, 0);
    for (int l = 0; l < n_levels; ++l) lvl_off[l + 1] = lvl_off[l] + lvl_word[l].size();
    if (lvl_off[n_levels] >= (1u << 24)) return SVLF_ERR_UNSUPPORTED;
    nodes.reserve(lvl_off[n_levels]);
    for (int l = 0; l < n_levels; ++l) {
        const uint32_t child_base = (l + 1 < n_levels) ? (uint32_t)lvl_off[l + 1] : 0u;
        for (uint32_t w : lvl_word[l]) {
            uint32_t first = (w & 0xFFFFFFu) + child_base;
            nodes.push_back((w & 0xFF000000u) | first);
        }
    }

    // Dense index over the level L-3 cells (the parents of the bricks, 8^3
    // finest cells each), x fastest: the node word where that node exists,
    // else (mask byte 0) log2 of the edge, in finest cells, of the largest
    // empty octree block that contains the cell; then each empty block is
    // grown into a larger empty box (OctreeView::pgrid). One load then answers
    // what a descent from the root would: the cell's brick or an empty region
    // around it.
    std::vector<uint32_t> pgrid;
    const int pshift = n_levels > 0 ? depth - 3 : 0;
    if (n_levels > 0 && n_leaves > 0) {
        const int64_t P = (int64_t)1 << pshift;
        pgrid.assign((size_t)(P * P * P), (uint32_t)depth);
        for (int l = 0; l < n_levels; ++l) {
            for (size_t q = 0; q < lvl_code[l].size(); ++q) {
                uint32_t x, y, z;
                unmorton3(lvl_code[l][q], x, y, z);
                const uint32_t w = nodes[lvl_off[l] + q];
                if (l == n_levels - 1) {
                    pgrid[(size_t)(((int64_t)z * P + y) * P + x)] = w;
                    continue;
                }
                const int64_t span = P >> (l + 1);  // index cells per axis under one child
                for (int o = 0; o < 8; ++o) {
                    if ((w >> (24 + o)) & 1u) continue;
                    const int64_t x0 = (2 * (int64_t)x + (o & 1)) * span;
                    const int64_t y0 = (2 * (int64_t)y + ((o >> 1) & 1)) * span;
                    const int64_t z0 = (2 * (int64_t)z + ((o >> 2) & 1)) * span;
                    for (int64_t k = z0; k < z0 + span; ++k)
                        for (int64_t j = y0; j < y0 + span; ++j)
                            std::fill_n(pgrid.begin() + (size_t)((k * P + j) * P + x0), (size_t)span,
                                        (uint32_t)(depth - l - 1));
                }
            }
        }
    }

    std::vector<uint2> pgrid2(pgrid.size());
    if (!pgrid.empty()) {
        const int G = 1 << pshift;
        const int64_t W = G + 1;
        std::vector<int32_t> S((size_t)(W * W * W), 0);
        for (int z = 0; z < G; ++z)
            for (int y = 0; y < G; ++y)
                for (int x = 0; x < G; ++x) {
                    const int64_t i = ((int64_t)z * G + y) * G + x;
                    const int32_t o = (pgrid[(size_t)i] >> 24) ? 1 : 0;
                    S[(size_t)(((z + 1) * W + y + 1) * W + x + 1)] =
                        o + S[(size_t)(((z + 1) * W + y + 1) * W + x)] + S[(size_t)(((z + 1) * W + y) * W + x + 1)] +
                        S[(size_t)((z * W + y + 1) * W + x + 1)] - S[(size_t)(((z + 1) * W + y) * W + x)] -
                        S[(size_t)((z * W + y + 1) * W + x)] - S[(size_t)((z * W + y) * W + x + 1)] +
                        S[(size_t)((z * W + y) * W + x)];
                }
        for (int z = 0; z < G; ++z)
            for (int y = 0; y < G; ++y)
                for (int x = 0; x < G; ++x) {
                    const size_t i = (size_t)(((int64_t)z * G + y) * G + x);
                    const uint32_t w = pgrid[i];
                    if (w >> 24) {
                        pgrid2[i] = make_uint2(w, 0u);
                        continue;
                    }
                    const int e = 1 << ((int)(w & 31u) - 3);  // block edge in level L-3 cells
                    int lo[3] = {x & ~(e - 1), y & ~(e - 1), z & ~(e - 1)};
                    const size_t corner = (size_t)(((int64_t)lo[2] * G + lo[1]) * G + lo[0]);
                    if (corner != i) {  // the block's corner comes first in x-fastest order
                        pgrid2[i] = pgrid2[corner];
                        continue;
                    }
                    int hi[3] = {lo[0] + e, lo[1] + e, lo[2] + e};
                    grow_empty_box(S.data(), G, lo, hi);
                    pgrid2[i] = make_uint2(pack_corner(lo), pack_corner(hi));
                }
    }

    svlf_octree_s *t = new (std::nothrow) svlf_octree_s;
    if (!t) return SVLF_ERR_CUDA;
    std::memset(t, 0, sizeof(*t));
    OctreeHost &H = t->h;
    H.view.depth = depth;
    H.view.n_node_levels = n_levels;
    H.view.n_leaves = n_leaves;
    H.view.n_nodes = (int)nodes.size();
    H.view.n_bricks = (int)bricks.size();
    H.view.root_is_brick = (n_levels == 0);
    H.view.empty = (n_leaves == 0);
    bool ok = true;
    std::vector<int32_t> rank_ijk((size_t)n_leaves * 3);
    for (int64_t q = 0; q < n_leaves; ++q) {
        uint32_t i, j, k;
        unmorton3(codes[q], i, j, k);
        rank_ijk[3 * q] = (int32_t)i;
        rank_ijk[3 * q + 1] = (int32_t)j;
        rank_ijk[3 * q + 2] = (int32_t)k;
    }
    size_t nb_ijk = sizeof(int32_t) * rank_ijk.size();
    size_t nb_nodes = sizeof(uint32_t) * (nodes.size() + 1);
    size_t nb_bricks = sizeof(uint4) * (bricks.size() + 1);
    size_t nb_pgrid = sizeof(uint2) * (pgrid2.size() + 1);
    ok = ok && cudaMalloc(&H.leaf_ijk_dev, nb_ijk > 0 ? nb_ijk : 16) == cudaSuccess;
    ok = ok && cudaMalloc(&H.pgrid_dev, nb_pgrid) == cudaSuccess;
    ok = ok && cudaMalloc(&H.nodes_dev, nb_nodes) == cudaSuccess;
    ok = ok && cudaMalloc(&H.bricks_dev, nb_bricks) == cudaSuccess;
    if (ok && nb_ijk)
        ok = cudaMemcpyAsync(H.leaf_ijk_dev, rank_ijk.data(), nb_ijk, cudaMemcpyHostToDevice, s) ==
             cudaSuccess;
    if (ok && !nodes.empty())
        ok = cudaMemcpyAsync(H.nodes_dev, nodes.data(), sizeof(uint32_t) * nodes.size(),
                             cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (ok && !bricks.empty())
        ok = cudaMemcpyAsync(H.bricks_dev, bricks.data(), sizeof(uint4) * bricks.size(),
                             cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (ok && !pgrid2.empty())
        ok = cudaMemcpyAsync(H.pgrid_dev, pgrid2.data(), sizeof(uint2) * pgrid2.size(),
                             cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaFree(H.leaf_ijk_dev);
        cudaFree(H.pgrid_dev);
        cudaFree(H.nodes_dev);
        cudaFree(H.bricks_dev);
        delete t;
        return SVLF_ERR_CUDA;
    }
    H.view.nodes = H.nodes_dev;
    H.view.bricks = H.bricks_dev;
    H.view.pgrid = H.pgrid_dev;
    H.view.pgrid_shift = pshift;
    *out = t;
    if (n_leaves_out) *n_leaves_out = n_leaves;
    return SVLF_OK;
}

extern "C" int svlf_octree_leaf_ijk(svlf_octree tree, int32_t *out_ijk, void *stream) {
    if (!tree || !out_ijk) return SVLF_ERR_ARG;
    size_t nb = sizeof(int32_t) * 3 * (size_t)tree->h.view.n_leaves;
    if (nb == 0) return SVLF_OK;
    return cudaMemcpyAsync(out_ijk, tree->h.leaf_ijk_dev, nb, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream) == cudaSuccess
               ? SVLF_OK
               : SVLF_ERR_CUDA;
}

extern "C" int svlf_octree_parent_index(svlf_octree tree, uint32_t *out, int64_t *n_entries, void *stream) {
    if (!tree || !n_entries) return SVLF_ERR_ARG;
    const OctreeView &v = tree->h.view;
    const int64_t G = v.n_node_levels > 0 && !v.empty ? (int64_t)1 << v.pgrid_shift : 0;
    *n_entries = G * G * G;
    if (!out || *n_entries == 0) return SVLF_OK;
    return cudaMemcpyAsync(out, tree->h.pgrid_dev, sizeof(uint2) * (size_t)*n_entries, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream) == cudaSuccess
               ? SVLF_OK
               : SVLF_ERR_CUDA;
}

extern "C" int svlf_octree_info(svlf_octree tree, int *depth, int64_t *n_leaves,
                                int64_t *n_nodes, int64_t *n_bricks) {
    if (!tree) return SVLF_ERR_ARG;
    if (depth) *depth = tree->h.view.depth;
    if (n_leaves) *n_leaves = tree->h.view.n_leaves;
    if (n_nodes) *n_nodes = tree->h.view.n_nodes;
    if (n_bricks) *n_bricks = tree->h.view.n_bricks;
    return SVLF_OK;
}

extern "C" int svlf_free_octree(svlf_octree tree) {
    if (!tree) return SVLF_ERR_ARG;
    cudaFree(tree->h.leaf_ijk_dev);
    cudaFree(tree->h.nodes_dev);
    cudaFree(tree->h.bricks_dev);
    cudaFree(tree->h.pgrid_dev);
    cudaFree(tree->h.vtx_dev);
    delete tree;
    return SVLF_OK;
}

// Vertex table of the two-decoder form (Sec. 4.1: one feature vector per
// octree vertex, shared by the voxels meeting there). Built on the host once
// per octree: every leaf corner as a lattice point (depth + 1 bits per axis),
// Morton-encoded, sorted and de-duplicated; a vertex id is the rank of its
// lattice point in that order.
extern "C" int svlf_octree_build_vertices(svlf_octree tree, int64_t *n_vertices, void *stream) {
    if (!tree) return SVLF_ERR_ARG;
    OctreeHost &H = tree->h;
    if (H.vtx_dev) {
        if (n_vertices) *n_vertices = H.view.n_vertices;
        return SVLF_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = H.view.n_leaves;
    std::vector<int32_t> ijk((size_t)n * 3);
    if (n > 0) {
        if (cudaMemcpyAsync(ijk.data(), H.leaf_ijk_dev, sizeof(int32_t) * 3 * (size_t)n,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SVLF_ERR_CUDA;
    }
    std::vector<uint64_t> code((size_t)n * 8);
    for (int64_t q = 0; q < n; ++q)
        for (int c = 0; c < 8; ++c)
            code[(size_t)q * 8 + c] = morton3((uint32_t)ijk[3 * q] + (c & 1), (uint32_t)ijk[3 * q + 1] + ((c >> 1) & 1),
                                              (uint32_t)ijk[3 * q + 2] + ((c >> 2) & 1));
    std::vector<uint64_t> uniq(code);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    if ((int64_t)uniq.size() >= ((int64_t)1 << 31)) return SVLF_ERR_UNSUPPORTED;
    std::vector<int32_t> vid(code.size());
    for (size_t i = 0; i < code.size(); ++i)
        vid[i] = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), code[i]) - uniq.begin());
    int32_t *dev = nullptr;
    const size_t nb = sizeof(int32_t) * (vid.size() > 0 ? vid.size() : 8);
    if (cudaMalloc(&dev, nb) != cudaSuccess) return SVLF_ERR_CUDA;
    if (!vid.empty() &&
        (cudaMemcpyAsync(dev, vid.data(), sizeof(int32_t) * vid.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
        cudaFree(dev);
        return SVLF_ERR_CUDA;
    }
    H.vtx_dev = dev;
    H.view.leaf_vertices = dev;
    H.view.n_vertices = (int64_t)uniq.size();
    if (n_vertices) *n_vertices = H.view.n_vertices;
    return SVLF_OK;
}

extern "C" int svlf_octree_leaf_vertices(svlf_octree tree, int32_t *out, void *stream) {
    if (!tree || !out) return SVLF_ERR_ARG;
    if (!tree->h.vtx_dev) return SVLF_ERR_ARG;
    const size_t nb = sizeof(int32_t) * 8 * (size_t)tree->h.view.n_leaves;
    if (nb == 0) return SVLF_OK;
    return cudaMemcpyAsync(out, tree->h.vtx_dev, nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) ==
                   cudaSuccess
               ? SVLF_OK
               : SVLF_ERR_CUDA;
}

namespace svlf {
const OctreeView &octree_view(svlf_octree t) { return t->h.view; }
}  // namespace svlf

// ============================================================================
// Octree built on the GPU from depth maps (Sec. 4.1: the scene's voxel grid
// comes from the dataset's depth maps; Sec. 4.5 builds it at 128^3).
//
// No sort is needed: a pixel's surface point x = o + D d marks bit
// Morton(floor(x 2^L)) of an occupancy bitmap, and in Morton order the 64
// leaves of one brick (level L-2 node) are one 64-bit word of that bitmap.
// So the bricks are the non-zero words, a leaf's rank is the exclusive
// prefix sum of the words' popcounts plus its rank inside the word, and each
// node level above is one pass over groups of 8 child-existence flags. The
// arrays produced are exactly those of svlf_build_octree for the same leaves.
// ============================================================================
namespace svlf {
namespace {

__device__ __forceinline__ uint64_t spread3_dev(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__device__ __forceinline__ uint32_t compact3_dev(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x ^ (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x ^ (x >> 8)) & 0x1F0000FF0000FFull;
    x = (x ^ (x >> 16)) & 0x1F00000000FFFFull;
    x = (x ^ (x >> 32)) & 0x1FFFFFull;
    return (uint32_t)x;
}

__global__ void backproject_kernel(const float *__restrict__ rays, const float *__restrict__ depth, int64_t n,
                                   int L, unsigned long long *__restrict__ bitmap) {
    const int nc = 1 << L;
    const float fn = (float)nc;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const float D = depth[p];
        if (!(D > 0.f) || !isfinite(D)) continue;
        uint32_t c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // the product rounded, then the sum rounded (no contraction into an FMA)
            const float x = __fadd_rn(rays[6 * p + a], __fmul_rn(D, rays[6 * p + 3 + a]));
            c[a] = (uint32_t)min(max((int)floorf(x * fn), 0), nc - 1);
        }
        const uint64_t code = spread3_dev(c[0]) | (spread3_dev(c[1]) << 1) | (spread3_dev(c[2]) << 2);
        atomicOr(bitmap + (code >> 6), 1ull << (code & 63));
    }
}

__global__ void word_stats_kernel(const unsigned long long *__restrict__ bitmap, int64_t W,
                                  uint32_t *__restrict__ flag, uint32_t *__restrict__ cnt) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long m = bitmap[w];
        flag[w] = m != 0ull;
        cnt[w] = (uint32_t)__popcll(m);
    }
}

// Exclusive scan of up to 1024 * gridDim values per launch: each block scans
// its 1024 (4 per thread), writes its total to sums[block].
__global__ void scan_block_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                                  uint32_t *__restrict__ sums) {
    __shared__ uint32_t s[256];
    const int64_t base = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t v[4], t = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[e] = base + e < n ? in[base + e] : 0u;
        t += v[e];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {  // inclusive Hillis-Steele over the thread totals
        const uint32_t x = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - t;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (base + e < n) out[base + e] = run;
        run += v[e];
    }
    if (threadIdx.x == 255) sums[blockIdx.x] = s[255];
}

__global__ void scan_add_kernel(uint32_t *__restrict__ out, int64_t n, const uint32_t *__restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (i + e < n) out[i + e] += offs[blockIdx.x];
}

__global__ void bricks_kernel(const unsigned long long *__restrict__ bitmap, int64_t W,
                              const uint32_t *__restrict__ brick_idx, const uint32_t *__restrict__ leaf_base,
                              uint4 *__restrict__ bricks, int32_t *__restrict__ leaf_ijk) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long m = bitmap[w];
        if (!m) continue;
        const uint32_t base = leaf_base[w];
        bricks[brick_idx[w]] = make_uint4((uint32_t)m, (uint32_t)(m >> 32), base, 0u);
        unsigned long long r = m;
        uint32_t k = 0;
        while (r) {
            const int b = __ffsll((long long)r) - 1;
            r &= r - 1;
            const uint64_t code = ((uint64_t)w << 6) | (uint64_t)b;
            leaf_ijk[3 * (int64_t)(base + k)] = (int32_t)compact3_dev(code);
            leaf_ijk[3 * (int64_t)(base + k) + 1] = (int32_t)compact3_dev(code >> 1);
            leaf_ijk[3 * (int64_t)(base + k) + 2] = (int32_t)compact3_dev(code >> 2);
            ++k;
        }
    }
}

// Parent level from child-existence flags (8 children per parent, Morton order).
__global__ void level_mask_kernel(const uint32_t *__restrict__ child_flag, int64_t n_parent,
                                  uint8_t *__restrict__ mask, uint32_t *__restrict__ flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_parent;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) m |= (child_flag[8 * p + c] ? 1u : 0u) << c;
        mask[p] = (uint8_t)m;
        flag[p] = m != 0u;
    }
}

// Node words of one level: mask << 24 | absolute index of the first child
// (the child level's compact index of child 8p + lowest set bit, plus the
// child level's offset in the node array; 0 offset when the children are bricks).
__global__ void node_words_kernel(const uint8_t *__restrict__ mask, const uint32_t *__restrict__ idx,
                                  int64_t n_cells, const uint32_t *__restrict__ child_idx, uint32_t child_off,
                                  uint32_t *__restrict__ nodes) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_cells;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = mask[p];
        if (!m) continue;
        const int first = __ffs((int)m) - 1;
        nodes[idx[p]] = (m << 24) | (child_off + child_idx[8 * p + first]);
    }
}

struct LevelPtrs {
    const uint32_t *flag[kMaxDepth];  // existence per cell of level l (Morton order)
};

// Dense parent index: per level-(L-3) cell (x fastest), its node word, or (mask
// 0) log2 of the edge of the largest empty block around it: the child, at
// level l + 1, of its deepest existing ancestor l. (box_grow_kernel and
// box_fill_kernel then turn the empty blocks into grown boxes.)
__global__ void pgrid_kernel(const __grid_constant__ LevelPtrs lv, int L, const uint32_t *__restrict__ node_idx,
                             const uint32_t *__restrict__ nodes, uint32_t off_top, uint2 *__restrict__ pgrid) {
    const int top = L - 3;
    const int64_t P = (int64_t)1 << top;
    const int64_t n = P * P * P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(i % P), y = (uint32_t)((i / P) % P), z = (uint32_t)(i / (P * P));
        const uint64_t m = spread3_dev(x) | (spread3_dev(y) << 1) | (spread3_dev(z) << 2);
        uint32_t v = (uint32_t)L;
        if (lv.flag[top][m]) {
            v = nodes[off_top + node_idx[m]];
        } else {
            for (int l = top - 1; l >= 0; --l)
                if (lv.flag[l][m >> (3 * (top - l))]) {
                    v = (uint32_t)(L - l - 1);
                    break;
                }
        }
        pgrid[i] = make_uint2(v, 0u);
    }
}

// Summed-volume table of the occupied parents (S zeroed before; (G+1)^3, x
// fastest), one axis per launch: pass 0 writes the running count along x,
// passes 1 and 2 accumulate it along y and then z in place.
__global__ void svt_kernel(const uint2 *__restrict__ pgrid, int G, int pass, int32_t *__restrict__ S) {
    const int64_t W = G + 1;
    const int64_t rows = (int64_t)G * G;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(r % G), v = (int)(r / G);
        int32_t acc = 0;
        for (int k = 0; k < G; ++k) {
            const int x = pass == 0 ? k : u;
            const int y = pass == 0 ? u : pass == 1 ? k : v;
            const int z = pass == 2 ? k : v;
            const int64_t o = ((int64_t)(z + 1) * W + y + 1) * W + x + 1;
            acc += pass == 0 ? ((pgrid[((int64_t)z * G + y) * G + x].x >> 24) ? 1 : 0) : S[o];
            S[o] = acc;
        }
    }
}

// Empty parent cell -> the corner of its empty block, in level L-3 cells.
__device__ __forceinline__ void empty_block_corner(uint32_t w, int G, int64_t i, int lo[3], int &e) {
    e = 1 << ((int)(w & 31u) - 3);
    lo[0] = (int)(i % G) & ~(e - 1);
    lo[1] = (int)((i / G) % G) & ~(e - 1);
    lo[2] = (int)(i / ((int64_t)G * G)) & ~(e - 1);
}

// The corner cell of each empty block grows the block into its empty box
// (written to `boxes` at the corner's index; pgrid is left as it is).
__global__ void box_grow_kernel(const uint2 *__restrict__ pgrid, int G, const int32_t *__restrict__ S,
                                uint2 *__restrict__ boxes) {
    const int64_t n = (int64_t)G * G * G;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = pgrid[i].x;
        if (w >> 24) continue;
        int lo[3], e;
        empty_block_corner(w, G, i, lo, e);
        if (((int64_t)lo[2] * G + lo[1]) * G + lo[0] != i) continue;
        int hi[3] = {lo[0] + e, lo[1] + e, lo[2] + e};
        grow_empty_box(S, G, lo, hi);
        boxes[i] = make_uint2(pack_corner(lo), pack_corner(hi));
    }
}

// Every cell of each empty block (its corner included) takes the block's box.
__global__ void box_fill_kernel(uint2 *__restrict__ pgrid, int G, const uint2 *__restrict__ boxes) {
    const int64_t n = (int64_t)G * G * G;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = pgrid[i].x;
        if (w >> 24) continue;
        int lo[3], e;
        empty_block_corner(w, G, i, lo, e);
        pgrid[i] = boxes[((int64_t)lo[2] * G + lo[1]) * G + lo[0]];
    }
}

unsigned grid_for_n(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Exclusive scan of n uint32 values (device) into out; returns the total
// (synchronises s). tmp: scratch of at least scan_tmp_words(n) words.
int64_t scan_tmp_words(int64_t n) {
    int64_t w = 0;
    while (n > 1) {
        n = (n + 1023) / 1024;
        w += 2 * n + 2;
    }
    return w + 4;
}

int exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s, uint32_t *total) {
    if (n <= 0) {
        *total = 0;
        return SVLF_OK;
    }
    const int64_t nb = (n + 1023) / 1024;
    uint32_t *sums = tmp, *sums_scan = tmp + nb;
    scan_block_kernel<<<(unsigned)nb, 256, 0, s>>>(in, out, n, sums);
    if (nb > 1) {
        uint32_t t = 0;
        int rc = exclusive_scan(sums, sums_scan, nb, tmp + 2 * nb, s, &t);
        if (rc) return rc;
        scan_add_kernel<<<(unsigned)nb, 256, 0, s>>>(out, n, sums_scan);
        *total = t;
    } else {
        if (cudaMemcpyAsync(total, sums, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SVLF_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

}  // namespace
}  // namespace svlf

namespace svlf {
namespace {

// One bit per given leaf in the Morton-indexed occupancy bitmap (duplicates
// merge); coordinates outside [0, 2^L) are counted in *bad and skipped.
__global__ void leaves_to_bitmap_kernel(const int32_t *__restrict__ ijk, int64_t n, int L,
                                        unsigned long long *__restrict__ bitmap, unsigned int *__restrict__ bad) {
    const int side = 1 << L;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int i = ijk[3 * p], j = ijk[3 * p + 1], k = ijk[3 * p + 2];
        if (i < 0 || j < 0 || k < 0 || i >= side || j >= side || k >= side) {
            atomicAdd(bad, 1u);
            continue;
        }
        const uint64_t code = spread3_dev((uint32_t)i) | (spread3_dev((uint32_t)j) << 1) | (spread3_dev((uint32_t)k) << 2);
        atomicOr(bitmap + (code >> 6), 1ull << (code & 63));
    }
}

// The octree of the leaves a fill step marks in a zeroed occupancy bitmap of
// 2^(3L) bits (one 64-bit word per level L-2 cell): brick and leaf ranks by
// prefix scans, node levels bottom-up, the parent index with its grown empty
// boxes. `fill(bitmap)` queues the marking on `s` and may return an error.
template <typename Fill>
int build_octree_gpu(int L, cudaStream_t s, Fill fill, svlf_octree *out, int64_t *n_leaves_out);

}  // namespace
}  // namespace svlf

extern "C" int svlf_build_octree(const int32_t *leaf_ijk, int64_t n, int depth, void *stream,
                                 svlf_octree *out, int64_t *n_leaves_out) {
    if (!out || n < 0 || (n > 0 && !leaf_ijk)) return SVLF_ERR_ARG;
    if (depth < 2 || depth > kMaxDepth) return SVLF_ERR_UNSUPPORTED;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    return build_octree_gpu(depth, s, [&](unsigned long long *bitmap) -> int {
        if (n == 0) return SVLF_OK;
        unsigned int *bad = nullptr;
        if (cudaMalloc(&bad, sizeof(unsigned int)) != cudaSuccess) return SVLF_ERR_CUDA;
        unsigned int h_bad = 0;
        int rc = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s) == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
        if (!rc) leaves_to_bitmap_kernel<<<grid_for_n(n), 256, 0, s>>>(leaf_ijk, n, depth, bitmap, bad);
        if (!rc && (cudaGetLastError() != cudaSuccess ||
                    cudaMemcpyAsync(&h_bad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess))
            rc = SVLF_ERR_CUDA;
        cudaFree(bad);
        if (!rc && h_bad) rc = SVLF_ERR_ARG;
        return rc;
    }, out, n_leaves_out);
}

extern "C" int svlf_build_octree_from_depth(const float *rays, const float *depth, int64_t n, int L, void *stream,
                                            svlf_octree *out, int64_t *n_leaves_out) {
    if (!out || n < 0 || (n > 0 && (!rays || !depth))) return SVLF_ERR_ARG;
    if (L < 2 || L > kMaxDepth) return SVLF_ERR_UNSUPPORTED;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    return build_octree_gpu(L, s, [&](unsigned long long *bitmap) -> int {
        if (n > 0) backproject_kernel<<<grid_for_n(n), 256, 0, s>>>(rays, depth, n, L, bitmap);
        return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
    }, out, n_leaves_out);
}

namespace svlf {
namespace {
template <typename Fill>
int build_octree_gpu(int L, cudaStream_t s, Fill fill, svlf_octree *out, int64_t *n_leaves_out) {
    const int n_levels = L - 2;
    const int64_t W = (int64_t)1 << (3 * L - 6);  // bitmap words = level L-2 cells
    std::vector<void *> scratch;
    auto dalloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes > 0 ? bytes : 16) != cudaSuccess) return nullptr;
        scratch.push_back(p);
        return p;
    };
    auto cleanup = [&]() {
        for (void *p : scratch) cudaFree(p);
        scratch.clear();
    };
    // per level: flags, compact index, masks; level n_levels = the bricks
    std::vector<uint32_t *> flag(n_levels + 1), idx(n_levels + 1);
    std::vector<uint8_t *> mask(n_levels + 1, nullptr);
    std::vector<uint32_t> count(n_levels + 1, 0);
    unsigned long long *bitmap = (unsigned long long *)dalloc(sizeof(unsigned long long) * (size_t)W);
    uint32_t *cnt = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)W);
    uint32_t *leaf_base = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)W);
    uint32_t *tmp = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)scan_tmp_words(W));
    flag[n_levels] = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)W);
    idx[n_levels] = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)W);
    if (!bitmap || !cnt || !leaf_base || !tmp || !flag[n_levels] || !idx[n_levels]) {
        cleanup();
        return SVLF_ERR_CUDA;
    }
    int rc = SVLF_OK;
    uint32_t n_leaves = 0;
    if (cudaMemsetAsync(bitmap, 0, sizeof(unsigned long long) * (size_t)W, s) != cudaSuccess) rc = SVLF_ERR_CUDA;
    if (!rc) rc = fill(bitmap);
    if (!rc) word_stats_kernel<<<grid_for_n(W), 256, 0, s>>>(bitmap, W, flag[n_levels], cnt);
    if (!rc) rc = exclusive_scan(flag[n_levels], idx[n_levels], W, tmp, s, &count[n_levels]);
    if (!rc) rc = exclusive_scan(cnt, leaf_base, W, tmp, s, &n_leaves);
    if (!rc && count[n_levels] >= (1u << 24)) rc = SVLF_ERR_UNSUPPORTED;
    // node levels bottom-up
    for (int l = n_levels - 1; l >= 0 && !rc; --l) {
        const int64_t cells = (int64_t)1 << (3 * l);
        mask[l] = (uint8_t *)dalloc((size_t)cells);
        flag[l] = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)cells);
        idx[l] = (uint32_t *)dalloc(sizeof(uint32_t) * (size_t)cells);
        if (!mask[l] || !flag[l] || !idx[l]) {
            rc = SVLF_ERR_CUDA;
            break;
        }
        level_mask_kernel<<<grid_for_n(cells), 256, 0, s>>>(flag[l + 1], cells, mask[l], flag[l]);
        rc = exclusive_scan(flag[l], idx[l], cells, tmp, s, &count[l]);
    }
    std::vector<uint32_t> off(n_levels + 1, 0);
    for (int l = 0; l < n_levels; ++l) off[l + 1] = off[l] + count[l];
    const uint32_t n_nodes = n_levels > 0 ? off[n_levels] : 0;
    if (!rc && n_nodes >= (1u << 24)) rc = SVLF_ERR_UNSUPPORTED;
    svlf_octree_s *t = nullptr;
    if (!rc) {
        t = new (std::nothrow) svlf_octree_s;
        if (!t) rc = SVLF_ERR_CUDA;
    }
    if (!rc) {
        std::memset(t, 0, sizeof(*t));
        OctreeHost &H = t->h;
        const int64_t P = n_levels > 0 ? (int64_t)1 << (L - 3) : 0;
        const int64_t n_pgrid = P * P * P;
        bool ok = cudaMalloc(&H.leaf_ijk_dev, sizeof(int32_t) * 3 * ((size_t)n_leaves + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&H.bricks_dev, sizeof(uint4) * ((size_t)count[n_levels] + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&H.nodes_dev, sizeof(uint32_t) * ((size_t)n_nodes + 1)) == cudaSuccess;
        ok = ok && cudaMalloc(&H.pgrid_dev, sizeof(uint2) * ((size_t)n_pgrid + 1)) == cudaSuccess;
        const int G = (int)P;
        const size_t svt_bytes = sizeof(int32_t) * (size_t)((G + 1) * (G + 1) * (G + 1));
        const bool want_boxes = n_levels > 0 && n_leaves > 0;
        int32_t *svt = want_boxes ? (int32_t *)dalloc(svt_bytes) : nullptr;
        uint2 *boxes = want_boxes ? (uint2 *)dalloc(sizeof(uint2) * (size_t)n_pgrid) : nullptr;
        ok = ok && ((svt && boxes) || !want_boxes);
        if (!ok) {
            rc = SVLF_ERR_CUDA;
        } else {
            bricks_kernel<<<grid_for_n(W), 256, 0, s>>>(bitmap, W, idx[n_levels], leaf_base, H.bricks_dev,
                                                        H.leaf_ijk_dev);
            for (int l = 0; l < n_levels; ++l) {
                const int64_t cells = (int64_t)1 << (3 * l);
                const uint32_t child_off = l + 1 < n_levels ? off[l + 1] : 0u;  // bricks are indexed from 0
                node_words_kernel<<<grid_for_n(cells), 256, 0, s>>>(mask[l], idx[l], cells, idx[l + 1], child_off,
                                                                    H.nodes_dev + off[l]);
            }
            if (n_levels > 0 && n_leaves > 0) {
                LevelPtrs lv;
                std::memset(&lv, 0, sizeof(lv));
                for (int l = 0; l < n_levels; ++l) lv.flag[l] = flag[l];
                pgrid_kernel<<<grid_for_n(n_pgrid), 256, 0, s>>>(lv, L, idx[n_levels - 1], H.nodes_dev,
                                                                 off[n_levels - 1], H.pgrid_dev);
                if (cudaMemsetAsync(svt, 0, svt_bytes, s) != cudaSuccess) rc = SVLF_ERR_CUDA;
                for (int pass = 0; pass < 3; ++pass)
                    svt_kernel<<<grid_for_n((int64_t)G * G), 256, 0, s>>>(H.pgrid_dev, G, pass, svt);
                box_grow_kernel<<<grid_for_n(n_pgrid), 256, 0, s>>>(H.pgrid_dev, G, svt, boxes);
                box_fill_kernel<<<grid_for_n(n_pgrid), 256, 0, s>>>(H.pgrid_dev, G, boxes);
            }
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = SVLF_ERR_CUDA;
        }
        H.view.depth = L;
        H.view.n_node_levels = n_levels;
        H.view.n_leaves = n_leaves;
        H.view.n_nodes = (int)n_nodes;
        H.view.n_bricks = (int)count[n_levels];
        H.view.root_is_brick = n_levels == 0;
        H.view.empty = n_leaves == 0;
        H.view.nodes = H.nodes_dev;
        H.view.bricks = H.bricks_dev;
        H.view.pgrid = H.pgrid_dev;
        H.view.pgrid_shift = n_levels > 0 ? L - 3 : 0;
        if (rc) {
            cudaFree(H.leaf_ijk_dev);
            cudaFree(H.bricks_dev);
            cudaFree(H.nodes_dev);
            cudaFree(H.pgrid_dev);
            delete t;
            t = nullptr;
        }
    }
    cleanup();
    if (rc) return rc;
    *out = t;
    if (n_leaves_out) *n_leaves_out = n_leaves;
    return SVLF_OK;
}
}  // namespace
}  // namespace svlf
