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

}  // namespace svlf

using namespace svlf;

struct svlf_octree_s {
    OctreeHost h;
};

extern "C" int svlf_build_octree(const int32_t *leaf_ijk, int64_t n, int depth, void *stream,
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
    // empty octree block that contains the cell. One load then answers what a
    // descent from the root would: the cell's brick or its empty block.
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
    size_t nb_pgrid = sizeof(uint32_t) * (pgrid.size() + 1);
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
    if (ok && !pgrid.empty())
        ok = cudaMemcpyAsync(H.pgrid_dev, pgrid.data(), sizeof(uint32_t) * pgrid.size(),
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
