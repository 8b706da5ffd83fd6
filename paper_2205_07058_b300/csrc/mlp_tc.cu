// The per-sample network on the 5th-generation tensor cores (tcgen05):
// SVLF_BF16 and SVLF_FP16 (16-bit operands, float32 accumulation in TMEM).
//
// Forward kernel (persistent, one CTA per SM, 2-4 warpgroups):
//  * The packed weights of every layer (16-bit, core-matrix layout, plus the
//    float32 biases) are copied once per CTA into shared memory with bulk
//    (TMA) copies and stay resident.
//  * Each warpgroup owns a tile of 128 samples at a time: thread t builds the
//    network input of sample t (feature gather with 16-byte loads, ray
//    parameterisation from an exactly formed point of the ray), rounds it to
//    16 bits and stores it in the warpgroup's activation buffer (the A
//    operand).
//  * One thread issues the layer's tcgen05.mma instructions (M = 128 samples,
//    N = layer width, K = 16 each) into the warpgroup's 128 TMEM columns and
//    commits them to an mbarrier. A hidden layer's first MMA multiplies a
//    block of ones by the bias split into 16-bit pieces, so the accumulator
//    starts at the bias with no TMEM store on the tile's critical path. The
//    warpgroup waits, reads its row of the accumulator (tcgen05.ld, lane =
//    sample), applies ReLU, rounds to 16 bits and writes the next layer's A
//    operand in place.
//  * The last layer (N padded 4 -> 16) writes sigmoid colour and ReLU optical
//    thickness per sample.
//  Warpgroups run independently, so the tensor core works on one tile while
//  the others gather inputs or run their epilogues.
//
// Batched form: one launch serves every scene of a SceneTable. Each CTA takes
// a contiguous range of the global tile list (scenes in order, tiles of 128
// samples of one scene each) and walks it scene segment by scene segment,
// reloading the resident weights only when the scene changes.
#include <cstring>

#include "svlf_internal.cuh"
#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace svlf {

constexpr int kTcTile = 128;     // samples per tile (MMA M)
constexpr int kMaxKSteps = 9;    // K = 16 steps of the longest K loop (K0 <= 144, tiles of 128)
constexpr int kTcOutN = 16;      // output layer width padded to the smallest legal N
constexpr int kHp = 128;         // hidden width inside the tensor-core path (zero-padded)

struct TcLayout {
    int K0;                      // first-layer K, in0 rounded up to 16
    int n_layers;                // nh + 1
    uint32_t w_off[kMaxLayers];  // byte offset of each layer's B tile in the image
    uint32_t w_rows[kMaxLayers]; // rows (N) of each B tile
    uint32_t w_cols[kMaxLayers]; // columns (K) of each B tile
    uint32_t bias_off;           // byte offset of the float32 biases
    uint32_t bias_l[kMaxLayers]; // float index of each layer's bias within the bias block
    uint32_t bytes;              // weights + float32 biases (multiple of 16): what the backward copies
    // Forward-only tail: each hidden layer's bias as the B operand of one extra
    // K = 16 MMA against a block of ones, so the accumulator starts at the bias
    // without a TMEM store. B tile l holds the 8-column K group 0 of an N = 128
    // tile: columns 0..2 = the bias split into three 16-bit pieces (hi + mid +
    // lo, exact for BF16), 3..7 = 0; its K group 1 (leading byte offset 2 KB) is
    // the next region, which the zero half of the ones block multiplies away.
    uint32_t bias_b_off[kMaxLayers];
    uint32_t ones_off;           // 2 KB of 16-bit 1.0 (A rows, K group 0), then 2 KB of zeros (group 1)
    uint32_t fwd_bytes;          // total image size, forward tail included
};

static TcLayout tc_layout(const MlpDims &md) {
    TcLayout t;
    memset(&t, 0, sizeof(t));
    t.K0 = (md.in0 + 15) & ~15;
    t.n_layers = md.nh + 1;
    uint32_t off = 0;
    for (int l = 0; l <= md.nh; ++l) {
        t.w_rows[l] = l == md.nh ? kTcOutN : kHp;
        t.w_cols[l] = l == 0 ? t.K0 : kHp;
        t.w_off[l] = off;
        off += t.w_rows[l] * t.w_cols[l] * 2;
    }
    t.bias_off = off;
    uint32_t nb = 0;
    for (int l = 0; l <= md.nh; ++l) {
        t.bias_l[l] = nb;
        nb += t.w_rows[l];
    }
    off += nb * 4;
    t.bytes = (off + 15) & ~15u;
    off = (t.bytes + 127) & ~127u;
    for (int l = 0; l < md.nh; ++l) {
        t.bias_b_off[l] = off;
        off += kHp * 16;
    }
    t.ones_off = off;
    t.fwd_bytes = off + 2 * kTcTile * 16;
    return t;
}

bool tc_supported(const MlpDims &md) {
    return md.H <= kHp && md.H % 16 == 0 && md.in0 <= 144 && md.nh >= 1 && md.nh <= 6 && md.out <= kTcOutN;
}

size_t packed_tc_bytes(const MlpDims &md) {
    if (!tc_supported(md)) return 0;
    return tc_layout(md).fwd_bytes;
}

// ---------------------------------------------------------------- packing
// One launch packs every scene of the table: blockIdx.y = scene.
__global__ void pack_tc_kernel(const __grid_constant__ SceneTable T, MlpDims md, TcLayout lay, int fp16,
                               uint8_t *__restrict__ packed, size_t stride) {
    const float *__restrict__ params = T.s[blockIdx.y].params;
    if (!params) return;  // a scene without rays may come without parameters; nothing reads its image
    uint8_t *__restrict__ image = packed + blockIdx.y * stride;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    for (int l = 0; l <= md.nh; ++l) {
        const int R = lay.w_rows[l], C = lay.w_cols[l];
        const int out = md.out_l[l], in = md.in_l[l];
        const float *W = params + md.w_off[l];
        for (int e = tid; e < R * C; e += nthr) {
            const int r = e / C, k = e % C;
            const float v = (r < out && k < in) ? W[r * in + k] : 0.f;
            uint16_t bits;
            if (fp16) {
                __half h = __float2half_rn(v);
                bits = *reinterpret_cast<uint16_t *>(&h);
            } else {
                __nv_bfloat16 h = __float2bfloat16_rn(v);
                bits = *reinterpret_cast<uint16_t *>(&h);
            }
            *reinterpret_cast<uint16_t *>(image + lay.w_off[l] + tc::cm_offset(r, k, R)) = bits;
        }
        float *bias = reinterpret_cast<float *>(image + lay.bias_off) + lay.bias_l[l];
        for (int r = tid; r < R; r += nthr) bias[r] = r < out ? W[out * in + r] : 0.f;
        if (l < md.nh) {
            // forward tail: the bias as three 16-bit pieces (K columns 0..2 of B)
            for (int r = tid; r < kHp; r += nthr) {
                const float b = r < out ? W[out * in + r] : 0.f;
                float piece[3];
                float rem = b;
                for (int j = 0; j < 3; ++j) {
                    piece[j] = fp16 ? __half2float(__float2half_rn(rem))
                                    : __bfloat162float(__float2bfloat16_rn(rem));
                    rem -= piece[j];
                }
                for (int k = 0; k < 8; ++k) {
                    const float v = k < 3 ? piece[k] : 0.f;
                    uint16_t bits;
                    if (fp16) {
                        __half h = __float2half_rn(v);
                        bits = *reinterpret_cast<uint16_t *>(&h);
                    } else {
                        __nv_bfloat16 h = __float2bfloat16_rn(v);
                        bits = *reinterpret_cast<uint16_t *>(&h);
                    }
                    *reinterpret_cast<uint16_t *>(image + lay.bias_b_off[l] + tc::cm_offset(r, k, kHp)) = bits;
                }
            }
        }
    }
    const uint16_t one = fp16 ? 0x3C00u : 0x3F80u;
    uint16_t *ones = reinterpret_cast<uint16_t *>(image + lay.ones_off);
    for (int e = tid; e < 2 * kTcTile * 8; e += nthr) ones[e] = e < kTcTile * 8 ? one : 0u;
}

int launch_pack_tc(const MlpDims &md, int precision, const SceneTable &T, void *packed,
                   size_t stride, cudaStream_t s) {
    if (!tc_supported(md)) return SVLF_ERR_UNSUPPORTED;
    const TcLayout lay = tc_layout(md);
    prof_begin("pack_weights_tc", s);
    if (T.n > 0)
        pack_tc_kernel<<<dim3(32, (unsigned)T.n), 256, 0, s>>>(T, md, lay, precision == SVLF_FP16, (uint8_t *)packed,
                                                               stride);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

// ---------------------------------------------------------------- forward
struct TcFwdParams {
    MlpDims md;
    TcLayout lay;
    int fp16;
    int feat_bf16;
    const uint8_t *images;  // packed weights, scene i at images + i * image_stride
    size_t image_stride;
    Sample *samples;     // read; the two-decoder colour pass also rewrites each tmid
    const unsigned int *counter;
    float4 *outputs;
    float4 *aux;         // two-decoder: (tau, eta, t_in, t_out) per sample, F^T pass -> F^C pass
    int n_wg;            // warpgroups per CTA
    uint32_t abuf_bytes; // activation buffer per warpgroup
    int bias_mma;        // 1: hidden biases enter through the MMA (image copied with its forward tail);
                         // 0: they are stored into TMEM before each layer (tail left out, to save shared memory)
    uint32_t wbytes;     // bytes of the image copied into shared memory: fwd_bytes or bytes
};

// Per-CTA view of the global tile list: scene s owns global tiles
// [tile0[s], tile0[s+1]); its tile t covers its samples [t*128, t*128+128) of
// the S[s] it wrote, which start at global sample index K * ray_begin_s.
struct TileMap {
    int64_t tile0[kMaxScenes + 1];
    int64_t S[kMaxScenes];
};

__device__ __forceinline__ void tile_map_build(const SceneTable &T, const unsigned int *counter,
                                               TileMap &m) {
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < T.n; ++i) {
            const int64_t cap = T.s[i].n_rays * (int64_t)T.K;
            // a scene without output gradients has no tiles in a backward
            const int64_t Si = T.s[i].grad ? min((int64_t)counter[kCtrScene + i], cap) : 0;
            m.S[i] = Si;
            m.tile0[i] = acc;
            acc += (Si + kTcTile - 1) / kTcTile;
        }
        m.tile0[T.n] = acc;
    }
    __syncthreads();
}

// Store one 16-bit row chunk (8 values packed in 4 words) at column block kb.
__device__ __forceinline__ void st_chunk(uint8_t *abuf, int row, int kb, uint32_t a, uint32_t b,
                                         uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4 *>(abuf + kb * (kTcTile * 16) + (row >> 3) * 128 + (row & 7) * 16) =
        make_uint4(a, b, c, d);
}

// Half a chunk (8 bytes: four 16-bit values) of row `row`, chunk `kb`.
__device__ __forceinline__ void st_half_chunk(uint8_t *abuf, int row, int kb, int half, uint32_t a, uint32_t b) {
    *reinterpret_cast<uint2 *>(abuf + kb * (kTcTile * 16) + (row >> 3) * 128 + (row & 7) * 16 + half * 8) =
        make_uint2(a, b);
}

// Network input h0 = [z | d | p~1 | p~2] of sample `s` written straight into
// row `row` of a 16-bit A operand (K0 columns): F/8 chunks of features, two
// chunks of ray direction and entry/exit parameters, zero chunks up to K0.
__device__ __forceinline__ void build_input_chunks(const MlpDims &md, int K0, int depth, int rparam,
                                                   const void *feats, int feat_bf16,
                                                   const float *rays, int64_t ray_begin,
                                                   const Sample &sm, bool valid, int fp16,
                                                   uint8_t *abuf, int row, int *leaf_out) {
    const int F = md.F;
    int kb = 0;
    if (valid) {
        if (leaf_out) *leaf_out = sm.leaf;
        // every load of the row is issued before the first use (up to 128 bytes of
        // features per batch, F <= 32 float32 or F <= 64 bfloat16 in one batch), so
        // the row costs one memory latency, not one per chunk
        const float2 *rp = reinterpret_cast<const float2 *>(rays + 6 * ((int64_t)sm.ray - ray_begin));
        const float2 ra = __ldg(rp), rb = __ldg(rp + 1), rc = __ldg(rp + 2);
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(feats) +
                                                           (int64_t)sm.leaf * F * (feat_bf16 ? 2 : 4));
        const int nq = feat_bf16 ? F / 8 : F / 4;  // 16-byte loads in the row
        for (int q0 = 0; q0 < nq; q0 += 8) {
            uint4 buf[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q0 + q < nq) buf[q] = __ldg(src + q0 + q);
            if (feat_bf16) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q0 + q >= nq) break;
                    uint4 v = buf[q];
                    if (fp16) {
                        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                        uint32_t o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            o[e] = tc::pack2(__uint_as_float(w[e] << 16), __uint_as_float(w[e] & 0xFFFF0000u), true);
                        v = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                    st_chunk(abuf, row, kb++, v.x, v.y, v.z, v.w);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    if (q0 + q >= nq) break;
                    const uint4 a = buf[q], b = buf[q + 1];
                    st_chunk(abuf, row, kb++, tc::pack2(__uint_as_float(a.x), __uint_as_float(a.y), fp16),
                             tc::pack2(__uint_as_float(a.z), __uint_as_float(a.w), fp16),
                             tc::pack2(__uint_as_float(b.x), __uint_as_float(b.y), fp16),
                             tc::pack2(__uint_as_float(b.z), __uint_as_float(b.w), fp16));
                }
            }
        }
        const float o[3] = {ra.x, ra.y, rb.x};
        const float d[3] = {rb.y, rc.x, rc.y};
        float p1[3], p2[3];
        voxel_param_at(rparam, o, d, sm.tmid, sm.cell, depth, p1, p2);
        st_chunk(abuf, row, kb++, tc::pack2(d[0], d[1], fp16), tc::pack2(d[2], p1[0], fp16),
                 tc::pack2(p1[1], p1[2], fp16), tc::pack2(p2[0], p2[1], fp16));
        st_chunk(abuf, row, kb++, tc::pack2(p2[2], 0.f, fp16), 0u, 0u, 0u);
    }
    for (; kb < K0 / 8; ++kb) st_chunk(abuf, row, kb, 0u, 0u, 0u, 0u);
}

// The part of build_input_chunks' row that warpgroup `half` of a tile shared by
// two warpgroups writes: the feature chunks (half 0), or the direction and
// entry/exit parameter chunks and the zero padding (half 1). F % 8 == 0.
__device__ __forceinline__ void build_input_chunks_half(int half, const MlpDims &md, int K0, int depth, int rparam,
                                                        const void *feats, int feat_bf16, const float *rays,
                                                        int64_t ray_begin, const Sample &sm, bool valid, int fp16,
                                                        uint8_t *abuf, int row) {
    const int F = md.F;
    if (half == 0) {
        if (!valid) {
            for (int kb = 0; kb < F / 8; ++kb) st_chunk(abuf, row, kb, 0u, 0u, 0u, 0u);
            return;
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(feats) +
                                                           (int64_t)sm.leaf * F * (feat_bf16 ? 2 : 4));
        const int nq = feat_bf16 ? F / 8 : F / 4;  // 16-byte loads in the row
        int kb = 0;
        for (int q0 = 0; q0 < nq; q0 += 8) {
            uint4 buf[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q0 + q < nq) buf[q] = __ldg(src + q0 + q);
            if (feat_bf16) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q0 + q >= nq) break;
                    uint4 v = buf[q];
                    if (fp16) {
                        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                        uint32_t o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            o[e] = tc::pack2(__uint_as_float(w[e] << 16), __uint_as_float(w[e] & 0xFFFF0000u), true);
                        v = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                    st_chunk(abuf, row, kb++, v.x, v.y, v.z, v.w);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    if (q0 + q >= nq) break;
                    const uint4 a = buf[q], b = buf[q + 1];
                    st_chunk(abuf, row, kb++, tc::pack2(__uint_as_float(a.x), __uint_as_float(a.y), fp16),
                             tc::pack2(__uint_as_float(a.z), __uint_as_float(a.w), fp16),
                             tc::pack2(__uint_as_float(b.x), __uint_as_float(b.y), fp16),
                             tc::pack2(__uint_as_float(b.z), __uint_as_float(b.w), fp16));
                }
            }
        }
        return;
    }
    int kb = F / 8;
    if (valid) {
        const float2 *rp = reinterpret_cast<const float2 *>(rays + 6 * ((int64_t)sm.ray - ray_begin));
        const float2 ra = __ldg(rp), rb = __ldg(rp + 1), rc = __ldg(rp + 2);
        const float o[3] = {ra.x, ra.y, rb.x};
        const float d[3] = {rb.y, rc.x, rc.y};
        float p1[3], p2[3];
        voxel_param_at(rparam, o, d, sm.tmid, sm.cell, depth, p1, p2);
        st_chunk(abuf, row, kb++, tc::pack2(d[0], d[1], fp16), tc::pack2(d[2], p1[0], fp16),
                 tc::pack2(p1[1], p1[2], fp16), tc::pack2(p2[0], p2[1], fp16));
        st_chunk(abuf, row, kb++, tc::pack2(p2[2], 0.f, fp16), 0u, 0u, 0u);
    }
    for (; kb < K0 / 8; ++kb) st_chunk(abuf, row, kb, 0u, 0u, 0u, 0u);
}

// ---------------------------------------------------------------- two-decoder
// Input rows of the two-decoder form (Sec. 4.1-4.2). Each leaf corner holds a
// feature vector (vertex table of the octree); psi(p; Z) is the trilinear
// interpolation of the hit voxel's eight corner features at p.
//  MODE 1 (F^T): [psi(x1; Z^T) | psi(x2; Z^T) | p~1 | p~2] with x1, x2 the
//    ray's entry and exit points of the voxel (slab test, t clipped at 0);
//    carries (t_in, t_out) to the output stage.
//  MODE 2 (F^C): [psi(x_s; Z^C) | p~1 | p~2] with x_s = o + t_s d,
//    t_s = eta t_in + (1 - eta) t_out from the F^T pass's (tau, eta, t_in,
//    t_out) in `prev`; carries (tau, t_s).
// Weights of the corners (slot a + 2b + 4c) of voxel `cell` at o + t d.
__device__ __forceinline__ void corner_weights(const float o[3], const float d[3], float t, const int cell[3],
                                               float n, float w[8]) {
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = fminf(fmaxf(fmaf(t, d[a], o[a]) * n - (float)cell[a], 0.f), 1.f);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        w[c] = ((c & 1) ? u[0] : 1.f - u[0]) * ((c & 2) ? u[1] : 1.f - u[1]) * ((c & 4) ? u[2] : 1.f - u[2]);
}

// d w_c / d p (c = a + 2b + 4c') for the corners of voxel `cell` at p = o + t d;
// zero along an axis where the position is clamped to the voxel.
__device__ __forceinline__ void corner_weight_grads(const float o[3], const float d[3], float t, const int cell[3],
                                                    float n, float g[8][3]) {
    float u[3];
    bool in[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float r = fmaf(t, d[a], o[a]) * n - (float)cell[a];
        in[a] = r > 0.f && r < 1.f;
        u[a] = fminf(fmaxf(r, 0.f), 1.f);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float f0 = (c & 1) ? u[0] : 1.f - u[0];
        const float f1 = (c & 2) ? u[1] : 1.f - u[1];
        const float f2 = (c & 4) ? u[2] : 1.f - u[2];
        g[c][0] = in[0] ? ((c & 1) ? n : -n) * f1 * f2 : 0.f;
        g[c][1] = in[1] ? ((c & 2) ? n : -n) * f0 * f2 : 0.f;
        g[c][2] = in[2] ? ((c & 4) ? n : -n) * f0 * f1 : 0.f;
    }
}

// Position of o + t d inside voxel `cell`, clamped to [0, 1]^3 (the
// trilinear coordinates behind corner_weights).
__device__ __forceinline__ void voxel_coords(const float o[3], const float d[3], float t, const int cell[3], float n,
                                             float u[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = fminf(fmaxf(fmaf(t, d[a], o[a]) * n - (float)cell[a], 0.f), 1.f);
}

// Weight of corner v (slot a + 2b + 4c) from the trilinear coordinates; the
// same products in the same order as corner_weights.
__device__ __forceinline__ float corner_weight(const float u[3], int v) {
    return ((v & 1) ? u[0] : 1.f - u[0]) * ((v & 2) ? u[1] : 1.f - u[1]) * ((v & 4) ? u[2] : 1.f - u[2]);
}

// The corner rows are gathered by the warp as a whole: in pass b the 32 lanes
// serve 32/G samples, G lanes per sample, and lane q of a group reads the
// 16-byte segments q, q + G, ... of each of the sample's eight corner rows, so
// a group reads G x 16 contiguous bytes of one vertex row per load instead of
// 32 lanes reading 16 bytes of 32 different rows (one L1 wavefront per lane).
// Eight loads (one per corner) are in flight per lane: more in flight per SM
// evicts from L1 the corner rows that neighbouring samples share, and runs
// slower. The sample's vertex ids and trilinear coordinates come from its
// owner lane by shuffle; per feature the corner sum runs v = 0..7 in the same
// order as a lane-per-sample loop would, so the result does not depend on the
// mapping. Lanes write their segment's 16-bit values straight into the
// sample's row of the A operand (the rows of one pass differ in row & 7, so
// the stores spread over the banks).
template <int MODE>
__device__ __forceinline__ void gather_corner_seg(const void *feats, int feat_bf16, int F, int nq, const int vs[8],
                                                  const float xa[8], const float xb[8], int seg, int fp16,
                                                  uint8_t *abuf, int r) {
    if (feat_bf16) {
        const uint4 *base = reinterpret_cast<const uint4 *>(feats);
        const int rq = F >> 3;  // 16-byte segments per row
        uint4 t[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) t[v] = __ldg(base + (int64_t)vs[v] * rq + seg);
        float acc_a[8], acc_b[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) acc_a[e] = acc_b[e] = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const uint32_t w[4] = {t[v].x, t[v].y, t[v].z, t[v].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float z0 = __uint_as_float(w[e] << 16), z1 = __uint_as_float(w[e] & 0xFFFF0000u);
                acc_a[2 * e] = fmaf(xa[v], z0, acc_a[2 * e]);
                acc_a[2 * e + 1] = fmaf(xa[v], z1, acc_a[2 * e + 1]);
                if (MODE == 1) {
                    acc_b[2 * e] = fmaf(xb[v], z0, acc_b[2 * e]);
                    acc_b[2 * e + 1] = fmaf(xb[v], z1, acc_b[2 * e + 1]);
                }
            }
        }
        st_chunk(abuf, r, seg, tc::pack2(acc_a[0], acc_a[1], fp16), tc::pack2(acc_a[2], acc_a[3], fp16),
                 tc::pack2(acc_a[4], acc_a[5], fp16), tc::pack2(acc_a[6], acc_a[7], fp16));
        if (MODE == 1)
            st_chunk(abuf, r, nq + seg, tc::pack2(acc_b[0], acc_b[1], fp16), tc::pack2(acc_b[2], acc_b[3], fp16),
                     tc::pack2(acc_b[4], acc_b[5], fp16), tc::pack2(acc_b[6], acc_b[7], fp16));
    } else {
        const float4 *base = reinterpret_cast<const float4 *>(feats);
        const int rq = F >> 2;
        float4 t[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) t[v] = __ldg(base + (int64_t)vs[v] * rq + seg);
        float acc_a[4], acc_b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc_a[e] = acc_b[e] = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const float z[4] = {t[v].x, t[v].y, t[v].z, t[v].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                acc_a[e] = fmaf(xa[v], z[e], acc_a[e]);
                if (MODE == 1) acc_b[e] = fmaf(xb[v], z[e], acc_b[e]);
            }
        }
        st_half_chunk(abuf, r, seg >> 1, seg & 1, tc::pack2(acc_a[0], acc_a[1], fp16),
                      tc::pack2(acc_a[2], acc_a[3], fp16));
        if (MODE == 1)
            st_half_chunk(abuf, r, nq + (seg >> 1), seg & 1, tc::pack2(acc_b[0], acc_b[1], fp16),
                          tc::pack2(acc_b[2], acc_b[3], fp16));
    }
}

template <int MODE>
__device__ __forceinline__ void build_input_two_decoder(const MlpDims &md, int K0, int depth,
                                                        const int32_t *__restrict__ leaf_vertices,
                                                        const void *feats, int feat_bf16,
                                                        const float *rays, int64_t ray_begin,
                                                        const Sample &sm, bool valid, float4 prev, int fp16,
                                                        uint8_t *abuf, int row, float &carry0, float &carry1) {
    const int nq = md.F / 8;
    float ua[3] = {0.f, 0.f, 0.f}, ub[3] = {0.f, 0.f, 0.f};
    int vid[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) vid[v] = 0;
    if (valid) {
        const float2 *rp = reinterpret_cast<const float2 *>(rays + 6 * ((int64_t)sm.ray - ray_begin));
        const float2 ra = __ldg(rp), rb = __ldg(rp + 1), rc = __ldg(rp + 2);
        const int4 *vp = reinterpret_cast<const int4 *>(leaf_vertices + 8 * (int64_t)sm.leaf);
        const int4 va = __ldg(vp), vb = __ldg(vp + 1);
        const float o[3] = {ra.x, ra.y, rb.x};
        const float d[3] = {rb.y, rc.x, rc.y};
        const int cell[3] = {(int)(sm.cell & 1023u), (int)((sm.cell >> 10) & 1023u), (int)((sm.cell >> 20) & 1023u)};
        const float n = (float)(1 << depth);
        const float h = ldexpf(1.0f, -depth);
        float ta, tb;
        if (MODE == 1) {
            float t0 = 0.f, t1 = INFINITY;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.f) continue;
                const float lo = ((float)cell[a] * h - o[a]) / d[a];
                const float hi = ((float)(cell[a] + 1) * h - o[a]) / d[a];
                t0 = fmaxf(t0, fminf(lo, hi));
                t1 = fminf(t1, fmaxf(lo, hi));
            }
            ta = t0;
            tb = t1;
            carry0 = t0;
            carry1 = t1;
        } else {
            const float ts = fmaf(prev.y, prev.z - prev.w, prev.w);  // eta t_in + (1 - eta) t_out
            ta = tb = ts;
            carry0 = prev.x;
            carry1 = ts;
        }
        voxel_coords(o, d, ta, cell, n, ua);
        if (MODE == 1) voxel_coords(o, d, tb, cell, n, ub);
        vid[0] = va.x; vid[1] = va.y; vid[2] = va.z; vid[3] = va.w;
        vid[4] = vb.x; vid[5] = vb.y; vid[6] = vb.z; vid[7] = vb.w;
        float p1[3], p2[3];
        sphere_param(o, d, sm.cell, depth, p1, p2);
        st_chunk(abuf, row, (MODE == 1 ? 2 : 1) * nq, tc::pack2(p1[0], p1[1], fp16), tc::pack2(p1[2], p2[0], fp16),
                 tc::pack2(p2[1], p2[2], fp16), 0u);
    }
    // ---- the owner's zero chunks (all of an empty row; after [p~1 | p~2] up to K0 otherwise): the
    // gathered feature chunks below are written by other lanes and never overlap them
    for (int kb = valid ? (MODE == 1 ? 2 : 1) * nq + 1 : 0; kb < K0 / 8; ++kb) st_chunk(abuf, row, kb, 0u, 0u, 0u, 0u);
    // ---- cooperative corner gather: G lanes per sample
    const int lane = threadIdx.x & 31;
    const int row0 = row - lane;                         // the warp's first row of the tile
    const int nseg = (md.F * (feat_bf16 ? 2 : 4)) >> 4;  // 16-byte segments of a vertex row
    const int G = nseg >= 5 ? 8 : (nseg >= 3 ? 4 : nseg);
    const int gsh = G == 8 ? 3 : (G == 4 ? 2 : (G == 2 ? 1 : 0));
    const int q = lane & (G - 1);
    const uint32_t full = 0xFFFFFFFFu;
    const int ok_self = valid ? 1 : 0;
#pragma unroll 1
    for (int b = 0; b < G; ++b) {
        const int src = (b << (5 - gsh)) + (lane >> gsh);  // sample (lane of the warp) served in this pass
        const int ok = __shfl_sync(full, ok_self, src);
        int vs[8];
        float u0[3], u1[3];
#pragma unroll
        for (int v = 0; v < 8; ++v) vs[v] = __shfl_sync(full, vid[v], src);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            u0[a] = __shfl_sync(full, ua[a], src);
            u1[a] = MODE == 1 ? __shfl_sync(full, ub[a], src) : 0.f;
        }
        if (!ok) continue;
        float xa[8], xb[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            xa[v] = corner_weight(u0, v);
            xb[v] = MODE == 1 ? corner_weight(u1, v) : 0.f;
        }
        for (int seg = q; seg < nseg; seg += G)
            gather_corner_seg<MODE>(feats, feat_bf16, md.F, nq, vs, xa, xb, seg, fp16, abuf, row0 + src);
    }
}

// The gather of a tile is latency-bound, so each warpgroup keeps the sample
// records of its next two tiles in registers and, one tile ahead, prefetches
// the next tile's feature rows and rays into L2 while the current tile runs
// through the tensor cores.
struct TilePrefetch {
    Sample cur, nxt;
    bool v_cur, v_nxt;
};

__device__ __forceinline__ bool load_record(const Sample *samples, int64_t sbase, int64_t tile0,
                                            int64_t tile, int64_t seg_end, int64_t S_sc, int row,
                                            Sample &r) {
    const int64_t sl = (tile - tile0) * kTcTile + row;
    const bool v = tile < seg_end && sl < S_sc;
    if (v) r = samples[sbase + sl];
    return v;
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_gather(const Sample &r, const void *feats, int feat_bf16,
                                                int F, const float *rays, int64_t ray_begin) {
    const size_t row_bytes = (size_t)F * (feat_bf16 ? 2 : 4);
    const char *f = reinterpret_cast<const char *>(feats) + (size_t)r.leaf * row_bytes;
    for (size_t b = 0; b < row_bytes; b += 128) prefetch_l2(f + b);
    const float *ray = rays + 6 * ((int64_t)r.ray - ray_begin);
    prefetch_l2(ray);
    prefetch_l2(ray + 5);
}

// The two-decoder passes: the sample's ray, its leaf's eight vertex ids and
// the eight corner rows into L2. The ids are loaded (the rows' addresses
// depend on them), so callers issue this where the thread would wait anyway.
__device__ __forceinline__ void prefetch_corners(const Sample &r, const int32_t *__restrict__ leaf_vertices,
                                                 const void *feats, int feat_bf16, int F, const float *rays,
                                                 int64_t ray_begin) {
    const float *ray = rays + 6 * ((int64_t)r.ray - ray_begin);
    prefetch_l2(ray);
    prefetch_l2(ray + 5);
    const int4 *vp = reinterpret_cast<const int4 *>(leaf_vertices + 8 * (int64_t)r.leaf);
    const int4 va = __ldg(vp), vb = __ldg(vp + 1);
    const int vid[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
    const size_t row_bytes = (size_t)F * (feat_bf16 ? 2 : 4);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const char *f = reinterpret_cast<const char *>(feats) + (size_t)vid[v] * row_bytes;
        for (size_t b = 0; b < row_bytes; b += 128) prefetch_l2(f + b);
    }
}

// ReLU, 16-bit packing and A-operand store of 16 accumulator columns (two
// 8-column chunks starting at chunk kb).
__device__ __forceinline__ void epi_chunk16(const uint32_t (&v)[16], uint8_t *abuf, int row, int kb, int fp16) {
    uint32_t p[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) p[e] = tc::relu_pack2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]), fp16);
    st_chunk(abuf, row, kb, p[0], p[1], p[2], p[3]);
    st_chunk(abuf, row, kb + 1, p[4], p[5], p[6], p[7]);
}

// EPI = hidden-layer epilogue form: 1 loads 32 TMEM columns per wait (registers
// low enough for 4 warpgroups); 2 loads 64 per wait (at most 3 warpgroups);
// 3 loads 16 columns at a time with the next load in flight while a chunk is
// packed.
template <int H, int EPI, int MODE>
__global__ void __launch_bounds__(EPI == 2 || MODE == 1 ? 384 : 512, 1)
    mlp_forward_tc_kernel(const __grid_constant__ SceneTable T, const TcFwdParams P) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t s_mbar[5];  // [0..3] per warpgroup, [4] weight load
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ TileMap s_map;

    const int tid = threadIdx.x;
    const int wg = tid >> 7;        // warpgroup
    const int row = tid & 127;      // sample row within the tile = TMEM lane
    const int warp = tid >> 5;
    const uint32_t ncols = P.n_wg <= 2 ? 256u : 512u;
    uint8_t *wimg = smem;
    uint8_t *abuf = smem + P.wbytes + wg * P.abuf_bytes;
    const float *bias = reinterpret_cast<const float *>(wimg + P.lay.bias_off);

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) tc::mbar_init(tc::smem_u32(&s_mbar[i]), 1);
        tc::mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&s_tmem), ncols);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tile_map_build(T, P.counter, s_map);
    tc::fence_after_sync();
    const uint32_t tmem_base = s_tmem;
    const uint32_t tmem_wg = tmem_base + (uint32_t)(wg * 128);            // column base
    const uint32_t tmem_row = tmem_wg + ((uint32_t)((warp & 3) * 32) << 16);  // lane base
    const uint32_t mbar = tc::smem_u32(&s_mbar[wg]);
    const uint32_t abuf_s = tc::smem_u32(abuf);
    const uint32_t wimg_s = tc::smem_u32(wimg);
    const int bf16 = P.fp16 ? 0 : 1;
    uint32_t phase = 0, wphase = 0;

    // this CTA's contiguous range of the global tile list
    const int64_t n_tiles = s_map.tile0[T.n];
    const int64_t lo = n_tiles * blockIdx.x / gridDim.x;
    const int64_t hi = n_tiles * (blockIdx.x + 1) / gridDim.x;
    int sc = 0;
    while (sc + 1 < T.n && s_map.tile0[sc + 1] <= lo) ++sc;
    for (int64_t seg = lo; seg < hi; ++sc) {
        const int64_t seg_end = min(hi, s_map.tile0[sc + 1]);
        if (seg_end <= seg) continue;
        const SceneDev &SD = T.s[sc];
        // resident weights of this scene: bulk copies into shared memory
        __syncthreads();
        if (s_abort) break;  // uniform: read after the barrier
        if (tid == 0) {
            const uint32_t mb = tc::smem_u32(&s_mbar[4]);
            const uint8_t *img = P.images + sc * P.image_stride;
            tc::mbar_expect_tx(mb, P.wbytes);
            for (uint32_t off = 0; off < P.wbytes; off += 32768u)
                tc::bulk_g2s(tc::smem_u32(wimg + off), img + off, min(32768u, P.wbytes - off), mb);
        }
        if (!tc::mbar_wait(tc::smem_u32(&s_mbar[4]), wphase)) {
            raise_status(SVLF_DEV_WAIT_TIMEOUT);
            atomicExch(&s_abort, 1);
        }
        wphase ^= 1u;
        __syncthreads();
        tc::fence_after_sync();
        if (s_abort) break;
        const int64_t S_sc = s_map.S[sc];
        const int64_t sbase = SD.ray_begin * T.K;  // the scene's first sample slot
        const int64_t tile0 = s_map.tile0[sc];
        const int depth = SD.tree.depth;
        bool aborted = false;
        TilePrefetch pf;
        pf.v_cur = load_record(P.samples, sbase, tile0, seg + wg, seg_end, S_sc, row, pf.cur);
        pf.v_nxt = load_record(P.samples, sbase, tile0, seg + wg + P.n_wg, seg_end, S_sc, row, pf.nxt);
        for (int64_t tile = seg + wg; !aborted && tile < seg_end; tile += P.n_wg) {
            const int64_t sl = (tile - tile0) * kTcTile + row;  // sample within the scene
            const int64_t s = sbase + sl;
            const Sample rec = pf.cur;
            const bool valid = pf.v_cur;
            if (MODE == 0 && pf.v_nxt) prefetch_gather(pf.nxt, SD.feats, P.feat_bf16, P.md.F, SD.rays, SD.ray_begin);
            pf.cur = pf.nxt;
            pf.v_cur = pf.v_nxt;
            pf.v_nxt = load_record(P.samples, sbase, tile0, tile + 2 * P.n_wg, seg_end, S_sc, row, pf.nxt);
            // ---- network input row -> A operand (K0 columns)
            float carry0 = 0.f, carry1 = 0.f;
            if (MODE == 0) {
                build_input_chunks(P.md, P.lay.K0, depth, T.rparam, SD.feats, P.feat_bf16, SD.rays, SD.ray_begin,
                                   rec, valid, P.fp16, abuf, row, nullptr);
            } else {
                const float4 prev = (MODE == 2 && valid) ? P.aux[s] : make_float4(0.f, 0.f, 0.f, 0.f);
                build_input_two_decoder<MODE>(P.md, P.lay.K0, depth, SD.tree.leaf_vertices, SD.feats, P.feat_bf16,
                                              SD.rays, SD.ray_begin, rec, valid, prev, P.fp16, abuf, row, carry0,
                                              carry1);
            }
            for (int l = 0; l < P.lay.n_layers; ++l) {
                const int N = P.lay.w_rows[l];
                const int Kl = P.lay.w_cols[l];
                const bool hidden = l + 1 < P.lay.n_layers;
                if (hidden && !P.bias_mma) {
                    // the accumulator starts at the bias: the MMAs add onto it in float32
                    const uint4 *b4 = reinterpret_cast<const uint4 *>(bias + P.lay.bias_l[l]);
#pragma unroll 1
                    for (int c = 0; c < H / 32; ++c) {
                        uint32_t v[32];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const uint4 t = b4[c * 8 + q];
                            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
                        }
                        tc::tmem_st32(tmem_row + (uint32_t)(c * 32), v);
                    }
                    tc::tmem_wait_st();
                }
                // A operand written by all threads -> visible to the tensor core
                tc::fence_async_smem();
                tc::fence_before_sync();
                tc::wg_sync(wg);
                if (row == 0) {
                    tc::fence_after_sync();
                    const uint32_t idesc = tc::idesc_f16(kTcTile, N, bf16, 0, 0);
                    const uint32_t b_base = wimg_s + P.lay.w_off[l];
                    if (hidden && P.bias_mma) {
                        // the accumulator starts at the bias (ones x bias pieces); the layer's MMAs add onto it
                        const uint64_t da = tc::sdesc(wimg_s + P.lay.ones_off, kTcTile * 16, 128);
                        const uint64_t db = tc::sdesc(wimg_s + P.lay.bias_b_off[l], N * 16, 128);
                        tc::mma_f16(tmem_wg, da, db, idesc, 0u);
                    }
                    tc::mma_f16_k<kMaxKSteps>(tmem_wg, tc::sdesc(abuf_s, kTcTile * 16, 128), (2 * kTcTile * 16) >> 4,
                                              tc::sdesc(b_base, N * 16, 128), (2 * N * 16) >> 4, idesc, Kl / 16,
                                              hidden);
                    tc::mma_commit(mbar);
                }
                // two-decoder passes: while the first layer runs, the next tile's corner rows go to L2
                // (its gather then waits on L2, not HBM)
                if (MODE != 0 && l == 0 && pf.v_cur)
                    prefetch_corners(pf.cur, SD.tree.leaf_vertices, SD.feats, P.feat_bf16, P.md.F, SD.rays,
                                     SD.ray_begin);
                const bool timeout = !tc::mbar_wait(mbar, phase);
                phase ^= 1u;
                if (tc::wg_sync_or(wg, timeout)) {
                    if (row == 0) {
                        raise_status(SVLF_DEV_WAIT_TIMEOUT);
                        atomicExch(&s_abort, 1);
                    }
                    aborted = true;
                    break;
                }
                tc::fence_after_sync();
                const float *b = bias + P.lay.bias_l[l];
                if (l + 1 < P.lay.n_layers) {
                    // hidden layer epilogue: ReLU of (bias + W x) -> 16-bit A operand of the next layer
                    if (EPI == 3) {
                        // 16-column chunks, the next chunk's TMEM load in flight while one is packed
                        uint32_t va[16], vb[16];
                        tc::tmem_ld16_async(tmem_row, va);
                        tc::tmem_wait_ld16(va);
#pragma unroll
                        for (int c = 0; c < H / 16; c += 2) {
                            tc::tmem_ld16_async(tmem_row + (uint32_t)((c + 1) * 16), vb);
                            epi_chunk16(va, abuf, row, 2 * c, P.fp16);
                            tc::tmem_wait_ld16(vb);
                            if (c + 2 < H / 16) tc::tmem_ld16_async(tmem_row + (uint32_t)((c + 2) * 16), va);
                            epi_chunk16(vb, abuf, row, 2 * c + 2, P.fp16);
                            if (c + 2 < H / 16) tc::tmem_wait_ld16(va);
                        }
                    }
#pragma unroll
                    for (int c0 = 0; EPI != 3 && c0 < H / 32; c0 += EPI) {
                        uint32_t v[EPI == 2 ? 2 : 1][32];
                        if (EPI == 2)
                            tc::tmem_ld64_wait(tmem_row + (uint32_t)(c0 * 32), reinterpret_cast<uint32_t(&)[64]>(v));
                        else
                            tc::tmem_ld32_wait(tmem_row + (uint32_t)(c0 * 32), reinterpret_cast<uint32_t(&)[32]>(v));
#pragma unroll
                        for (int u = 0; u < (EPI == 2 ? 2 : 1); ++u) {
                            const int c = c0 + u;
                            uint32_t p[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e)
                                p[e] = tc::relu_pack2(__uint_as_float(v[u][2 * e]), __uint_as_float(v[u][2 * e + 1]),
                                                      P.fp16);
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                st_chunk(abuf, row, c * 4 + q, p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                        }
                    }
                } else {
                    uint32_t v[4];
                    tc::tmem_ld4_wait(tmem_row, v);
                    if (sl < S_sc) {
                        const float o0 = __uint_as_float(v[0]) + b[0], o1 = __uint_as_float(v[1]) + b[1];
                        const float o2 = __uint_as_float(v[2]) + b[2], o3 = __uint_as_float(v[3]) + b[3];
                        if (MODE == 0) {
                            P.outputs[s] = output_activation(o0, o1, o2, o3);
                        } else if (MODE == 1) {  // (tau, eta, t_in, t_out) for the colour pass
                            P.aux[s] = make_float4(fmaxf(o0, 0.f), sigmoidf_(o1), carry0, carry1);
                        } else {                 // (colour, tau); the sample's depth parameter becomes t_s
                            P.outputs[s] = make_float4(sigmoidf_(o0), sigmoidf_(o1), sigmoidf_(o2), carry0);
                            P.samples[s].tmid = carry1;
                        }
                    }
                }
            }
            // all TMEM reads of this tile are done before the next tile's MMAs
            tc::fence_before_sync();
        }
        seg = seg_end;
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, ncols);
    }
}

// Warpgroups that fit next to `wbytes` of resident image (0 if none does).
static int tc_forward_wgs(uint32_t wbytes, uint32_t abuf, size_t &smem) {
    const size_t limit = 227 * 1024 - sizeof(TileMap) - 256;  // static shared memory comes off the top
    for (int n_wg = 4; n_wg >= 1; --n_wg) {
        smem = wbytes + (size_t)n_wg * abuf + 128;  // + alignment slack
        if (smem <= limit) return n_wg;
    }
    return 0;
}

// Launch shape: the biases go through the MMA unless the image's forward tail
// would cost a warpgroup (or the whole launch), in which case they are stored
// into TMEM and the tail stays in global memory.
static int tc_forward_config(const MlpDims &md, const TcLayout &lay, TcFwdParams &P, size_t &smem) {
    const int kmax = lay.K0 > kHp ? lay.K0 : kHp;
    P.abuf_bytes = (uint32_t)(kTcTile * kmax * 2);
    size_t smem_mma, smem_st;
    const int wg_mma = tc_forward_wgs(lay.fwd_bytes, P.abuf_bytes, smem_mma);
    const int wg_st = tc_forward_wgs(lay.bytes, P.abuf_bytes, smem_st);
    if (wg_st < 1) return SVLF_ERR_UNSUPPORTED;
    P.bias_mma = wg_mma == wg_st ? 1 : 0;
    P.n_wg = P.bias_mma ? wg_mma : wg_st;
    P.wbytes = P.bias_mma ? lay.fwd_bytes : lay.bytes;
    smem = P.bias_mma ? smem_mma : smem_st;
    if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM: it owns all TMEM columns it asks for
    return SVLF_OK;
}

template <int H, int EPI, int MODE>
static int fwd_tc(const SceneTable &T, const TcFwdParams &P0, const MlpDims &md, const TcLayout &lay,
                  cudaStream_t s, int n_wg_override) {
    TcFwdParams P = P0;
    size_t smem;
    int rc = tc_forward_config(md, lay, P, smem);
    if (rc) return rc;
    if (n_wg_override > 0 && n_wg_override < P.n_wg) P.n_wg = n_wg_override;
    if ((EPI == 2 || MODE == 1) && P.n_wg > 3) P.n_wg = 3;
    if (cudaFuncSetAttribute(mlp_forward_tc_kernel<H, EPI, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    prof_begin(MODE == 0 ? "mlp_forward_tc" : MODE == 1 ? "two_decoder_ft_tc" : "two_decoder_fc_tc", s);
    mlp_forward_tc_kernel<H, EPI, MODE><<<num_sms(), 128 * P.n_wg, smem, s>>>(T, P);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

int launch_mlp_forward_tc(const MlpDims &md, int precision, int fb, const SceneTable &T,
                          const Workspace &ws, cudaStream_t s, int mode, float4 *aux) {
    if (!tc_supported(md)) return SVLF_ERR_UNSUPPORTED;
    TcFwdParams P;
    memset(&P, 0, sizeof(P));
    P.md = md;
    P.lay = tc_layout(md);
    P.fp16 = precision == SVLF_FP16;
    P.feat_bf16 = fb;
    P.images = (const uint8_t *)ws.packed_w;
    P.image_stride = ws.packed_stride;
    P.samples = ws.samples;
    P.counter = ws.counter;
    P.outputs = ws.outputs;
    P.aux = aux;
    const svlf_tuning &tu = tuning();
    if (mode == 1) return fwd_tc<kHp, 1, 1>(T, P, md, P.lay, s, tu.mlp_warpgroups);
    if (mode == 2) return fwd_tc<kHp, 1, 2>(T, P, md, P.lay, s, tu.mlp_warpgroups);
    if (tu.mlp_epilogue_batch == 2) return fwd_tc<kHp, 2, 0>(T, P, md, P.lay, s, tu.mlp_warpgroups);
    if (tu.mlp_epilogue_batch == 3) return fwd_tc<kHp, 3, 0>(T, P, md, P.lay, s, tu.mlp_warpgroups);
    return fwd_tc<kHp, 1, 0>(T, P, md, P.lay, s, tu.mlp_warpgroups);
}

// ---------------------------------------------------------------- backward
// Backward kernel (persistent, one warpgroup per CTA, one CTA per SM). Per
// tile of 128 samples (thread t = sample t = TMEM lane t):
//  1. network input X_0 and dL/d(output) G_out (from the compositing
//     backward) are written as 16-bit A operands;
//  2. the forward is recomputed layer by layer, keeping every layer's input
//     X_l in shared memory (activations are recomputed, never stored in HBM);
//  3. from the output down, per layer one commit group of MMAs:
//       dW_l  += G_{l+1}^T X_l     (M = out features, N = in features, K = 128
//                                   samples; both operands read MN-major)
//       db_l  += G_{l+1}^T 1       (the same with a block of ones, N = 16)
//       G_l    = G_{l+1} W_l       (M = samples, N = in features, K = out;
//                                   W_l read MN-major from the forward image)
//     and the epilogue masks G_l with the ReLU pattern X_l > 0 in place of X_l;
//     for layer 0 only the first F columns of G_0 (dL/dz) are formed and
//     scattered to the feature gradient, one float4 atomic group per distinct
//     leaf in a warp (warp-aggregated).
//  dW and db stay in TMEM across all tiles of the CTA and are added to the
//  global gradient once at the end.
//  With float16 operands the deltas are scaled by a power of two chosen from
//  the largest |dL/d(output)| of the launch (so that they stay clear of the
//  float16 underflow range), and every gradient is unscaled in float32 before
//  it leaves the kernel. bfloat16 has float32's exponent range and is not
//  scaled.
struct TcBwdParams {
    MlpDims md;
    TcLayout lay;
    int fp16, feat_bf16;
    int want_feat, want_params;  // which gradients to form
    int l_min, l_top, with_out;  // this pass: dW of hidden layers [l_min, l_top] (+ output layer)
    const uint8_t *images;
    size_t image_stride;
    const Sample *samples;
    const unsigned int *counter;
    const float4 *dout;
    // two-decoder form: per-sample (tau, eta, t_in, t_out) from the render, replaced by
    // the colour pass's (dL/dtau_pre, dL/deta_pre) for the optical-thickness pass;
    // dL/d(depth parameter) per sample; the running max |dL/d(output)| (fp16 scaling)
    float4 *aux;
    const float *w_dD;
    const float *deta;   // direct dL/d(eta) per sample (a loss term on eta), or null
    unsigned int *gmax;
    uint32_t x_off[kMaxLayers];  // X_l buffers (byte offsets after the weight image)
    uint32_t gout_off, ones_off;
    uint32_t col_dwout, col_dw[kMaxLayers], col_db[kMaxLayers], tmem_cols;
    // Streamed weights (networks whose full image and activations do not fit
    // together): only the image tail from w_off[nh] (output layer + biases) is
    // resident at offset 0; hidden W_l is loaded into slot l % 2 when needed.
    int stream;
    uint32_t res_bytes;    // bytes of the image resident from img0 (whole image, or its tail when streamed)
    int bias_mma;          // the image's forward tail is resident: recompute biases enter through the MMA
    uint32_t slot_off[2];  // byte offsets of the two weight slots
};

// Shared-memory and TMEM plan of one backward pass (P.l_min, P.l_top,
// P.with_out set by the caller). TMEM holds the work accumulator and the dW /
// db accumulators of the pass's layers; networks whose accumulators do not
// fit in 512 columns are split into several passes over the same tiles.
static uint32_t tc_bwd_cols(const MlpDims &md, const TcLayout &lay, int l_min, int l_top,
                            int with_out) {
    uint32_t col = kHp;
    for (int l = l_min; l <= l_top; ++l) col += (l == 0 ? lay.K0 : kHp) + 16;
    if (with_out) col += kTcOutN;
    return col;
}

static bool tc_bwd_plan(const MlpDims &md, TcBwdParams &P, size_t &smem) {
    const TcLayout &lay = P.lay;
    // activations, deltas and ones take this many bytes after the weights
    const uint32_t act = (uint32_t)(kTcTile * lay.K0 * 2 + md.nh * kTcTile * kHp * 2 +
                                    2 * kTcTile * kTcOutN * 2);
    const size_t limit = 227 * 1024 - 2048;
    // stream the hidden layers' weights through two slots when the image and the
    // activations do not fit together; keep the forward tail (bias MMA operands)
    // resident when it fits as well
    P.stream = (size_t)lay.bytes + act + 128 > limit ? 1 : 0;
    const uint32_t img0 = P.stream ? lay.w_off[md.nh] : 0u;
    const uint32_t slot = (uint32_t)(kHp * (lay.K0 > kHp ? lay.K0 : kHp) * 2);
    const uint32_t slots = P.stream ? 2 * slot : 0u;
    P.bias_mma = (size_t)(((lay.fwd_bytes - img0) + 127) & ~127u) + slots + act + 128 <= limit ? 1 : 0;
    P.res_bytes = (P.bias_mma ? lay.fwd_bytes : lay.bytes) - img0;
    uint32_t off = (P.res_bytes + 127) & ~127u;
    if (P.stream) {
        P.slot_off[0] = off;
        P.slot_off[1] = off + slot;
        off += 2 * slot;
    }
    P.x_off[0] = off;
    off += kTcTile * lay.K0 * 2;
    for (int l = 1; l <= md.nh; ++l) {
        P.x_off[l] = off;
        off += kTcTile * kHp * 2;
    }
    P.gout_off = off;
    off += kTcTile * kTcOutN * 2;
    P.ones_off = off;
    off += kTcOutN * kTcTile * 2;
    smem = off + 128;
    // TMEM columns: [0, 128) work accumulator, then the 128-wide dW_l (l >= 1)
    // at multiples of 128, dW_0 (K0 wide), and the 16-wide dW_out^T and db_l.
    uint32_t col = kHp;
    for (int l = P.l_min; l <= P.l_top; ++l) {
        if (l == 0) continue;
        P.col_dw[l] = col;
        col += kHp;
    }
    if (P.l_min == 0) {
        P.col_dw[0] = col;
        col += lay.K0;
    }
    if (P.with_out) {
        P.col_dwout = col;
        col += kTcOutN;
    }
    for (int l = P.l_min; l <= P.l_top; ++l) {
        P.col_db[l] = col;
        col += 16;
    }
    if (col > 512 || smem > 227 * 1024 - 2048) return false;
    uint32_t n = 32;
    while (n < col) n <<= 1;
    P.tmem_cols = n;
    return true;
}

// Layer-0 epilogue of the two-decoder backward: dL/dpsi (fp32 in TMEM columns
// [0, F) and, for F^T, [F, 2F) for the exit point) spread to the hit voxel's
// corner features by their trilinear weights (16-byte float reductions). The
// colour pass (MODE 2) also carries dL/dpsi through the surface point:
// dL/dx_s = sum_c (Z^C_c . dL/dpsi) grad w_c(x_s), dL/dt_s = w dL/dD + dL/dx_s . d,
// dL/deta = dL/dt_s (t_in - t_out), and leaves (dL/dtau_pre, dL/deta_pre) in
// aux for the optical-thickness pass.
//
// The corner rows are updated by the warp as a whole, as the forward gathers
// them: per block of 32 columns each lane stages its sample's dL/dpsi (and
// dL/dpsi2) in `stage` (a free 32 KB activation buffer: 128 rows of 64
// floats, 16-byte segment q of row r at position q ^ (r & 7) so that both the
// owners' writes and the groups' reads spread over the banks), then in pass b
// the 8 lanes of a group serve one sample, lane q reducing segment q into the
// eight corner rows: 128 contiguous bytes of a row per group and instruction.
// Vertex ids and trilinear coordinates come from the owner by shuffle; the
// weights are recomputed with the owner's products. MODE 2's Z^C . dL/dpsi per
// corner is summed over the group's lanes (a fixed tree order) into the spare
// half of the sample's stage row, where its owner reads it. Every lane runs the
// TMEM loads; rows without a sample skip the rest.
template <int MODE>
__device__ __forceinline__ void two_decoder_dz(const MlpDims &md, const SceneDev &SD, const Sample &rec, bool valid,
                                               int64_t s, float carry0, float carry1, float4 prev,
                                               float *__restrict__ dZ, uint32_t trow, float ginv,
                                               const TcBwdParams &P, float *stage) {
    const int F = md.F;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
    int cell[3] = {0, 0, 0};
    int vid[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float ua[3] = {0.f, 0.f, 0.f}, ub[3] = {0.f, 0.f, 0.f};
    const float n = (float)(1 << SD.tree.depth);
    if (valid) {
        const float2 *rp = reinterpret_cast<const float2 *>(SD.rays + 6 * ((int64_t)rec.ray - SD.ray_begin));
        const float2 ra = __ldg(rp), rb = __ldg(rp + 1), rc = __ldg(rp + 2);
        o[0] = ra.x; o[1] = ra.y; o[2] = rb.x;
        d[0] = rb.y; d[1] = rc.x; d[2] = rc.y;
        cell[0] = (int)(rec.cell & 1023u);
        cell[1] = (int)((rec.cell >> 10) & 1023u);
        cell[2] = (int)((rec.cell >> 20) & 1023u);
        const int4 *vp = reinterpret_cast<const int4 *>(SD.tree.leaf_vertices + 8 * (int64_t)rec.leaf);
        const int4 va = __ldg(vp), vb = __ldg(vp + 1);
        vid[0] = va.x; vid[1] = va.y; vid[2] = va.z; vid[3] = va.w;
        vid[4] = vb.x; vid[5] = vb.y; vid[6] = vb.z; vid[7] = vb.w;
        if (MODE == 1) {  // carry = (t_in, t_out)
            voxel_coords(o, d, carry0, cell, n, ua);
            voxel_coords(o, d, carry1, cell, n, ub);
        } else {          // carry = (tau, t_s)
            voxel_coords(o, d, carry1, cell, n, ua);
        }
    }
    const int lane = threadIdx.x & 31;
    const int row = threadIdx.x;        // this lane's sample row (the backward runs one warpgroup)
    const int row0 = row - lane;
    const int q = lane & 7;             // the group lane's 16-byte segment of a 32-column block
    const uint32_t full = 0xFFFFFFFFu;
    const int ok_self = valid ? 1 : 0;
    float *my = stage + row * 64;
    for (int c0 = 0; c0 < F; c0 += 32) {
        // ---- the owner stages its columns c0..c0+31 (those below F)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + 16 * h;
            if (c >= F) break;
            uint32_t a[16], b[16];
            if (MODE == 1)
                tc::tmem_ld16x2_wait(trow + (uint32_t)c, trow + (uint32_t)(F + c), a, b);
            else
                tc::tmem_ld16_wait(trow + (uint32_t)c, a);
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int pos = ((4 * h + j) ^ (row & 7)) * 4;
                *reinterpret_cast<float4 *>(my + pos) =
                    make_float4(__uint_as_float(a[4 * j]), __uint_as_float(a[4 * j + 1]),
                                __uint_as_float(a[4 * j + 2]), __uint_as_float(a[4 * j + 3]));
                if (MODE == 1)
                    *reinterpret_cast<float4 *>(my + 32 + pos) =
                        make_float4(__uint_as_float(b[4 * j]), __uint_as_float(b[4 * j + 1]),
                                    __uint_as_float(b[4 * j + 2]), __uint_as_float(b[4 * j + 3]));
            }
        }
        __syncwarp();
        // ---- 8 passes: 4 samples per pass, 8 lanes per sample
#pragma unroll 1
        for (int pb = 0; pb < 8; ++pb) {
            const int src = 4 * pb + (lane >> 3);
            const int ok = __shfl_sync(full, ok_self, src);
            int vs[8];
            float u0[3], u1[3];
#pragma unroll
            for (int v = 0; v < 8; ++v) vs[v] = __shfl_sync(full, vid[v], src);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                u0[k] = __shfl_sync(full, ua[k], src);
                u1[k] = MODE == 1 ? __shfl_sync(full, ub[k], src) : 0.f;
            }
            const bool act = ok && c0 + 4 * q < F;
            const float *srow = stage + (row0 + src) * 64;
            const int pos = (q ^ ((row0 + src) & 7)) * 4;
            float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
            if (act) {
                ga = *reinterpret_cast<const float4 *>(srow + pos);
                if (MODE == 1) gb = *reinterpret_cast<const float4 *>(srow + 32 + pos);
            }
            // MODE 2: the eight corner segments of Z^C are loaded before the first reduction
            // (a reduction orders the memory accesses around it)
            float4 zc[8];
            if (MODE == 2 && act) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    if (P.feat_bf16) {
                        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(
                            reinterpret_cast<const __nv_bfloat16 *>(SD.feats) + (int64_t)vs[v] * F + c0 + 4 * q));
                        zc[v] = make_float4(__uint_as_float(t.x << 16), __uint_as_float(t.x & 0xFFFF0000u),
                                            __uint_as_float(t.y << 16), __uint_as_float(t.y & 0xFFFF0000u));
                    } else {
                        zc[v] = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(SD.feats) +
                                                                        (int64_t)vs[v] * F + c0 + 4 * q));
                    }
                }
            }
            float zp[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                zp[v] = 0.f;
                if (!act) continue;
                const float wa = corner_weight(u0, v);
                if (MODE == 2) {
                    const float z[4] = {zc[v].x, zc[v].y, zc[v].z, zc[v].w};
                    zp[v] = fmaf(z[0], ga.x * ginv, zp[v]);
                    zp[v] = fmaf(z[1], ga.y * ginv, zp[v]);
                    zp[v] = fmaf(z[2], ga.z * ginv, zp[v]);
                    zp[v] = fmaf(z[3], ga.w * ginv, zp[v]);
                }
                if (dZ) {
                    float g[4];
                    const float gav[4] = {ga.x, ga.y, ga.z, ga.w};
                    const float gbv[4] = {gb.x, gb.y, gb.z, gb.w};
                    const float wb = MODE == 1 ? corner_weight(u1, v) : 0.f;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float gv = wa * gav[e];
                        if (MODE == 1) gv = fmaf(wb, gbv[e], gv);
                        g[e] = gv * ginv;
                    }
                    red_add_f4(reinterpret_cast<float4 *>(dZ + (int64_t)vs[v] * F + c0 + 4 * q), g[0], g[1], g[2],
                               g[3]);
                }
            }
            if (MODE == 2) {
                // the group's sum per corner (lanes of inactive segments add 0), kept in the
                // spare half of the sample's stage row across 32-column blocks
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    zp[v] += __shfl_xor_sync(full, zp[v], 1);
                    zp[v] += __shfl_xor_sync(full, zp[v], 2);
                    zp[v] += __shfl_xor_sync(full, zp[v], 4);
                }
                if (ok && q == 0) {
                    float *zs = stage + (row0 + src) * 64 + 32;
#pragma unroll
                    for (int v = 0; v < 8; ++v) zs[v] = c0 == 0 ? zp[v] : zs[v] + zp[v];
                }
            }
        }
        __syncwarp();
    }
    if (MODE == 2 && valid) {
        float gw[8][3];
        corner_weight_grads(o, d, carry1, cell, n, gw);
        const float *zs = my + 32;
        float dx[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
            for (int a = 0; a < 3; ++a) dx[a] = fmaf(zs[v], gw[v][a], dx[a]);
        const float dts = P.w_dD[s] + dx[0] * d[0] + dx[1] * d[1] + dx[2] * d[2];
        const float eta = prev.y;
        const float deta = fmaf(dts, prev.z - prev.w, P.deta ? P.deta[s] : 0.f);
        const float geta = deta * eta * (1.f - eta);
        P.aux[s] = make_float4(P.dout[s].w, geta, 0.f, 0.f);
        if (geta != 0.f) atomicMax(P.gmax, __float_as_uint(fabsf(geta)));
    }
}

__device__ __forceinline__ void mma_seq(uint32_t tmem_d, uint32_t a_base, uint32_t a_kstep,
                                        uint32_t a_lbo, uint32_t a_sbo, uint32_t b_base,
                                        uint32_t b_kstep, uint32_t b_lbo, uint32_t b_sbo, int K,
                                        uint32_t idesc, bool accumulate) {
    tc::mma_f16_k<kMaxKSteps, true>(tmem_d, tc::sdesc(a_base, a_lbo, a_sbo), a_kstep >> 4,
                                    tc::sdesc(b_base, b_lbo, b_sbo), b_kstep >> 4, idesc, K / 16, accumulate);
}

// NWG = 2 (MODE 0 with resident weights): two warpgroups share each tile.
// Warpgroup `half` builds its part of the input row (build_input_chunks_half)
// and takes columns [64 half, 64 half + 64) of every epilogue and of the
// gradient flush, and its half of the feature-gradient columns; half 0 writes
// G_out, sums the output bias gradient and issues the MMAs. TMEM, shared
// memory and the MMAs are those of NWG = 1: the second warpgroup only adds
// warps to cover the epilogues' latencies (one warpgroup leaves one warp per
// scheduler).
template <int MODE, int NWG = 1>
__global__ void __launch_bounds__(128 * NWG, 1) mlp_backward_tc_kernel(const __grid_constant__ SceneTable T,
                                                                       const TcBwdParams P) {
    static_assert(NWG == 1 || (NWG == 2 && MODE == 0), "two warpgroups: MODE 0 only");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t s_mbar[2];  // [0] MMA commits, [1] weight load
    __shared__ uint32_t s_tmem;
    __shared__ float s_dbout[4];
    __shared__ TileMap s_map;

    const int row = threadIdx.x & 127;  // sample within the tile = TMEM lane
    const int warp = row >> 5, lane = row & 31;  // warp = the TMEM lane quarter it may access
    const int half = NWG == 2 ? (int)(threadIdx.x >> 7) : 0;
    const bool lead = threadIdx.x == 0;  // initialises, issues the MMAs and the bulk copies
    // barrier over the CTA returning the OR of `pred`
    auto sync_or = [&](bool pred) -> bool {
        return NWG == 1 ? tc::wg_sync_or(0, pred) : __syncthreads_or(pred) != 0;
    };
    // 32-column chunks of the 128-wide accumulator this warpgroup handles
    const int c32_lo = half * (kHp / 32) / NWG, c32_hi = (half + 1) * (kHp / 32) / NWG;
    const MlpDims &md = P.md;
    const TcLayout &lay = P.lay;
    uint8_t *wimg = smem;
    // image offset of what sits at shared offset 0 (the whole image, or its tail)
    const uint32_t img0 = P.stream ? lay.w_off[md.nh] : 0u;
    const float *bias = reinterpret_cast<const float *>(wimg + lay.bias_off - img0);
    const uint32_t s_base = tc::smem_u32(smem);
    __shared__ __align__(8) uint64_t s_wslot[2];  // streamed weight slots

    if (lead) {
        tc::mbar_init(tc::smem_u32(&s_mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[1]), 1);
        tc::mbar_init(tc::smem_u32(&s_wslot[0]), 1);
        tc::mbar_init(tc::smem_u32(&s_wslot[1]), 1);
        tc::mbar_init_fence();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tc::smem_u32(&s_tmem), P.tmem_cols);
        tc::tmem_relinquish();
    }
    // block of ones (B operand of the bias sums): every 16-bit value = 1.0
    {
        const uint32_t one2 = tc::pack2(1.f, 1.f, P.fp16);
        uint4 *o = reinterpret_cast<uint4 *>(smem + P.ones_off);
        for (int i = threadIdx.x; i < kTcOutN * kTcTile * 2 / 16; i += 128 * NWG)
            o[i] = make_uint4(one2, one2, one2, one2);
    }
    __syncthreads();
    tile_map_build(T, P.counter, s_map);
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const uint32_t mbar = tc::smem_u32(&s_mbar[0]);
    const int bf16 = P.fp16 ? 0 : 1;
    const int nh = md.nh;
    // columns of dL/d(network input) formed at layer 0: the features (both
    // interpolated blocks in the two-decoder optical-thickness pass)
    const int Fn = ((MODE == 1 ? 2 * md.F : md.F) + 15) & ~15;
    uint32_t phase = 0, wphase = 0;
    bool aborted = false;

    float gscale = 1.f;
    if (P.fp16) {
        const float gmax = __uint_as_float(P.counter[kCtrMaxAbsDout]);
        if (gmax > 0.f && isfinite(gmax)) {
            int e;
            frexpf(gmax, &e);                                 // gmax in [2^(e-1), 2^e)
            gscale = ldexpf(1.f, max(-60, min(60, 12 - e)));  // largest |delta_out| -> [2^11, 2^12)
        }
    }
    const float ginv = 1.f / gscale;

    // issue (by row 0) the MMAs queued by `fn`, commit, wait; returns false on timeout
    // `during` runs in every thread between the MMAs' issue and the wait for them
    // A wait that gives up sets `pend`, which the next barrier (the next call's, or the
    // flush's) turns into a uniform abort: no barrier is spent after each wait, since
    // every thread reads only its own TMEM lanes and rewrites only its own rows once its
    // wait has seen the MMAs complete.
    bool pend = false;
    auto run_and = [&](auto &&fn, auto &&during) -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (sync_or(pend)) {
            if (lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
            return false;
        }
        if (lead) {
            tc::fence_after_sync();
            fn();
            tc::mma_commit(mbar);
        }
        during();
        pend |= !tc::mbar_wait(mbar, phase);
        phase ^= 1u;
        tc::fence_after_sync();
        return true;
    };
    auto run = [&](auto &&fn) -> bool { return run_and(fn, [] {}); };

    // ---- streamed weights: slot l % 2 holds W_l (uniform state in every thread)
    struct Pair { int a0, a1; __device__ int &operator[](int k) { return k ? a1 : a0; } };
    struct PairB { bool a0, a1; __device__ bool &operator[](int k) { return k ? a1 : a0; } };
    struct PairU { uint32_t a0, a1; __device__ uint32_t &operator[](int k) { return k ? a1 : a0; } };
    Pair slot_w{-1, -1};
    PairB slot_busy{false, false};
    PairU slot_phase{0u, 0u};
    const uint8_t *img_sc = nullptr;     // the current scene's packed image
    auto issue_load = [&](int l) {
        const int k = l & 1;
        const uint32_t bytes = (uint32_t)(lay.w_rows[l] * lay.w_cols[l] * 2);
        if (lead) {
            const uint32_t mb = tc::smem_u32(&s_wslot[k]);
            tc::mbar_expect_tx(mb, bytes);
            tc::bulk_g2s(s_base + P.slot_off[k], img_sc + lay.w_off[l], bytes, mb);
        }
        slot_w[k] = l;
        slot_busy[k] = true;
    };
    // W_l resident and complete; false on timeout
    auto ensure = [&](int l) -> bool {
        if (!P.stream) return true;
        const int k = l & 1;
        if (slot_w[k] != l) issue_load(l);
        if (slot_busy[k]) {
            const bool to = !tc::mbar_wait(tc::smem_u32(&s_wslot[k]), slot_phase[k]);
            slot_phase[k] ^= 1u;
            slot_busy[k] = false;
            if (sync_or(to)) {
                if (lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
                return false;
            }
        }
        return true;
    };
    // start loading W_next while W_cur is in use, if they sit in different slots
    // (the other slot's previous weights were last read by MMAs already complete)
    auto prefetch = [&](int next, int cur) {
        if (!P.stream || next < 0 || next >= md.nh || ((next ^ cur) & 1) == 0) return;
        if (slot_w[next & 1] == next) return;
        if (slot_busy[next & 1]) return;  // not reached: every issued load is waited for before reuse
        issue_load(next);
    };
    // wait for every weight load still in flight (before a scene change and
    // before the CTA exits: no bulk copy may outlive its destination); false on timeout
    auto drain = [&]() -> bool {
        bool to = false;
        for (int k = 0; k < 2; ++k)
            if (slot_busy[k]) {
                to |= !tc::mbar_wait(tc::smem_u32(&s_wslot[k]), slot_phase[k]);
                slot_phase[k] ^= 1u;
                slot_busy[k] = false;
            }
        return !sync_or(to);
    };
    auto waddr = [&](int l) -> uint32_t {
        if (!P.stream) return s_base + lay.w_off[l];
        return l == md.nh ? s_base : s_base + P.slot_off[l & 1];
    };
    // does the backward at layer l form G_l = G W_l (reads W_l)?
    auto uses_dx = [&](int l, bool feat) { return l > P.l_min || (l == 0 && feat); };

    const int64_t n_tiles = s_map.tile0[T.n];
    const int64_t lo = n_tiles * blockIdx.x / gridDim.x;
    const int64_t hi = n_tiles * (blockIdx.x + 1) / gridDim.x;
    int sc = 0;
    while (sc + 1 < T.n && s_map.tile0[sc + 1] <= lo) ++sc;
    for (int64_t seg = lo; seg < hi && !aborted; ++sc) {
        const int64_t seg_end = min(hi, s_map.tile0[sc + 1]);
        if (seg_end <= seg) continue;
        const SceneDev &SD = T.s[sc];
        // this scene's resident weights
        __syncthreads();
        if (threadIdx.x < 4) s_dbout[threadIdx.x] = 0.f;
        if (!drain()) {
            if (lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
            aborted = true;
            break;
        }
        img_sc = P.images + sc * P.image_stride;
        if (lead) {
            // the whole image, or (streamed weights) its tail: output layer + biases
            const uint32_t mb = tc::smem_u32(&s_mbar[1]);
            const uint32_t nbytes = P.res_bytes;
            tc::mbar_expect_tx(mb, nbytes);
            for (uint32_t off = 0; off < nbytes; off += 32768u)
                tc::bulk_g2s(tc::smem_u32(wimg + off), img_sc + img0 + off, min(32768u, nbytes - off), mb);
        }
        slot_w[0] = slot_w[1] = -1;  // drained above
        aborted = sync_or(!tc::mbar_wait(tc::smem_u32(&s_mbar[1]), wphase));
        wphase ^= 1u;
        tc::fence_after_sync();
        if (aborted) {
            if (lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
            break;
        }
        const int64_t S_sc = s_map.S[sc];
        const int64_t sbase = SD.ray_begin * T.K;
        const int depth = SD.tree.depth;
        float *d_feat = (P.want_feat && P.l_min == 0) ? SD.d_feat : nullptr;
        // the colour pass always forms dL/dpsi at layer 0: it carries the surface
        // point's gradient to eta
        const bool form_dz = MODE == 2 ? P.l_min == 0 : d_feat != nullptr;
        int tiles_done = 0;
        const int64_t tile0 = s_map.tile0[sc];
        TilePrefetch pf;
        pf.v_cur = load_record(P.samples, sbase, tile0, seg, seg_end, S_sc, row, pf.cur);
        pf.v_nxt = load_record(P.samples, sbase, tile0, seg + 1, seg_end, S_sc, row, pf.nxt);
        for (int64_t tile = seg; !aborted && tile < seg_end; ++tile) {
            const int64_t sl = (tile - tile0) * kTcTile + row;
            const int64_t s = sbase + sl;
            const Sample rec = pf.cur;
            const bool valid = pf.v_cur;
            if (MODE == 0 && half == 0 && pf.v_nxt)
                prefetch_gather(pf.nxt, SD.feats, P.feat_bf16, md.F, SD.rays, SD.ray_begin);
            pf.cur = pf.nxt;
            pf.v_cur = pf.v_nxt;
            pf.v_nxt = load_record(P.samples, sbase, tile0, tile + 2, seg_end, S_sc, row, pf.nxt);
            int leaf = -1;
            float carry0 = 0.f, carry1 = 0.f;
            float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
            // ---- 1. X_0 and G_out
            {
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (MODE == 0 && NWG == 2) {
                    build_input_chunks_half(half, md, lay.K0, depth, T.rparam, SD.feats, P.feat_bf16, SD.rays,
                                            SD.ray_begin, rec, valid, P.fp16, smem + P.x_off[0], row);
                    if (valid) leaf = rec.leaf;
                    if (valid && half == 0) g = P.dout[s];
                } else if (MODE == 0) {
                    build_input_chunks(md, lay.K0, depth, T.rparam, SD.feats, P.feat_bf16, SD.rays, SD.ray_begin,
                                       rec, valid, P.fp16, smem + P.x_off[0], row, &leaf);
                    if (valid) g = P.dout[s];
                } else {
                    if (valid) prev = P.aux[s];
                    build_input_two_decoder<MODE>(md, lay.K0, depth, SD.tree.leaf_vertices, SD.feats, P.feat_bf16,
                                                  SD.rays, SD.ray_begin, rec, valid, prev, P.fp16, smem + P.x_off[0],
                                                  row, carry0, carry1);
                    if (valid) {
                        if (MODE == 2) {  // colour: the compositing gradients of the three colour outputs
                            const float4 d4 = P.dout[s];
                            g = make_float4(d4.x, d4.y, d4.z, 0.f);
                        } else {          // optical thickness: (dL/dtau_pre, dL/deta_pre) from the colour pass
                            g = make_float4(prev.x, prev.y, 0.f, 0.f);
                        }
                    }
                }
                if (half == 0) {
                    uint8_t *go = smem + P.gout_off;
                    st_chunk(go, row, 0, tc::pack2(g.x * gscale, g.y * gscale, P.fp16),
                             tc::pack2(g.z * gscale, g.w * gscale, P.fp16), 0u, 0u);
                    st_chunk(go, row, 1, 0u, 0u, 0u, 0u);
                    // bias gradient of the output layer: warp sums, then shared atomics
                    float gs[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float v = gs[c];
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                        if (lane == 0) atomicAdd(&s_dbout[c], v);
                    }
                }
            }
            // ---- 2. forward recompute: X_{l+1} = relu(W_l X_l + b_l)
            for (int l = 0; l < nh && !aborted; ++l) {
                const int Kl = l == 0 ? lay.K0 : kHp;
                const uint32_t xa = s_base + P.x_off[l];
                if (!ensure(l)) {
                    aborted = true;
                    break;
                }
                // next weights needed: layer l + 1 (or, after the top layer, the first
                // backward use below it)
                prefetch(l + 1 < nh ? l + 1 : (uses_dx(nh - 1, form_dz) ? nh - 2 : nh - 1), l);
                const uint32_t wb = waddr(l);
                if (!P.bias_mma) {  // the accumulator starts at the bias
                    const uint4 *b4 = reinterpret_cast<const uint4 *>(bias + lay.bias_l[l]);
#pragma unroll 1
                    for (int c = c32_lo; c < c32_hi; ++c) {
                        uint32_t v[32];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const uint4 t = b4[c * 8 + q];
                            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
                        }
                        tc::tmem_st32(tmem + lane_off + (uint32_t)(c * 32), v);
                    }
                    tc::tmem_wait_st();
                }
                if (!run_and(
                        [&] {
                            const uint32_t idesc = tc::idesc_f16(kTcTile, kHp, bf16, 0, 0);
                            if (P.bias_mma)  // the accumulator starts at the bias: ones x bias pieces
                                tc::mma_f16(tmem, tc::sdesc(s_base + (lay.ones_off - img0), kTcTile * 16, 128),
                                            tc::sdesc(s_base + (lay.bias_b_off[l] - img0), kHp * 16, 128), idesc,
                                            0u);
                            mma_seq(tmem, xa, 2 * kTcTile * 16, kTcTile * 16, 128, wb, 2 * kHp * 16, kHp * 16,
                                    128, Kl, idesc, true);
                        },
                        [&] {
                            // two-decoder passes: the next tile's corner rows to L2 while layer 0 runs
                            if (MODE != 0 && l == 0 && pf.v_cur)
                                prefetch_corners(pf.cur, SD.tree.leaf_vertices, SD.feats, P.feat_bf16, md.F,
                                                 SD.rays, SD.ray_begin);
                        })) {
                    aborted = true;
                    break;
                }
                uint8_t *xn = smem + P.x_off[l + 1];
#pragma unroll 1
                for (int c = c32_lo; c < c32_hi; ++c) {
                    uint32_t v[32];
                    tc::tmem_ld32_wait(tmem + lane_off + (uint32_t)(c * 32), v);
                    uint32_t p[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        p[e] = tc::relu_pack2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]), P.fp16);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        st_chunk(xn, row, c * 4 + q, p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                }
                tc::fence_before_sync();
            }
            if (aborted) break;
            const bool acc = tiles_done > 0;
            // ---- 3. output layer: dW_out^T += X_nh^T G_out ; G_nh = G_out W_out (masked)
            {
                const uint32_t xa = s_base + P.x_off[nh];
                const uint32_t go = s_base + P.gout_off;
                const uint32_t wo = waddr(nh);
                if (!run([&] {
                        if (P.with_out)
                            mma_seq(tmem + P.col_dwout, xa, 256, 128, kTcTile * 16, go, 256, 128, kTcTile * 16,
                                    kTcTile, tc::idesc_f16(kHp, kTcOutN, bf16, 1, 1), acc);
                        mma_seq(tmem, go, 0, kTcTile * 16, 128, wo, 0, 128, kTcOutN * 16, kTcOutN,
                                tc::idesc_f16(kTcTile, kHp, bf16, 0, 1), false);
                    })) {
                    aborted = true;
                    break;
                }
            }
            // masked delta in place of the layer input X_l
            auto mask_epilogue = [&](int l) {
                uint8_t *x = smem + P.x_off[l];
#pragma unroll 1
                for (int c = c32_lo; c < c32_hi; ++c) {
                    uint32_t v[32];
                    tc::tmem_ld32_wait(tmem + lane_off + (uint32_t)(c * 32), v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 *ptr = reinterpret_cast<uint4 *>(x + (c * 4 + q) * (kTcTile * 16) +
                                                               (row >> 3) * 128 + (row & 7) * 16);
                        const uint4 xv = *ptr;
                        const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
                        uint32_t o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)  // delta where the activation is positive, else 0
                            o[e] = tc::mask_pack2(__uint_as_float(v[q * 8 + 2 * e]), __uint_as_float(v[q * 8 + 2 * e + 1]),
                                                  xw[e], P.fp16);
                        *ptr = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                }
                tc::fence_before_sync();
            };
            mask_epilogue(nh);
            // ---- 4. hidden layers, from the top down
            for (int l = nh - 1; l >= P.l_min && !aborted; --l) {
                const uint32_t g = s_base + P.x_off[l + 1];  // G_{l+1} (delta of layer l's output)
                const uint32_t xa = s_base + P.x_off[l];
                const int Nin = l == 0 ? lay.K0 : kHp;
                const bool want_dw = l <= P.l_top;
                const bool want_dx = uses_dx(l, form_dz);
                const int Ndx = l > 0 ? kHp : Fn;
                if (!want_dw && !want_dx) continue;
                if (want_dx) {
                    if (!ensure(l)) {
                        aborted = true;
                        break;
                    }
                    // next: the layer below if it forms a delta, else the next tile's layer 0
                    prefetch(l - 1 >= P.l_min && uses_dx(l - 1, form_dz) ? l - 1 : 0, l);
                }
                const uint32_t wb = waddr(l);
                if (!run([&] {
                        if (want_dw) {
                            // dW_l += G^T X_l  (A: G MN-major, B: X_l MN-major)
                            mma_seq(tmem + P.col_dw[l], g, 256, 128, kTcTile * 16, xa, 256, 128, kTcTile * 16,
                                    kTcTile, tc::idesc_f16(kHp, Nin, bf16, 1, 1), acc);
                            // db_l += G^T 1
                            mma_seq(tmem + P.col_db[l], g, 256, 128, kTcTile * 16, s_base + P.ones_off,
                                    2 * kTcOutN * 16, kTcOutN * 16, 128, kTcTile,
                                    tc::idesc_f16(kHp, kTcOutN, bf16, 1, 0), acc);
                        }
                        // G_l = G W_l  (A: G K-major, B: W_l MN-major)
                        if (want_dx)
                            mma_seq(tmem, g, 2 * kTcTile * 16, kTcTile * 16, 128, wb, 256, 128, kHp * 16,
                                    kHp, tc::idesc_f16(kTcTile, Ndx, bf16, 0, 1), false);
                    })) {
                    aborted = true;
                    break;
                }
                if (l > 0) {
                    if (want_dx) mask_epilogue(l);
                } else if (MODE != 0) {
                    if (form_dz)
                        two_decoder_dz<MODE>(md, SD, rec, valid && sl < S_sc, s, carry0, carry1, prev, d_feat,
                                             tmem + lane_off, ginv, P,
                                             reinterpret_cast<float *>(smem + P.x_off[1]));
                } else if (d_feat) {
                    // dL/dz scatter, aggregated over the lanes of a warp that hit the same leaf: a
                    // lane alone with its leaf adds its row straight from the accumulator; groups
                    // stage their rows in shared memory (X_1's buffer is free now; feature-major,
                    // [f][sample], so a warp's stores hit distinct banks) and the group's lowest
                    // lane adds their sum. 16-byte vector atomics throughout.
                    float *stage = reinterpret_cast<float *>(smem + P.x_off[1]);
                    const int F = md.F;
                    const unsigned grp = __match_any_sync(0xFFFFFFFFu, leaf);
                    const bool solo = __popc(grp) == 1;
                    float4 *dst = reinterpret_cast<float4 *>(d_feat + (int64_t)(leaf >= 0 ? leaf : 0) * F);
                    // this warpgroup's 16-column chunks of dL/dz
                    const int c16_lo = half * (Fn / 16) / NWG * 16, c16_hi = (half + 1) * (Fn / 16) / NWG * 16;
                    for (int c = c16_lo; c < c16_hi; c += 16) {
                        uint32_t v[16];
                        tc::tmem_ld16_wait(tmem + lane_off + (uint32_t)c, v);
                        if (leaf < 0) continue;
                        if (solo) {
#pragma unroll
                            for (int e = 0; e < 16; e += 4)
                                if (c + e < F)
                                    red_add_f4(dst + ((c + e) >> 2), __uint_as_float(v[e]) * ginv,
                                               __uint_as_float(v[e + 1]) * ginv, __uint_as_float(v[e + 2]) * ginv,
                                               __uint_as_float(v[e + 3]) * ginv);
                        } else {
#pragma unroll
                            for (int e = 0; e < 16; ++e)
                                if (c + e < F) stage[(c + e) * kTcTile + row] = __uint_as_float(v[e]) * ginv;
                        }
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (leaf >= 0 && !solo && lane == __ffs(grp) - 1) {
                        for (int f4 = c16_lo / 4; f4 < min(F, c16_hi) / 4; ++f4) {
                            float a[4] = {0.f, 0.f, 0.f, 0.f};
                            unsigned m = grp;
                            while (m) {
                                const int src = (warp << 5) + __ffs(m) - 1;
                                m &= m - 1;
#pragma unroll
                                for (int q = 0; q < 4; ++q) a[q] += stage[(4 * f4 + q) * kTcTile + src];
                            }
                            red_add_f4(dst + f4, a[0], a[1], a[2], a[3]);
                        }
                    }
                    __syncwarp();
                }
            }
            if (!aborted) ++tiles_done;
        }
        // ---- flush this scene's TMEM gradient accumulators (one atomic per element, or per 4
        // where a row is 16-byte aligned)
        if (__syncthreads_or(pend) && !aborted) {  // a give-up in the segment's last MMAs
            if (lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
            aborted = true;
        }
        tc::fence_after_sync();
        if (!aborted && tiles_done > 0 && P.want_params) {
            const int H = md.H;
            float *dpar = SD.d_params;
            // dW_out^T: lane = input feature k, columns = output j (< 4)
            if (P.with_out && half == 0) {
                uint32_t v[16];
                tc::tmem_ld16_wait(tmem + lane_off + P.col_dwout, v);
                if (row < H) {
                    float *dW = dpar + md.w_off[nh];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j < md.out) atomicAdd(dW + j * H + row, __uint_as_float(v[j]) * ginv);
                }
                if (row < md.out) atomicAdd(dpar + md.w_off[nh] + md.out * H + row, s_dbout[row]);
            }
            for (int l = P.l_min; l <= P.l_top; ++l) {
                const int in = md.in_l[l];
                const int ncol = l == 0 ? lay.K0 : kHp;
                float *dW = dpar + md.w_off[l];
                for (int c = half * (ncol / 16) / NWG * 16; c < (half + 1) * (ncol / 16) / NWG * 16; c += 16) {
                    uint32_t v[16];
                    tc::tmem_ld16_wait(tmem + lane_off + P.col_dw[l] + (uint32_t)c, v);
                    if (row < H) {
                        float *dst = dW + row * in + c;
#pragma unroll
                        for (int e = 0; e < 16; e += 4) {
                            if (c + e + 4 <= in && ((uintptr_t)(dst + e) & 15u) == 0) {  // 16-byte vector atomic
                                red_add_f4(reinterpret_cast<float4 *>(dst + e), __uint_as_float(v[e]) * ginv,
                                           __uint_as_float(v[e + 1]) * ginv, __uint_as_float(v[e + 2]) * ginv,
                                           __uint_as_float(v[e + 3]) * ginv);
                            } else {
#pragma unroll
                                for (int q = e; q < e + 4; ++q)
                                    if (c + q < in) atomicAdd(dst + q, __uint_as_float(v[q]) * ginv);
                            }
                        }
                    }
                }
                if (half == 0) {
                    uint32_t v[4];
                    tc::tmem_ld4_wait(tmem + lane_off + P.col_db[l], v);
                    if (row < H) atomicAdd(dW + H * in + row, __uint_as_float(v[0]) * ginv);
                }
            }
        }
        tc::fence_before_sync();
        seg = seg_end;
    }
    if (!drain() && lead) raise_status(SVLF_DEV_WAIT_TIMEOUT);
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, P.tmem_cols);
    }
}

// Split the layers into backward passes from the top down, as few as the
// 512 TMEM columns allow. Returns the number of passes (0 = cannot).
static int tc_bwd_passes(const MlpDims &md, const TcLayout &lay, int l_min[], int l_top[],
                         int with_out[]) {
    int n = 0, top = md.nh - 1, out = 1;
    while (top >= 0 && n < kMaxLayers) {
        int lo = top + 1;
        while (lo - 1 >= 0 && tc_bwd_cols(md, lay, lo - 1, top, out) <= 512) --lo;
        if (lo > top) {  // not even one layer fits
            if (out && tc_bwd_cols(md, lay, top + 1, top, out) <= 512 && n == 0) {
                l_min[n] = top + 1; l_top[n] = top; with_out[n] = 1; ++n; out = 0;
                continue;
            }
            return 0;
        }
        l_min[n] = lo; l_top[n] = top; with_out[n] = out; ++n;
        out = 0;
        top = lo - 1;
    }
    return n;
}

bool tc_backward_supported(const MlpDims &md) {
    if (!tc_supported(md)) return false;
    const TcLayout lay = tc_layout(md);
    int a[kMaxLayers], b[kMaxLayers], c[kMaxLayers];
    const int n = tc_bwd_passes(md, lay, a, b, c);
    if (n == 0) return false;
    for (int pass = 0; pass < n; ++pass) {
        TcBwdParams P;
        memset(&P, 0, sizeof(P));
        P.md = md;
        P.lay = lay;
        P.l_min = a[pass];
        P.l_top = b[pass];
        P.with_out = c[pass];
        size_t smem;
        if (!tc_bwd_plan(md, P, smem)) return false;
    }
    return true;
}

int launch_mlp_backward_tc(const MlpDims &md, int precision, int fb, const SceneTable &T,
                           const Workspace &ws, bool want_feat, bool want_params, cudaStream_t s, int mode,
                           float4 *aux, const float *w_dD, const float *deta) {
    if (!tc_supported(md)) return SVLF_ERR_UNSUPPORTED;
    TcBwdParams P;
    memset(&P, 0, sizeof(P));
    P.md = md;
    P.lay = tc_layout(md);
    int pl_min[kMaxLayers], pl_top[kMaxLayers], pout[kMaxLayers];
    const int n_pass = tc_bwd_passes(md, P.lay, pl_min, pl_top, pout);
    if (n_pass == 0) return SVLF_ERR_UNSUPPORTED;
    P.fp16 = precision == SVLF_FP16;
    P.feat_bf16 = fb;
    P.want_feat = want_feat;
    P.want_params = want_params;
    P.images = (const uint8_t *)ws.packed_w;
    P.image_stride = ws.packed_stride;
    P.samples = ws.samples;
    P.counter = ws.counter;
    P.dout = ws.dout;
    P.aux = aux;
    P.w_dD = w_dD;
    P.deta = deta;
    P.gmax = ws.counter + kCtrMaxAbsDout;
    for (int pass = 0; pass < n_pass; ++pass) {
        if (pl_min[pass] > 0 && !want_params) continue;  // only the last pass forms dL/dz
        P.l_min = pl_min[pass];
        P.l_top = pl_top[pass];
        P.with_out = pout[pass];
        size_t smem;
        if (!tc_bwd_plan(md, P, smem)) return SVLF_ERR_UNSUPPORTED;
        if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM (it owns the TMEM it asks for)
        // two warpgroups per tile: the plain form, one pass, resident weights
        const int bwg = tuning().mlp_bwd_warpgroups;
        if (mode == 0 && n_pass == 1 && !P.stream && bwg != 1) {
            if (cudaFuncSetAttribute(mlp_backward_tc_kernel<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return SVLF_ERR_CUDA;
            prof_begin("mlp_backward_tc", s);
            mlp_backward_tc_kernel<0, 2><<<num_sms(), 256, smem, s>>>(T, P);
            prof_end(s);
            if (cudaGetLastError() != cudaSuccess) return SVLF_ERR_CUDA;
            continue;
        }
        if (mode == 0) {
            if (cudaFuncSetAttribute(mlp_backward_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return SVLF_ERR_CUDA;
        } else if (mode == 1) {
            if (cudaFuncSetAttribute(mlp_backward_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return SVLF_ERR_CUDA;
        } else if (cudaFuncSetAttribute(mlp_backward_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem) != cudaSuccess) {
            return SVLF_ERR_CUDA;
        }
        prof_begin(mode == 0 ? "mlp_backward_tc" : mode == 1 ? "two_decoder_ft_bwd_tc" : "two_decoder_fc_bwd_tc", s);
        if (mode == 0) mlp_backward_tc_kernel<0><<<num_sms(), 128, smem, s>>>(T, P);
        else if (mode == 1) mlp_backward_tc_kernel<1><<<num_sms(), 128, smem, s>>>(T, P);
        else mlp_backward_tc_kernel<2><<<num_sms(), 128, smem, s>>>(T, P);
        prof_end(s);
        if (cudaGetLastError() != cudaSuccess) return SVLF_ERR_CUDA;
    }
    return SVLF_OK;
}

}  // namespace svlf
