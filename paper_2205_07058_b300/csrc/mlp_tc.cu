// The per-sample network on the 5th-generation tensor cores (tcgen05):
// SVLF_BF16 and SVLF_FP16 (16-bit operands, float32 accumulation in TMEM).
//
// Forward kernel (persistent, one CTA per SM, 2-4 warpgroups):
//  * The packed weights of every layer (16-bit, core-matrix layout, plus the
//    float32 biases) are copied once per CTA into shared memory with bulk
//    (TMA) copies and stay resident.
//  * Each warpgroup owns a tile of 128 samples at a time: thread t builds the
//    network input of sample t (feature gather with 16-byte loads, ray
//    parameterisation in double-float), rounds it to 16 bits and stores it in
//    the warpgroup's activation buffer (the A operand).
//  * One thread issues the layer's tcgen05.mma instructions (M = 128 samples,
//    N = layer width, K = 16 each) into the warpgroup's 128 TMEM columns and
//    commits them to an mbarrier; the warpgroup waits, reads its row of the
//    accumulator (tcgen05.ld, lane = sample), adds the bias, applies ReLU,
//    rounds to 16 bits and writes the next layer's A operand in place.
//  * The last layer (N padded 4 -> 16) writes sigmoid colour and ReLU optical
//    thickness per sample.
//  Warpgroups run independently, so the tensor core works on one tile while
//  the others gather inputs or run their epilogues.
#include <cstring>

#include "svlf_internal.cuh"
#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace svlf {

constexpr int kTcTile = 128;     // samples per tile (MMA M)
constexpr int kTcOutN = 16;      // output layer width padded to the smallest legal N

struct TcLayout {
    int K0;                      // first-layer K, in0 rounded up to 16
    int n_layers;                // nh + 1
    uint32_t w_off[kMaxLayers];  // byte offset of each layer's B tile in the image
    uint32_t w_rows[kMaxLayers]; // rows (N) of each B tile
    uint32_t w_cols[kMaxLayers]; // columns (K) of each B tile
    uint32_t bias_off;           // byte offset of the float32 biases
    uint32_t bias_l[kMaxLayers]; // float index of each layer's bias within the bias block
    uint32_t bytes;              // total image size (multiple of 16)
};

static TcLayout tc_layout(const MlpDims &md) {
    TcLayout t;
    memset(&t, 0, sizeof(t));
    t.K0 = (md.in0 + 15) & ~15;
    t.n_layers = md.nh + 1;
    uint32_t off = 0;
    for (int l = 0; l <= md.nh; ++l) {
        t.w_rows[l] = l == md.nh ? kTcOutN : md.H;
        t.w_cols[l] = l == 0 ? t.K0 : md.H;
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
    return t;
}

bool tc_supported(const MlpDims &md) {
    return (md.H == 64 || md.H == 128) && md.in0 <= 80 && md.nh >= 1 && md.nh <= 6;
}

size_t packed_tc_bytes(const MlpDims &md) {
    if (!tc_supported(md)) return 0;
    return tc_layout(md).bytes;
}

// ---------------------------------------------------------------- packing
__global__ void pack_tc_kernel(MlpDims md, TcLayout lay, int fp16, const float *__restrict__ params,
                               uint8_t *__restrict__ image) {
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
    }
}

int launch_pack_tc(const MlpDims &md, int precision, const float *params, void *packed,
                   cudaStream_t s) {
    if (!tc_supported(md)) return SVLF_ERR_UNSUPPORTED;
    const TcLayout lay = tc_layout(md);
    prof_begin("pack_weights_tc", s);
    pack_tc_kernel<<<64, 256, 0, s>>>(md, lay, precision == SVLF_FP16, params, (uint8_t *)packed);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

// ---------------------------------------------------------------- forward
struct TcFwdParams {
    MlpDims md;
    TcLayout lay;
    int depth;
    int fp16;
    const void *feats;
    int feat_bf16;
    const uint8_t *image;
    const float *rays;
    const Sample *samples;
    const unsigned int *counter;
    int64_t max_samples;
    float4 *outputs;
    int n_wg;            // warpgroups per CTA
    uint32_t abuf_bytes; // activation buffer per warpgroup
};

// Store one 16-bit row chunk (8 values packed in 4 words) at column block kb.
__device__ __forceinline__ void st_chunk(uint8_t *abuf, int row, int kb, uint32_t a, uint32_t b,
                                         uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4 *>(abuf + kb * (kTcTile * 16) + (row >> 3) * 128 + (row & 7) * 16) =
        make_uint4(a, b, c, d);
}

template <int H>
__global__ void __launch_bounds__(512, 1) mlp_forward_tc_kernel(const TcFwdParams P) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t s_mbar[5];  // [0..3] per warpgroup, [4] weight load
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int wg = tid >> 7;        // warpgroup
    const int row = tid & 127;      // sample row within the tile = TMEM lane
    const int warp = tid >> 5;
    const uint32_t ncols = P.n_wg <= 2 ? 256u : 512u;
    uint8_t *wimg = smem;
    uint8_t *abuf = smem + P.lay.bytes + wg * P.abuf_bytes;
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
    // resident weights: bulk copies into shared memory
    if (tid == 0) {
        const uint32_t mb = tc::smem_u32(&s_mbar[4]);
        tc::mbar_expect_tx(mb, P.lay.bytes);
        for (uint32_t off = 0; off < P.lay.bytes; off += 32768u) {
            const uint32_t n = min(32768u, P.lay.bytes - off);
            tc::bulk_g2s(tc::smem_u32(wimg + off), P.image + off, n, mb);
        }
    }
    if (!tc::mbar_wait(tc::smem_u32(&s_mbar[4]), 0)) {
        raise_status(SVLF_DEV_WAIT_TIMEOUT);
        atomicExch(&s_abort, 1);
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem_base = s_tmem;
    const uint32_t tmem_wg = tmem_base + (uint32_t)(wg * 128);            // column base
    const uint32_t tmem_row = tmem_wg + ((uint32_t)((warp & 3) * 32) << 16);  // lane base
    const uint32_t mbar = tc::smem_u32(&s_mbar[wg]);
    const uint32_t abuf_s = tc::smem_u32(abuf);
    const uint32_t wimg_s = tc::smem_u32(wimg);
    const int bf16 = P.fp16 ? 0 : 1;
    uint32_t phase = 0;

    const int64_t S = min((int64_t)P.counter[0], P.max_samples);
    const int64_t n_tiles = (S + kTcTile - 1) / kTcTile;
    bool aborted = s_abort != 0;
    for (int64_t tile = (int64_t)blockIdx.x * P.n_wg + wg; !aborted && tile < n_tiles;
         tile += (int64_t)gridDim.x * P.n_wg) {
        const int64_t s = tile * kTcTile + row;
        // ---- network input row -> A operand (K0 columns)
        {
            float h0[kMaxIn];
            const bool valid = s < S;
            if (valid) make_input_row(P.md, P.depth, P.feats, P.feat_bf16, P.rays, P.samples[s], h0);
            for (int kb = 0; kb < P.lay.K0 / 8; ++kb) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = kb * 8 + e;
                    v[e] = (valid && k < P.md.in0) ? h0[k] : 0.f;
                }
                st_chunk(abuf, row, kb, tc::pack2(v[0], v[1], P.fp16), tc::pack2(v[2], v[3], P.fp16),
                         tc::pack2(v[4], v[5], P.fp16), tc::pack2(v[6], v[7], P.fp16));
            }
        }
        for (int l = 0; l < P.lay.n_layers; ++l) {
            const int N = P.lay.w_rows[l];
            const int Kl = P.lay.w_cols[l];
            // A operand written by all threads -> visible to the tensor core
            tc::fence_async_smem();
            tc::fence_before_sync();
            tc::wg_sync_or(wg, false);
            if (row == 0) {
                tc::fence_after_sync();
                const uint32_t idesc = tc::idesc_f16(kTcTile, N, bf16, 0, 0);
                const uint32_t b_base = wimg_s + P.lay.w_off[l];
                for (int k = 0; k < Kl; k += 16) {
                    const uint64_t da = tc::sdesc(abuf_s + (k >> 3) * (kTcTile * 16), kTcTile * 16, 128);
                    const uint64_t db = tc::sdesc(b_base + (k >> 3) * (N * 16), N * 16, 128);
                    tc::mma_f16(tmem_wg, da, db, idesc, k > 0 ? 1u : 0u);
                }
                tc::mma_commit(mbar);
            }
            const bool timeout = !tc::mbar_wait(mbar, phase);
            phase ^= 1u;
            if (tc::wg_sync_or(wg, timeout)) {
                if (row == 0) raise_status(SVLF_DEV_WAIT_TIMEOUT);
                aborted = true;
                break;
            }
            tc::fence_after_sync();
            const float *b = bias + P.lay.bias_l[l];
            if (l + 1 < P.lay.n_layers) {
                // hidden layer epilogue: bias + ReLU -> 16-bit A operand of the next layer
#pragma unroll
                for (int c = 0; c < H / 32; ++c) {
                    uint32_t v[32];
                    tc::tmem_ld32(tmem_row + (uint32_t)(c * 32), v);
                    tc::tmem_wait_ld();
                    uint32_t p[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float x0 = fmaxf(__uint_as_float(v[2 * e]) + b[c * 32 + 2 * e], 0.f);
                        const float x1 = fmaxf(__uint_as_float(v[2 * e + 1]) + b[c * 32 + 2 * e + 1], 0.f);
                        p[e] = tc::pack2(x0, x1, P.fp16);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        st_chunk(abuf, row, c * 4 + q, p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                }
            } else {
                uint32_t v[4];
                tc::tmem_ld4(tmem_row, v);
                tc::tmem_wait_ld();
                if (s < S)
                    P.outputs[s] = output_activation(__uint_as_float(v[0]) + b[0], __uint_as_float(v[1]) + b[1],
                                                     __uint_as_float(v[2]) + b[2], __uint_as_float(v[3]) + b[3]);
            }
        }
        // all TMEM reads of this tile are done before the next tile's MMAs
        tc::fence_before_sync();
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, ncols);
    }
}

static int tc_forward_config(const MlpDims &md, const TcLayout &lay, int &n_wg, uint32_t &abuf,
                             size_t &smem) {
    const int kmax = lay.K0 > md.H ? lay.K0 : md.H;
    abuf = (uint32_t)(kTcTile * kmax * 2);
    const size_t limit = 227 * 1024 - 256;
    for (n_wg = 4; n_wg >= 1; --n_wg) {
        smem = lay.bytes + (size_t)n_wg * abuf + 128;  // + alignment slack
        if (smem <= limit) break;
    }
    if (n_wg < 1) return SVLF_ERR_UNSUPPORTED;
    if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM: it owns all TMEM columns it asks for
    return SVLF_OK;
}

template <int H>
static int fwd_tc(const TcFwdParams &P0, const MlpDims &md, const TcLayout &lay, cudaStream_t s,
                  int n_wg_override) {
    TcFwdParams P = P0;
    size_t smem;
    int rc = tc_forward_config(md, lay, P.n_wg, P.abuf_bytes, smem);
    if (rc) return rc;
    if (n_wg_override > 0 && n_wg_override < P.n_wg) P.n_wg = n_wg_override;
    if (cudaFuncSetAttribute(mlp_forward_tc_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    prof_begin("mlp_forward_tc", s);
    mlp_forward_tc_kernel<H><<<num_sms(), 128 * P.n_wg, smem, s>>>(P);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

static int g_tc_wg_override = 0;

int launch_mlp_forward_tc(const MlpDims &md, int precision, int depth, const void *feats, int fb,
                          const void *packed, const float *rays, const Workspace &ws,
                          int64_t max_samples, cudaStream_t s) {
    if (!tc_supported(md)) return SVLF_ERR_UNSUPPORTED;
    TcFwdParams P;
    memset(&P, 0, sizeof(P));
    P.md = md;
    P.lay = tc_layout(md);
    P.depth = depth;
    P.fp16 = precision == SVLF_FP16;
    P.feats = feats;
    P.feat_bf16 = fb;
    P.image = (const uint8_t *)packed;
    P.rays = rays;
    P.samples = ws.samples;
    P.counter = ws.counter;
    P.max_samples = max_samples;
    P.outputs = ws.outputs;
    if (md.H == 64) return fwd_tc<64>(P, md, P.lay, s, g_tc_wg_override);
    return fwd_tc<128>(P, md, P.lay, s, g_tc_wg_override);
}

int launch_mlp_backward_tc(const MlpDims &, int, int, const void *, int, const void *,
                           const float *, const Workspace &, int64_t, float *, float *,
                           cudaStream_t) {
    return SVLF_ERR_UNSUPPORTED;
}

}  // namespace svlf
