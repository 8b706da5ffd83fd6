// The per-sample network in plain float32 on the SIMT cores (SVLF_FP32), and
// the shared pieces every network path uses: the input row
// h0 = [z | d | p~1 | p~2] (Sec. 4.1 ray parameterisation) and the output
// activations (sigmoid colour, ReLU optical thickness; Sec. 4.5).
//
// Forward: tiles of 128 samples, activations feature-major in shared memory
// ([k][s]), each of 256 threads computing an (H/16) x 8 block of the next
// layer; weights are read transposed (packed as W^T) through the read-only
// cache.
// Backward: tiles of 64 samples; the forward is recomputed and every layer's
// input kept in shared memory; dW = delta^T a is formed per tile in 4 x 4
// register blocks and added to the global gradient with one atomic per
// element per tile; dz (the feature gradient) is scattered with atomics.
#include "svlf_internal.cuh"
#include "mlp_common.cuh"
#include "mlp_simt.h"

namespace svlf {

constexpr int kTsF = 128;  // forward tile (samples)
constexpr int kTsB = 64;   // backward tile (samples)
constexpr int kPadB = 68;  // row stride (floats) of backward tiles
constexpr int kBwdWRows = 32;  // rows of W^T staged at a time in the backward's recompute

// Y[j][s] = relu(b_j + sum_k WT[k][j] X[k][s]) for j < H, s < TS (row stride ts),
// also in three parts so that a caller can stage W^T in shared memory in row
// ranges: gemm_init (the bias), gemm_rows (the K steps [k0, k1), with WT
// pointing at row k0 of W^T), gemm_store (ReLU and the store of Y).
// W^T is read from shared memory (W_SMEM, staged by the caller) or through
// the read-only cache. Thread (ty, tx) of 256 computes rows j0 .. j0 + H/16 - 1
// for SPT samples in SPT/4 groups of four, group g at g TS / (SPT/4) + 4 tx:
// the eight lanes of a quarter warp then read 128 contiguous bytes of X per
// load (no bank conflict). The loads of step k + 1 are issued before the FMAs
// of step k. Each output is the same fmaf chain in ascending k whatever the
// thread mapping and the row ranges.
template <int H, int SPT>
__device__ __forceinline__ void gemm_init(float (&acc)[H / 16][SPT], const float *__restrict__ bias) {
    const int j0 = (threadIdx.x >> 4) * (H / 16);
#pragma unroll
    for (int j = 0; j < H / 16; ++j) {
        const float b = __ldg(bias + j0 + j);
#pragma unroll
        for (int s = 0; s < SPT; ++s) acc[j][s] = b;
    }
}

template <int H, int TS, int SPT, bool W_SMEM, int KF = 0>
__device__ __forceinline__ void gemm_rows(float (&acc)[H / 16][SPT], const float *__restrict__ X, int k0, int k1,
                                          int ts, const float *__restrict__ WT) {
    if (KF > 0) k1 = k0 + KF;  // a K known at compile time (even): no bounds checks in the loop
    constexpr int JT = H / 16;
    constexpr int NG = SPT / 4;
    static_assert(SPT % 4 == 0 && TS == 16 * SPT, "16 threads x SPT samples cover the tile");
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int j0 = ty * JT;
    auto load = [&](int k, float (&x)[SPT], float (&w)[JT]) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const float4 a = *reinterpret_cast<const float4 *>(X + k * ts + g * (TS / NG) + 4 * tx);
            x[4 * g] = a.x; x[4 * g + 1] = a.y; x[4 * g + 2] = a.z; x[4 * g + 3] = a.w;
        }
        if (JT % 4 == 0) {
#pragma unroll
            for (int j4 = 0; j4 < JT / 4; ++j4) {
                const float4 *p = reinterpret_cast<const float4 *>(WT + (k - k0) * H + j0 + 4 * j4);
                const float4 v = W_SMEM ? *p : __ldg(p);
                w[4 * j4] = v.x; w[4 * j4 + 1] = v.y; w[4 * j4 + 2] = v.z; w[4 * j4 + 3] = v.w;
            }
        } else {  // H = 32: two rows per thread
            static_assert(JT % 4 == 0 || JT == 2, "rows per thread");
            const float2 *p = reinterpret_cast<const float2 *>(WT + (k - k0) * H + j0);
            const float2 v = W_SMEM ? *p : __ldg(p);
            w[0] = v.x; w[JT - 1] = v.y;
        }
    };
    auto fma_step = [&](const float (&x)[SPT], const float (&w)[JT]) {
#pragma unroll
        for (int j = 0; j < JT; ++j)
#pragma unroll
            for (int s = 0; s < SPT; ++s) acc[j][s] = fmaf(w[j], x[s], acc[j][s]);
    };
    float xa[SPT], wa[JT], xb[SPT], wb[JT];
    if (KF > 0) {
        static_assert(KF % 2 == 0, "even K");
        load(k0, xa, wa);
#pragma unroll 2
        for (int k = k0; k < k0 + KF; k += 2) {
            load(k + 1, xb, wb);
            fma_step(xa, wa);
            if (k + 2 < k0 + KF) load(k + 2, xa, wa);
            fma_step(xb, wb);
        }
        return;
    }
    if (k0 < k1) load(k0, xa, wa);
    for (int k = k0; k < k1; k += 2) {
        if (k + 1 < k1) load(k + 1, xb, wb);
        fma_step(xa, wa);
        if (k + 1 < k1) {
            if (k + 2 < k1) load(k + 2, xa, wa);
            fma_step(xb, wb);
        }
    }
}

template <int H, int TS, int SPT>
__device__ __forceinline__ void gemm_store(const float (&acc)[H / 16][SPT], float *__restrict__ Y, int ts, bool relu) {
    constexpr int NG = SPT / 4;
    const int tx = threadIdx.x & 15;
    const int j0 = (threadIdx.x >> 4) * (H / 16);
#pragma unroll
    for (int j = 0; j < H / 16; ++j)
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            float4 v;
            v.x = relu ? fmaxf(acc[j][4 * g], 0.f) : acc[j][4 * g];
            v.y = relu ? fmaxf(acc[j][4 * g + 1], 0.f) : acc[j][4 * g + 1];
            v.z = relu ? fmaxf(acc[j][4 * g + 2], 0.f) : acc[j][4 * g + 2];
            v.w = relu ? fmaxf(acc[j][4 * g + 3], 0.f) : acc[j][4 * g + 3];
            *reinterpret_cast<float4 *>(Y + (j0 + j) * ts + g * (TS / NG) + 4 * tx) = v;
        }
}

template <int H, int TS, int SPT, bool W_SMEM = false>
__device__ __forceinline__ void gemm_relu_f32(const float *__restrict__ X, int in, int ts,
                                              const float *__restrict__ WT,
                                              const float *__restrict__ bias, float *__restrict__ Y,
                                              bool relu) {
    float acc[H / 16][SPT];
    gemm_init<H, SPT>(acc, bias);
    gemm_rows<H, TS, SPT, W_SMEM>(acc, X, 0, in, ts, WT);
    gemm_store<H, TS, SPT>(acc, Y, ts, relu);
}

// Write h0 of sample s (or zeros) into column `col` of X (row stride ts).
__device__ __forceinline__ void build_input_column(const MlpDims &md, int depth, int rparam,
                                                   const void *feats, int feat_bf16,
                                                   const float *rays, const Sample *samples,
                                                   int64_t s, int64_t S, float *X, int ts,
                                                   int col, int rows_padded) {
    if (s < S) {
        make_input_row(md, depth, rparam, feats, feat_bf16, rays, samples[s], X + col, ts);
    } else {
        for (int k = 0; k < md.in0; ++k) X[k * ts + col] = 0.f;
    }
    for (int k = md.in0; k < rows_padded; ++k) X[k * ts + col] = 0.f;
}

// WSTAGE: each layer's W^T is copied into shared memory before the layer
// (when it fits next to the two activation tiles): read from L1 / L2 instead,
// the rows of W^T of the network's layers together exceed L1, and every K
// step of the GEMM waited on a miss.
template <int H, bool WSTAGE>
__global__ void __launch_bounds__(256) mlp_forward_f32_kernel(
    const __grid_constant__ MlpDims md, int depth, int rparam, const void *__restrict__ feats, int feat_bf16,
    const float *__restrict__ packed, const float *__restrict__ rays,
    const Sample *__restrict__ samples, const unsigned int *__restrict__ counter,
    int64_t max_samples, float4 *__restrict__ outputs) {
    extern __shared__ float4 smem_f4[];
    float *X = reinterpret_cast<float *>(smem_f4);
    const int dmax = md.in0 > H ? md.in0 : H;
    float *Y = X + dmax * kTsF;
    float *Wsm = Y + H * kTsF;
    const int64_t S = min((int64_t)counter[kCtrScene], max_samples);
    const int64_t n_tiles = (S + kTsF - 1) / kTsF;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTsF;
        if (threadIdx.x < kTsF)
            build_input_column(md, depth, rparam, feats, feat_bf16, rays, samples, s0 + threadIdx.x, S, X,
                               kTsF, threadIdx.x, md.in0);
        __syncthreads();
        int in = md.in0;
        float *A = X, *B = Y;
        for (int l = 0; l < md.nh; ++l) {
            if (WSTAGE) {
                const float4 *src = reinterpret_cast<const float4 *>(packed + md.wt_off[l]);
                float4 *dst = reinterpret_cast<float4 *>(Wsm);
                for (int i = threadIdx.x; i < in * H / 4; i += blockDim.x) dst[i] = __ldg(src + i);
                __syncthreads();
                gemm_relu_f32<H, kTsF, 8, true>(A, in, kTsF, Wsm, packed + md.b_off[l], B, true);
            } else {
                gemm_relu_f32<H, kTsF, 8>(A, in, kTsF, packed + md.wt_off[l], packed + md.b_off[l], B, true);
            }
            __syncthreads();
            float *t = A; A = B; B = t;
            in = H;
        }
        if (threadIdx.x < kTsF && s0 + threadIdx.x < S) {
            const float *WT = packed + md.wt_off[md.nh];
            const float *b = packed + md.b_off[md.nh];
            float o0 = __ldg(b), o1 = __ldg(b + 1), o2 = __ldg(b + 2), o3 = __ldg(b + 3);
            for (int k = 0; k < H; ++k) {
                const float a = A[k * kTsF + threadIdx.x];
                const float4 w = __ldg(reinterpret_cast<const float4 *>(WT + 4 * k));
                o0 = fmaf(w.x, a, o0); o1 = fmaf(w.y, a, o1);
                o2 = fmaf(w.z, a, o2); o3 = fmaf(w.w, a, o3);
            }
            outputs[s0 + threadIdx.x] = output_activation(o0, o1, o2, o3);
        }
        __syncthreads();
    }
}

// Weights-resident form: the whole packed float32 network (every layer's W^T)
// copied into shared memory once per CTA, next to one activation tile of
// kTsR samples that each layer overwrites in place (its outputs are held in
// registers until every thread has read the layer's input); all 256 threads
// build a tile's input columns (two per sample: feature chunks c with
// c % 2 = q, and q = 1 also the direction and entry/exit parameters) and form
// its outputs (two per thread). Every value is the one the staged form
// computes: the same input row, the same ascending-k fmaf chain per output
// (biases read from the packed buffer in global memory).
constexpr int kTsR = 128;

template <int H>
__global__ void __launch_bounds__(256) mlp_forward_f32_res_kernel(
    const __grid_constant__ MlpDims md, int depth, int rparam, const void *__restrict__ feats, int feat_bf16,
    const float *__restrict__ packed, int packed_floats, const float *__restrict__ rays,
    const Sample *__restrict__ samples, const unsigned int *__restrict__ counter,
    int64_t max_samples, float4 *__restrict__ outputs) {
    extern __shared__ float4 smem_f4[];
    float *Wsm = reinterpret_cast<float *>(smem_f4);
    float *X = Wsm + packed_floats;  // max(in0, H) x kTsR
    {
        const float4 *src = reinterpret_cast<const float4 *>(packed);
        for (int i = threadIdx.x; i < packed_floats / 4; i += blockDim.x) smem_f4[i] = __ldg(src + i);
    }
    const int F = md.F;
    const int col = threadIdx.x & (kTsR - 1);  // sample within the tile
    const int q = threadIdx.x >> 7;            // which half of its input row / of its outputs
    const int64_t S = min((int64_t)counter[kCtrScene], max_samples);
    const int64_t n_tiles = (S + kTsR - 1) / kTsR;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTsR;
        const int64_t s = s0 + col;
        if (s < S) {
            const Sample sm = samples[s];
            if (feat_bf16) {
                const uint4 *src = reinterpret_cast<const uint4 *>(
                    reinterpret_cast<const __nv_bfloat16 *>(feats) + (int64_t)sm.leaf * F);
                for (int c = q; c < F / 8; c += 2) {
                    const uint4 v = __ldg(src + c);
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        X[(8 * c + 2 * e) * kTsR + col] = __uint_as_float(w[e] << 16);
                        X[(8 * c + 2 * e + 1) * kTsR + col] = __uint_as_float(w[e] & 0xFFFF0000u);
                    }
                }
            } else {
                const float4 *src = reinterpret_cast<const float4 *>(
                    reinterpret_cast<const float *>(feats) + (int64_t)sm.leaf * F);
                for (int c = q; c < F / 4; c += 2) {
                    const float4 v = __ldg(src + c);
                    X[(4 * c) * kTsR + col] = v.x;
                    X[(4 * c + 1) * kTsR + col] = v.y;
                    X[(4 * c + 2) * kTsR + col] = v.z;
                    X[(4 * c + 3) * kTsR + col] = v.w;
                }
            }
            if (q == 1) {
                const float2 *rp = reinterpret_cast<const float2 *>(rays + 6 * (int64_t)sm.ray);
                const float2 a = __ldg(rp), b = __ldg(rp + 1), c = __ldg(rp + 2);
                const float o[3] = {a.x, a.y, b.x};
                const float d[3] = {b.y, c.x, c.y};
                float p1[3], p2[3];
                voxel_param_at(rparam, o, d, sm.tmid, sm.cell, depth, p1, p2);
                const float v[9] = {d[0], d[1], d[2], p1[0], p1[1], p1[2], p2[0], p2[1], p2[2]};
#pragma unroll
                for (int k = 0; k < 9; ++k) X[(F + k) * kTsR + col] = v[k];
            }
        } else {
            for (int k = q; k < md.in0; k += 2) X[k * kTsR + col] = 0.f;
        }
        __syncthreads();
        int in = md.in0;
        for (int l = 0; l < md.nh; ++l) {
            float acc[H / 16][8];
            gemm_init<H, 8>(acc, packed + md.b_off[l]);
            if (l > 0)
                gemm_rows<H, kTsR, 8, true, H>(acc, X, 0, H, kTsR, Wsm + md.wt_off[l]);
            else
                gemm_rows<H, kTsR, 8, true>(acc, X, 0, in, kTsR, Wsm + md.wt_off[l]);
            __syncthreads();  // every thread has read the layer's input
            gemm_store<H, kTsR, 8>(acc, X, kTsR, true);
            __syncthreads();
            in = H;
        }
        if (s < S) {
            const float *WT = Wsm + md.wt_off[md.nh];  // H x 4
            const int o0 = 2 * q;
            float a0 = __ldg(packed + md.b_off[md.nh] + o0), a1 = __ldg(packed + md.b_off[md.nh] + o0 + 1);
            for (int k = 0; k < H; ++k) {
                const float x = X[k * kTsR + col];
                const float2 w = *reinterpret_cast<const float2 *>(WT + 4 * k + o0);
                a0 = fmaf(w.x, x, a0);
                a1 = fmaf(w.y, x, a1);
            }
            float2 r;
            r.x = sigmoidf_(a0);
            r.y = q == 0 ? sigmoidf_(a1) : fmaxf(a1, 0.f);
            reinterpret_cast<float2 *>(outputs)[2 * s + q] = r;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- backward
// dW[j][k] += sum_s D[j][s] A[k][s] over a tile (rows j < nj, k < nk). A
// thread's block is rows j0 .. j0 + 3 of D and four rows of A: k0 .. k0 + 3,
// or, where nk is a multiple of 32 (STRIDED), rows k0, k0 + 8, k0 + 16,
// k0 + 24 of a 32-row group, so that the lanes of a warp read rows one apart
// (at the 68-float row stride, consecutive rows fall on different banks;
// rows four apart share two bank groups).
template <bool STRIDED>
__device__ __forceinline__ void accumulate_dw(const float *D, const float *A, int nj, int nk,
                                              float *__restrict__ dW, int ld) {
    const int bj = (nj + 3) / 4, bk = (nk + 3) / 4;
    for (int blk = threadIdx.x; blk < bj * bk; blk += blockDim.x) {
        const int j0 = (blk / bk) * 4, kb = blk % bk;
        const int k0 = STRIDED ? (kb >> 3) * 32 + (kb & 7) : kb * 4;
        constexpr int ks = STRIDED ? 8 : 1;  // row step within the block
        float acc[4][4] = {};
        for (int s = 0; s < kTsB; s += 4) {
            float4 d[4], a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d[q] = *reinterpret_cast<const float4 *>(D + (j0 + q) * kPadB + s);
                a[q] = *reinterpret_cast<const float4 *>(A + (k0 + ks * q) * kPadB + s);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    acc[p][q] += d[p].x * a[q].x + d[p].y * a[q].y + d[p].z * a[q].z +
                                 d[p].w * a[q].w;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + p < nj && k0 + ks * q < nk) atomicAdd(dW + (j0 + p) * ld + k0 + ks * q, acc[p][q]);
    }
}

// Dst[k][s] = (sum_j W[j][k] D[j][s]) * mask(A[k][s] > 0), k < nk (W row-major, ld = nk_full)
template <bool MASK>
__device__ __forceinline__ void backprop_delta(const float *__restrict__ W, int nj, int nk,
                                               int ldw, const float *D, const float *A,
                                               float *Dst) {
    const int bk = (nk + 3) / 4;
    for (int blk = threadIdx.x; blk < bk * (kTsB / 4); blk += blockDim.x) {
        const int k0 = (blk % bk) * 4, s0 = (blk / bk) * 4;
        float acc[4][4] = {};
        for (int j = 0; j < nj; ++j) {
            const float4 d = *reinterpret_cast<const float4 *>(D + j * kPadB + s0);
            float w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = (k0 + q < nk) ? __ldg(W + j * ldw + k0 + q) : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[q][0] = fmaf(w[q], d.x, acc[q][0]);
                acc[q][1] = fmaf(w[q], d.y, acc[q][1]);
                acc[q][2] = fmaf(w[q], d.z, acc[q][2]);
                acc[q][3] = fmaf(w[q], d.w, acc[q][3]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (k0 + q >= nk) continue;
            float4 v = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
            if (MASK) {
                const float4 a = *reinterpret_cast<const float4 *>(A + (k0 + q) * kPadB + s0);
                v.x = a.x > 0.f ? v.x : 0.f;
                v.y = a.y > 0.f ? v.y : 0.f;
                v.z = a.z > 0.f ? v.z : 0.f;
                v.w = a.w > 0.f ? v.w : 0.f;
            }
            *reinterpret_cast<float4 *>(Dst + (k0 + q) * kPadB + s0) = v;
        }
    }
}

// The same product with W read from shared memory: rows [j0, j0 + kBwdWRows)
// of W are staged into Wst (row stride nk rounded up to 4) by all threads,
// then every thread adds their terms to its (up to two) 4 x 4 blocks, in
// ascending j as above, so every output is the same fmaf chain. Called by
// all threads of the block (it synchronises); nk <= 128, and the staged rows
// (kBwdWRows x nk rounded up to 4) fit the caller's buffer.
template <bool MASK>
__device__ __forceinline__ void backprop_delta_staged(const float *__restrict__ W, int nj, int nk, int ldw,
                                                      const float *D, const float *A, float *Dst, float *Wst) {
    const int bk = (nk + 3) / 4;
    const int nblk = bk * (kTsB / 4);
    const int nk4 = bk * 4;
    float acc[2][4][4] = {};
    for (int j0 = 0; j0 < nj; j0 += kBwdWRows) {
        const int nr = min(nj - j0, kBwdWRows);
        for (int e = threadIdx.x; e < nr * nk4; e += blockDim.x) {
            const int r = e / nk4, c = e % nk4;
            Wst[e] = c < nk ? __ldg(W + (size_t)(j0 + r) * ldw + c) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int blk = threadIdx.x + b * blockDim.x;
            if (blk >= nblk) break;
            const int k0 = (blk % bk) * 4, s0 = (blk / bk) * 4;
            for (int r = 0; r < nr; ++r) {
                const float4 d = *reinterpret_cast<const float4 *>(D + (j0 + r) * kPadB + s0);
                const float4 w4 = *reinterpret_cast<const float4 *>(Wst + r * nk4 + k0);
                const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[b][q][0] = fmaf(w[q], d.x, acc[b][q][0]);
                    acc[b][q][1] = fmaf(w[q], d.y, acc[b][q][1]);
                    acc[b][q][2] = fmaf(w[q], d.z, acc[b][q][2]);
                    acc[b][q][3] = fmaf(w[q], d.w, acc[b][q][3]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int blk = threadIdx.x + b * blockDim.x;
        if (blk >= nblk) break;
        const int k0 = (blk % bk) * 4, s0 = (blk / bk) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (k0 + q >= nk) continue;
            float4 v = make_float4(acc[b][q][0], acc[b][q][1], acc[b][q][2], acc[b][q][3]);
            if (MASK) {
                const float4 a = *reinterpret_cast<const float4 *>(A + (k0 + q) * kPadB + s0);
                v.x = a.x > 0.f ? v.x : 0.f;
                v.y = a.y > 0.f ? v.y : 0.f;
                v.z = a.z > 0.f ? v.z : 0.f;
                v.w = a.w > 0.f ? v.w : 0.f;
            }
            *reinterpret_cast<float4 *>(Dst + (k0 + q) * kPadB + s0) = v;
        }
    }
}

// Up to kBwdWRows rows of a row-major matrix with H floats per row (16-byte
// aligned), held in registers between their global load and their store to
// shared memory: the next chunk's loads are issued before the current
// chunk's products, so their latency hides behind them.
template <int H>
struct RowStage {
    static constexpr int NV = (kBwdWRows * H / 4 + 255) / 256;  // float4 per thread (256 threads)
    float4 v[NV];
    __device__ __forceinline__ void load(const float *__restrict__ src, int nrows) {
        const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = threadIdx.x + i * 256;
            if (e < nrows * H / 4) v[i] = __ldg(p + e);
        }
    }
    __device__ __forceinline__ void store(float *dst, int nrows) const {
        float4 *d = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = threadIdx.x + i * 256;
            if (e < nrows * H / 4) d[e] = v[i];
        }
    }
};

// backprop_delta_staged for nk = H with W's rows 16-byte aligned: the next
// chunk of W rows is loaded into registers while the current one is used.
// The same products in the same order (every output the same fmaf chain).
template <int H, bool MASK>
__device__ __forceinline__ void backprop_delta_pipe(const float *__restrict__ W, int nj, const float *D,
                                                    const float *A, float *Dst, float *Wst) {
    constexpr int bk = H / 4;
    constexpr int nblk = bk * (kTsB / 4);
    static_assert(nblk <= 512, "two blocks per thread");
    float acc[2][4][4] = {};
    RowStage<H> st;
    int j0 = 0, nr = min(nj, kBwdWRows);
    st.load(W, nr);
    st.store(Wst, nr);
    __syncthreads();
    for (;;) {
        const int n0 = j0 + nr, nn = min(nj - n0, kBwdWRows);
        const bool more = n0 < nj;
        if (more) st.load(W + (size_t)n0 * H, nn);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int blk = threadIdx.x + b * 256;
            if (blk >= nblk) break;
            const int k0 = (blk % bk) * 4, s0 = (blk / bk) * 4;
            for (int r = 0; r < nr; ++r) {
                const float4 d = *reinterpret_cast<const float4 *>(D + (j0 + r) * kPadB + s0);
                const float4 w4 = *reinterpret_cast<const float4 *>(Wst + r * H + k0);
                const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[b][q][0] = fmaf(w[q], d.x, acc[b][q][0]);
                    acc[b][q][1] = fmaf(w[q], d.y, acc[b][q][1]);
                    acc[b][q][2] = fmaf(w[q], d.z, acc[b][q][2]);
                    acc[b][q][3] = fmaf(w[q], d.w, acc[b][q][3]);
                }
            }
        }
        __syncthreads();
        if (!more) break;
        st.store(Wst, nn);
        __syncthreads();
        j0 = n0;
        nr = nn;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int blk = threadIdx.x + b * 256;
        if (blk >= nblk) break;
        const int k0 = (blk % bk) * 4, s0 = (blk / bk) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 v = make_float4(acc[b][q][0], acc[b][q][1], acc[b][q][2], acc[b][q][3]);
            if (MASK) {
                const float4 a = *reinterpret_cast<const float4 *>(A + (k0 + q) * kPadB + s0);
                v.x = a.x > 0.f ? v.x : 0.f;
                v.y = a.y > 0.f ? v.y : 0.f;
                v.z = a.z > 0.f ? v.z : 0.f;
                v.w = a.w > 0.f ? v.w : 0.f;
            }
            *reinterpret_cast<float4 *>(Dst + (k0 + q) * kPadB + s0) = v;
        }
    }
}

template <int H, bool WST>
__global__ void __launch_bounds__(256) mlp_backward_f32_kernel(
    const __grid_constant__ MlpDims md, int depth, int rparam, const void *__restrict__ feats, int feat_bf16,
    const float *__restrict__ params, const float *__restrict__ packed,
    const float *__restrict__ rays, const Sample *__restrict__ samples,
    const unsigned int *__restrict__ counter, int64_t max_samples,
    const float4 *__restrict__ dout, float *__restrict__ d_feat, float *__restrict__ d_params) {
    extern __shared__ float4 smem_f4[];
    float *base = reinterpret_cast<float *>(smem_f4);
    const int in0p = (md.in0 + 3) & ~3;
    // activations: A(0) = h0 (in0p rows), A(l) = input of layer l (H rows)
    auto A = [&](int l) { return l == 0 ? base : base + in0p * kPadB + (l - 1) * H * kPadB; };
    const int dmax = in0p > H ? in0p : H;
    float *Dc = A(md.nh) + H * kPadB;  // delta of the current layer's output
    float *Dn = Dc + dmax * kPadB;     // delta one layer down (or dL/dz)
    float *Wst = Dn + dmax * kPadB;    // kBwdWRows rows of W^T (recompute)
    __shared__ int s_leaf[kTsB];
    const int64_t S = min((int64_t)counter[kCtrScene], max_samples);
    const int64_t n_tiles = (S + kTsB - 1) / kTsB;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTsB;
        if (threadIdx.x < kTsB) {
            const int64_t s = s0 + threadIdx.x;
            build_input_column(md, depth, rparam, feats, feat_bf16, rays, samples, s, S, A(0), kPadB,
                               threadIdx.x, in0p);
            s_leaf[threadIdx.x] = s < S ? samples[s].leaf : -1;
            const float4 g = s < S ? dout[s] : make_float4(0.f, 0.f, 0.f, 0.f);
            Dc[0 * kPadB + threadIdx.x] = g.x;
            Dc[1 * kPadB + threadIdx.x] = g.y;
            Dc[2 * kPadB + threadIdx.x] = g.z;
            Dc[3 * kPadB + threadIdx.x] = g.w;
        }
        __syncthreads();
        // recompute the forward (inputs of every layer), W^T staged in shared memory
        // kBwdWRows rows at a time (read from L1 / L2 instead, every K step waited on a miss)
        for (int l = 0; l < md.nh; ++l) {
            const int in = l == 0 ? md.in0 : H;
            if (!WST) {
                gemm_relu_f32<H, kTsB, 4>(A(l), in, kPadB, packed + md.wt_off[l], packed + md.b_off[l], A(l + 1),
                                          true);
                __syncthreads();
                continue;
            }
            float acc[H / 16][4];
            gemm_init<H, 4>(acc, packed + md.b_off[l]);
            // the next chunk of W^T rows is loaded into registers while the current one is used
            const float *WT = packed + md.wt_off[l];
            RowStage<H> st;
            int r0 = 0, r1 = min(in, kBwdWRows);
            st.load(WT, r1);
            st.store(Wst, r1);
            __syncthreads();
            for (;;) {
                const int n1 = min(in, r1 + kBwdWRows);
                const bool more = r1 < in;
                if (more) st.load(WT + (size_t)r1 * H, n1 - r1);
                if (r1 - r0 == kBwdWRows)
                    gemm_rows<H, kTsB, 4, true, kBwdWRows>(acc, A(l), r0, r1, kPadB, Wst);
                else
                    gemm_rows<H, kTsB, 4, true>(acc, A(l), r0, r1, kPadB, Wst);
                __syncthreads();
                if (!more) break;
                st.store(Wst, n1 - r1);
                __syncthreads();
                r0 = r1;
                r1 = n1;
            }
            gemm_store<H, kTsB, 4>(acc, A(l + 1), kPadB, true);
            __syncthreads();
        }
        // layers from the output down
        for (int l = md.nh; l >= 0; --l) {
            const int nj = (l == md.nh) ? 4 : H;
            const int nk = (l == 0) ? md.in0 : H;
            float *dW = d_params + md.w_off[l];
            float *db = dW + nj * nk;
            if (d_params) {
                if (nk % 32 == 0)
                    accumulate_dw<true>(Dc, A(l), nj, nk, dW, nk);
                else
                    accumulate_dw<false>(Dc, A(l), nj, nk, dW, nk);
                for (int j = threadIdx.x; j < nj; j += blockDim.x) {
                    float acc = 0.f;
                    for (int s = 0; s < kTsB; ++s) acc += Dc[j * kPadB + s];
                    atomicAdd(db + j, acc);
                }
            }
            const float *W = params + md.w_off[l];
            if (l > 0) {
                if (WST && H <= 128 && reinterpret_cast<uintptr_t>(W) % 16 == 0)
                    backprop_delta_pipe<H, true>(W, nj, Dc, A(l), Dn, Wst);
                else if (WST && H <= 128)
                    backprop_delta_staged<true>(W, nj, nk, nk, Dc, A(l), Dn, Wst);
                else
                    backprop_delta<true>(W, nj, nk, nk, Dc, A(l), Dn);
            } else if (d_feat) {
                if (WST && (md.F + 3) / 4 * 4 <= H)  // the staged rows fit the H-wide buffer
                    backprop_delta_staged<false>(W, nj, md.F, nk, Dc, nullptr, Dn, Wst);
                else
                    backprop_delta<false>(W, nj, md.F, nk, Dc, nullptr, Dn);
            }
            __syncthreads();
            float *t = Dc; Dc = Dn; Dn = t;
        }
        // feature gradient: Dc now holds dL/dz (F rows)
        if (d_feat) {
            for (int e = threadIdx.x; e < kTsB * md.F; e += blockDim.x) {
                const int s = e / md.F, f = e % md.F;
                const int leaf = s_leaf[s];
                if (leaf >= 0) atomicAdd(d_feat + (int64_t)leaf * md.F + f, Dc[f * kPadB + s]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- packing
__global__ void pack_f32_kernel(MlpDims md, const float *__restrict__ params,
                                float *__restrict__ packed) {
    for (int l = 0; l <= md.nh; ++l) {
        const int out = md.out_l[l], in = md.in_l[l];
        const float *W = params + md.w_off[l];
        const float *b = W + out * in;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < out * in; e += gridDim.x * blockDim.x) {
            const int j = e / in, k = e % in;
            packed[md.wt_off[l] + k * out + j] = W[e];
        }
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < out; j += gridDim.x * blockDim.x)
            packed[md.b_off[l] + j] = b[j];
    }
}

size_t packed_f32_floats(const MlpDims &md) {
    return (size_t)md.b_off[md.nh] + 4;
}

int launch_pack_f32(const MlpDims &md, const float *params, float *packed, cudaStream_t s) {
    prof_begin("pack_weights_f32", s);
    pack_f32_kernel<<<64, 256, 0, s>>>(md, params, packed);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

template <int H>
static int fwd_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb, const float *packed,
                   const float *rays, const Workspace &ws, int64_t max_samples, cudaStream_t s) {
    const int dmax = md.in0 > H ? md.in0 : H;
    // the weights-resident form where the whole packed network fits beside its activation tile
    const int pf = (int)packed_f32_floats(md);
    const size_t res = sizeof(float) * ((size_t)pf + (size_t)dmax * kTsR);
    if (res <= 227 * 1024 && pf % 4 == 0 && md.out == 4 && md.F % 4 == 0 && H % 32 == 0) {
        const auto kernel = mlp_forward_f32_res_kernel<H>;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res) != cudaSuccess)
            return SVLF_ERR_CUDA;
        prof_begin("mlp_forward_f32", s);
        kernel<<<num_sms() * (res <= 100 * 1024 ? 2 : 1), 256, res, s>>>(
            md, depth, rparam, feats, fb, packed, pf, rays, ws.samples, ws.counter, max_samples, ws.outputs);
        prof_end(s);
        return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
    }
    const size_t act = sizeof(float) * (size_t)(dmax + H) * kTsF;
    const size_t wst = sizeof(float) * (size_t)dmax * H;  // the widest layer's W^T
    if (act > 227 * 1024) return SVLF_ERR_UNSUPPORTED;    // two activation tiles do not fit
    const bool stage = act + wst <= 227 * 1024 && (md.in0 * H) % 4 == 0;
    const size_t smem = stage ? act + wst : act;
    const auto kernel = stage ? mlp_forward_f32_kernel<H, true> : mlp_forward_f32_kernel<H, false>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    int blocks = num_sms() * (smem <= 100 * 1024 ? 2 : 1);
    prof_begin("mlp_forward_f32", s);
    kernel<<<blocks, 256, smem, s>>>(md, depth, rparam, feats, fb, packed, rays, ws.samples, ws.counter,
                                     max_samples, ws.outputs);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

bool f32_forward_fits(const MlpDims &md) {
    const int H = md.H;
    if (H != 32 && H != 64 && H != 128 && H != 256) return false;
    const size_t dmax = (size_t)(md.in0 > H ? md.in0 : H);
    const size_t res = sizeof(float) * (packed_f32_floats(md) + dmax * kTsR);
    const size_t act = sizeof(float) * (dmax + (size_t)H) * kTsF;
    return res <= 227 * 1024 || act <= 227 * 1024;
}

int launch_mlp_forward_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb,
                           const float *packed, const float *rays, const Workspace &ws,
                           int64_t max_samples, cudaStream_t s) {
    switch (md.H) {
        case 32: return fwd_f32<32>(md, depth, rparam, feats, fb, packed, rays, ws, max_samples, s);
        case 64: return fwd_f32<64>(md, depth, rparam, feats, fb, packed, rays, ws, max_samples, s);
        case 128: return fwd_f32<128>(md, depth, rparam, feats, fb, packed, rays, ws, max_samples, s);
        case 256: return fwd_f32<256>(md, depth, rparam, feats, fb, packed, rays, ws, max_samples, s);
        default: return SVLF_ERR_UNSUPPORTED;
    }
}

// Shared memory of the backward: the activation and delta tiles, plus (when
// `staged`) the rows of W^T the recompute stages.
static size_t backward_f32_smem_with(const MlpDims &md, bool staged) {
    const int in0p = (md.in0 + 3) & ~3;
    const int dmax = in0p > md.H ? in0p : md.H;
    return sizeof(float) * ((size_t)kPadB * (size_t)(in0p + md.nh * md.H + 2 * dmax) +
                            (staged ? (size_t)kBwdWRows * md.H : 0));
}

size_t backward_f32_smem(const MlpDims &md) {
    return backward_f32_smem_with(md, backward_f32_smem_with(md, true) <= 220 * 1024);
}

bool f32_backward_fits(const MlpDims &md) {
    return (md.H == 32 || md.H == 64 || md.H == 128) && backward_f32_smem(md) <= 220 * 1024;
}

template <int H>
static int bwd_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb, const float *params,
                   const float *packed, const float *rays, const Workspace &ws,
                   int64_t max_samples, float *d_feat, float *d_params, cudaStream_t s) {
    const bool staged = backward_f32_smem_with(md, true) <= 220 * 1024 && (md.in0 * H) % 4 == 0;
    const size_t smem = backward_f32_smem_with(md, staged);
    if (smem > 220 * 1024) return SVLF_ERR_UNSUPPORTED;
    const auto kernel = staged ? mlp_backward_f32_kernel<H, true> : mlp_backward_f32_kernel<H, false>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    prof_begin("mlp_backward_f32", s);
    kernel<<<num_sms(), 256, smem, s>>>(md, depth, rparam, feats, fb, params, packed, rays, ws.samples, ws.counter,
                                        max_samples, ws.dout, d_feat, d_params);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

int launch_mlp_backward_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb,
                            const float *params, const float *packed, const float *rays,
                            const Workspace &ws, int64_t max_samples, float *d_feat,
                            float *d_params, cudaStream_t s) {
    switch (md.H) {
        case 32: return bwd_f32<32>(md, depth, rparam, feats, fb, params, packed, rays, ws, max_samples, d_feat, d_params, s);
        case 64: return bwd_f32<64>(md, depth, rparam, feats, fb, params, packed, rays, ws, max_samples, d_feat, d_params, s);
        case 128: return bwd_f32<128>(md, depth, rparam, feats, fb, params, packed, rays, ws, max_samples, d_feat, d_params, s);
        default: return SVLF_ERR_UNSUPPORTED;
    }
}

}  // namespace svlf
