// Network shapes and the per-sample input/output shared by the SIMT and the
// tensor-core network kernels.
#pragma once

#include "svlf_internal.cuh"

namespace svlf {

constexpr int kMaxLayers = 8;     // n_hidden <= 6 plus the output layer
constexpr int kMaxIn = 64 + 9;    // feat_dim <= 64

struct MlpDims {
    int F, in0, H, nh;
    int out;                 // output width (4: colour + tau; two-decoder: 2 or 3)
    int in_l[kMaxLayers], out_l[kMaxLayers];
    int w_off[kMaxLayers];   // W_l in the flat parameters (b_l follows it)
    int wt_off[kMaxLayers];  // W_l^T in the packed float32 buffer
    int b_off[kMaxLayers];   // b_l in the packed float32 buffer
};

MlpDims make_dims(const svlf_mlp_desc &d);
// a network of feature width F, input width in0, nh hidden layers of H, out outputs
MlpDims make_dims_io(int F, int in0, int H, int nh, int out);
size_t packed_f32_floats(const MlpDims &md);
int launch_pack_f32(const MlpDims &md, const float *params, float *packed, cudaStream_t s);
int launch_mlp_forward_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb,
                           const float *packed, const float *rays, const Workspace &ws,
                           int64_t max_samples, cudaStream_t s);
int launch_mlp_backward_f32(const MlpDims &md, int depth, int rparam, const void *feats, int fb,
                            const float *params, const float *packed, const float *rays,
                            const Workspace &ws, int64_t max_samples, float *d_feat,
                            float *d_params, cudaStream_t s);
size_t backward_f32_smem(const MlpDims &md);

// h0 = [z | d | p~1 | p~2] of one sample, in float32 (rparam: SVLF_RPARAM_*),
// value k written to h0[k * stride] (a column of a feature-major tile).
__device__ __forceinline__ void make_input_row(const MlpDims &md, int depth, int rparam, const void *feats,
                                               int feat_bf16, const float *rays, const Sample &sm,
                                               float *h0, int stride) {
    const int F = md.F;
    if (feat_bf16) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            reinterpret_cast<const __nv_bfloat16 *>(feats) + (int64_t)sm.leaf * F);
        for (int q = 0; q < F / 8; ++q) {
            const uint4 v = __ldg(src + q);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                h0[(8 * q + 2 * e) * stride] = __uint_as_float(w[e] << 16);
                h0[(8 * q + 2 * e + 1) * stride] = __uint_as_float(w[e] & 0xFFFF0000u);
            }
        }
    } else {
        const float4 *src = reinterpret_cast<const float4 *>(
            reinterpret_cast<const float *>(feats) + (int64_t)sm.leaf * F);
        for (int q = 0; q < F / 4; ++q) {
            const float4 v = __ldg(src + q);
            h0[(4 * q) * stride] = v.x;
            h0[(4 * q + 1) * stride] = v.y;
            h0[(4 * q + 2) * stride] = v.z;
            h0[(4 * q + 3) * stride] = v.w;
        }
    }
    const float2 *rp = reinterpret_cast<const float2 *>(rays + 6 * (int64_t)sm.ray);
    const float2 a = __ldg(rp), b = __ldg(rp + 1), c = __ldg(rp + 2);
    const float o[3] = {a.x, a.y, b.x};
    const float d[3] = {b.y, c.x, c.y};
    float p1[3], p2[3];
    voxel_param_at(rparam, o, d, sm.tmid, sm.cell, depth, p1, p2);
    h0[(F + 0) * stride] = d[0]; h0[(F + 1) * stride] = d[1]; h0[(F + 2) * stride] = d[2];
    h0[(F + 3) * stride] = p1[0]; h0[(F + 4) * stride] = p1[1]; h0[(F + 5) * stride] = p1[2];
    h0[(F + 6) * stride] = p2[0]; h0[(F + 7) * stride] = p2[1]; h0[(F + 8) * stride] = p2[2];
}

// colour = sigmoid(o[0:3]), optical thickness tau = max(o[3], 0) (Sec. 4.5)
__device__ __forceinline__ float4 output_activation(float o0, float o1, float o2, float o3) {
    return make_float4(sigmoidf_(o0), sigmoidf_(o1), sigmoidf_(o2), fmaxf(o3, 0.f));
}

}  // namespace svlf

namespace svlf {
// tensor-core (tcgen05) network path, mlp_tc.cu
bool tc_supported(const MlpDims &md);
bool tc_backward_supported(const MlpDims &md);
size_t packed_tc_bytes(const MlpDims &md);
void set_tc_warpgroups(int n);
int launch_pack_tc(const MlpDims &md, int precision, const SceneTable &T, void *packed,
                   size_t stride, cudaStream_t s);
// mode 0: the single network; 1 / 2: the two-decoder form's F^T / F^C pass
// (aux: per-sample (tau, eta, t_in, t_out), written by mode 1, read by mode 2)
int launch_mlp_forward_tc(const MlpDims &md, int precision, int fb, const SceneTable &T,
                          const Workspace &ws, cudaStream_t s, int mode = 0, float4 *aux = nullptr);
int launch_mlp_backward_tc(const MlpDims &md, int precision, int fb, const SceneTable &T,
                           const Workspace &ws, bool want_feat, bool want_params, cudaStream_t s,
                           int mode = 0, float4 *aux = nullptr, const float *w_dD = nullptr,
                           const float *deta = nullptr);
}  // namespace svlf
