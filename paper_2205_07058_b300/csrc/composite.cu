// Compositing (Sec. 4.3, Eq. 3), the training loss and the compositing
// backward pass. One thread per ray; a ray's samples are contiguous in the
// sample list, in hit order.
#include "svlf_internal.cuh"

namespace svlf {

// C = sum_i T_i alpha_i c_i + T_{n+1} bg,  alpha_i = 1 - exp(-tau_i),
// T_{i+1} = T_i exp(-tau_i);  D = sum_i T_i alpha_i tmid_i.
__global__ void composite_kernel(const __grid_constant__ SceneTable Tb,
                                 const int2 *__restrict__ ray_span,
                                 const Sample *__restrict__ samples,
                                 const float4 *__restrict__ outputs, float bg0, float bg1,
                                 float bg2) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Tb.total_rays;
         r += (int64_t)gridDim.x * blockDim.x) {
        const SceneDev &S = Tb.s[scene_of_ray(Tb, r)];
        const int64_t rl = r - S.ray_begin;  // ray index within its scene
        const int2 sp = ray_span[r];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
        for (int j = 0; j < sp.y; ++j) {
            const float4 o = outputs[sp.x + j];
            const float tm = samples[sp.x + j].tmid;
            const float w = T * -expm1f(-o.w);
            C0 = fmaf(w, o.x, C0);
            C1 = fmaf(w, o.y, C1);
            C2 = fmaf(w, o.z, C2);
            D = fmaf(w, tm, D);
            T *= expf(-o.w);
        }
        S.rgb[3 * rl + 0] = fmaf(T, bg0, C0);
        S.rgb[3 * rl + 1] = fmaf(T, bg1, C1);
        S.rgb[3 * rl + 2] = fmaf(T, bg2, C2);
        S.depth[rl] = D;
    }
}

// Adjoint of the compositing for one ray, given dL/dC and dL/dD:
//   dL/dc_i   = w_i dL/dC
//   dL/dtau_i = dL/dC . (T_{i+1} c_i - S_i) + dL/dD (T_{i+1} tmid_i - U_i)
// with S_i = sum_{j>i} w_j c_j + T_{n+1} bg and U_i = sum_{j>i} w_j tmid_j,
// accumulated from the back. T_i is exp(-(sum_{j<i} tau_j)) from the running
// suffix sum of tau, so no division by a small transmittance is needed.
// Then through the output activations: sigmoid'(x) = c (1 - c) for the colour
// and the ReLU step (tau > 0) for the optical thickness.
__global__ void composite_backward_kernel(const __grid_constant__ SceneTable Tb,
                                          const int2 *__restrict__ ray_span,
                                          const Sample *__restrict__ samples,
                                          const float4 *__restrict__ outputs, float bg0,
                                          float bg1, float bg2, float4 *__restrict__ dout,
                                          unsigned int *__restrict__ max_abs_bits,
                                          float *__restrict__ w_dD) {
    float gmax = 0.f;
    // the rays of the scenes that take part in the backward (scenes without
    // output gradients are skipped)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Tb.grad_rays;
         i += (int64_t)gridDim.x * blockDim.x) {
        const SceneDev &S = Tb.s[scene_of_grad_ray(Tb, i)];
        const int64_t rl = i - S.grad_begin;  // ray index within its scene
        const int64_t r = S.ray_begin + rl;
        const int2 sp = ray_span[r];
        if (sp.y == 0) continue;
        const float g0 = S.d_rgb[3 * rl + 0], g1 = S.d_rgb[3 * rl + 1], g2 = S.d_rgb[3 * rl + 2];
        const float gD = S.d_depth[rl];
        float tau_sum = 0.f;
        for (int j = 0; j < sp.y; ++j) tau_sum += outputs[sp.x + j].w;
        const float Tn = expf(-tau_sum);
        float S0 = Tn * bg0, S1 = Tn * bg1, S2 = Tn * bg2, U = 0.f, Q = 0.f;
        for (int j = sp.y - 1; j >= 0; --j) {
            const float4 o = outputs[sp.x + j];
            const float tm = samples[sp.x + j].tmid;
            const float before = tau_sum - Q - o.w;  // sum_{k<j} tau_k
            const float Ti = expf(-before);
            const float Ti1 = expf(-(before + o.w));
            const float w = Ti * -expm1f(-o.w);
            const float dtau = g0 * (Ti1 * o.x - S0) + g1 * (Ti1 * o.y - S1) +
                               g2 * (Ti1 * o.z - S2) + gD * (Ti1 * tm - U);
            float4 g;
            g.x = w * g0 * o.x * (1.f - o.x);
            g.y = w * g1 * o.y * (1.f - o.y);
            g.z = w * g2 * o.z * (1.f - o.z);
            g.w = o.w > 0.f ? dtau : 0.f;
            dout[sp.x + j] = g;
            if (w_dD) w_dD[sp.x + j] = w * gD;  // dL/d(depth parameter of the sample): D = sum_i w_i t_i
            gmax = fmaxf(gmax, fmaxf(fmaxf(fabsf(g.x), fabsf(g.y)), fmaxf(fabsf(g.z), fabsf(g.w))));
            S0 = fmaf(w, o.x, S0);
            S1 = fmaf(w, o.y, S1);
            S2 = fmaf(w, o.z, S2);
            U = fmaf(w, tm, U);
            Q += o.w;
        }
    }
    // largest |dL/d(network output)| of the launch (non-negative float bits
    // order like unsigned integers); the FP16 backward scales by it
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xFFFFFFFFu, gmax, o));
    if ((threadIdx.x & 31) == 0 && gmax > 0.f) atomicMax(max_abs_bits, __float_as_uint(gmax));
}

// L = (1/n_norm) sum_{r < n} [ |C - C*|^2 + lambda m |D - D*| ]  (n_norm = n: the mean)
__global__ void loss_kernel(const float *__restrict__ rgb, const float *__restrict__ depth,
                            const float *__restrict__ rgb_t, const float *__restrict__ depth_t,
                            const float *__restrict__ mask, int64_t n, int64_t n_norm, float lambda,
                            float *__restrict__ d_rgb, float *__restrict__ d_depth,
                            double *__restrict__ loss_accum) {
    __shared__ double red[32];
    double acc = 0.0;
    const float inv_n = 1.0f / (float)n_norm;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        float e = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float diff = rgb[3 * r + c] - rgb_t[3 * r + c];
            e = fmaf(diff, diff, e);
            d_rgb[3 * r + c] = 2.0f * diff * inv_n;
        }
        const float m = mask ? mask[r] : 1.0f;
        const float dd = depth[r] - depth_t[r];
        const float sgn = dd > 0.f ? 1.f : (dd < 0.f ? -1.f : 0.f);
        d_depth[r] = lambda * m * sgn * inv_n;
        acc += (double)e + (double)lambda * (double)m * fabs((double)dd);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
        if (threadIdx.x == 0) atomicAdd(loss_accum, acc / (double)n_norm);
    }
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

int launch_composite(const SceneTable &T, const Workspace &ws, const float bg[3], cudaStream_t s) {
    prof_begin("composite", s);
    composite_kernel<<<grid_for(T.total_rays, 256), 256, 0, s>>>(T, ws.ray_span, ws.samples,
                                                                 ws.outputs, bg[0], bg[1], bg[2]);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

int launch_composite_backward(const SceneTable &T, const Workspace &ws, const float bg[3],
                              cudaStream_t s, float *w_dD) {
    prof_begin("composite_backward", s);
    composite_backward_kernel<<<grid_for(T.grad_rays, 256), 256, 0, s>>>(
        T, ws.ray_span, ws.samples, ws.outputs, bg[0], bg[1], bg[2], ws.dout,
        ws.counter + kCtrMaxAbsDout, w_dD);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_loss_shard(const float *rgb, const float *depth, const float *rgb_target,
                               const float *depth_target, const float *mask, int64_t n, int64_t n_total,
                               float depth_weight, float *d_rgb, float *d_depth, double *loss_accum,
                               void *stream) {
    if (n <= 0 || n_total < n || !rgb || !depth || !rgb_target || !depth_target || !d_rgb || !d_depth ||
        !loss_accum)
        return SVLF_ERR_ARG;
    prof_begin("loss", (cudaStream_t)stream);
    loss_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        rgb, depth, rgb_target, depth_target, mask, n, n_total, depth_weight, d_rgb, d_depth, loss_accum);
    prof_end((cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

extern "C" int svlf_loss(const float *rgb, const float *depth, const float *rgb_target,
                         const float *depth_target, const float *mask, int64_t n,
                         float depth_weight, float *d_rgb, float *d_depth, double *loss_accum,
                         void *stream) {
    return svlf_loss_shard(rgb, depth, rgb_target, depth_target, mask, n, n, depth_weight, d_rgb, d_depth,
                           loss_accum, stream);
}
