// Adam (Kingma & Ba), the optimiser Sec. 4.5 trains with: one elementwise
// pass over the float32 parameters, bias-corrected, optionally refreshing a
// bfloat16 copy of the parameters that the renderer reads.
#include <cmath>

#include "svlf_internal.cuh"

namespace svlf {

// beta^step by repeated squaring in float64: the same sequence of IEEE
// multiplications on the host and on the device, so a bias correction formed
// from a device-side step count equals the one formed from a host argument.
__host__ __device__ inline double pow_step(double beta, int64_t step) {
    double r = 1.0, b = beta;
    for (int64_t e = step; e > 0; e >>= 1) {
        if (e & 1) r *= b;
        b *= b;
    }
    return r;
}

// Bias corrections 1 / (1 - beta^t) for t = *step_dev, formed once per block
// and shared through shared memory.
__device__ __forceinline__ void device_corrections(const int64_t *step_dev, float b1, float b2, float &c1,
                                                   float &c2) {
    __shared__ float s_c[2];
    if (threadIdx.x == 0) {
        const int64_t t = *step_dev < 1 ? 1 : *step_dev;
        s_c[0] = (float)(1.0 / (1.0 - pow_step((double)b1, t)));
        s_c[1] = (float)(1.0 / (1.0 - pow_step((double)b2, t)));
    }
    __syncthreads();
    c1 = s_c[0];
    c2 = s_c[1];
}

__device__ __forceinline__ float adam_update(float &pi, float gi, float &mi, float &vi, float lr,
                                             float b1, float b2, float eps, float c1, float c2) {
    mi = fmaf(b1, mi, (1.f - b1) * gi);
    vi = fmaf(b2, vi, (1.f - b2) * gi * gi);
    pi = pi - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    return pi;
}

// Four parameters per thread with 16-byte loads and stores (the optimiser is a
// pure stream: 28 bytes per parameter), plus a scalar tail.
__global__ void adam4_kernel(float4 *__restrict__ p, const float4 *__restrict__ g,
                             float4 *__restrict__ m, float4 *__restrict__ v, int64_t n4, float lr,
                             float b1, float b2, float eps, float c1, float c2,
                             uint2 *__restrict__ shadow, const int64_t *__restrict__ step_dev) {
    if (step_dev) device_corrections(step_dev, b1, b2, c1, c2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 pi = p[i], mi = m[i], vi = v[i];
        const float4 gi = __ldcs(g + i);
        adam_update(pi.x, gi.x, mi.x, vi.x, lr, b1, b2, eps, c1, c2);
        adam_update(pi.y, gi.y, mi.y, vi.y, lr, b1, b2, eps, c1, c2);
        adam_update(pi.z, gi.z, mi.z, vi.z, lr, b1, b2, eps, c1, c2);
        adam_update(pi.w, gi.w, mi.w, vi.w, lr, b1, b2, eps, c1, c2);
        p[i] = pi;
        m[i] = mi;
        v[i] = vi;
        if (shadow) {
            __nv_bfloat162 a = __floats2bfloat162_rn(pi.x, pi.y), b = __floats2bfloat162_rn(pi.z, pi.w);
            shadow[i] = make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
        }
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *__restrict__ shadow, const int64_t *__restrict__ step_dev) {
    if (step_dev) device_corrections(step_dev, b1, b2, c1, c2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (shadow) shadow[i] = __float2bfloat16_rn(pi);
    }
}

}  // namespace svlf

using namespace svlf;

namespace {

int launch_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr, float beta1,
                float beta2, float eps, float c1, float c2, const int64_t *step_dev, void *bf16_shadow,
                cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(grads) |
                      reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(bf16_shadow) % 8 == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    prof_begin("adam", s);
    if (n4 > 0) {
        int64_t blocks = (n4 + 255) / 256;
        const int64_t cap = (int64_t)num_sms() * 8;
        if (blocks > cap) blocks = cap;
        adam4_kernel<<<(unsigned)blocks, 256, 0, s>>>(
            (float4 *)params, (const float4 *)grads, (float4 *)m, (float4 *)v, n4, lr, beta1, beta2,
            eps, c1, c2, (uint2 *)bf16_shadow, step_dev);
    }
    const int64_t done = 4 * n4;
    if (done < n) {
        const int64_t rest = n - done;
        int64_t blocks = (rest + 255) / 256;
        const int64_t cap = (int64_t)num_sms() * 16;
        if (blocks > cap) blocks = cap;
        adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(
            params + done, grads + done, m + done, v + done, rest, lr, beta1, beta2, eps, c1, c2,
            bf16_shadow ? (__nv_bfloat16 *)bf16_shadow + done : nullptr, step_dev);
    }
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

__global__ void step_advance_kernel(int64_t *step) { *step += 1; }

}  // namespace

extern "C" int svlf_adam_step(float *params, const float *grads, float *m, float *v, int64_t n,
                              float lr, float beta1, float beta2, float eps, int64_t step,
                              void *bf16_shadow, void *stream) {
    if (n < 0 || step < 1 || (n > 0 && (!params || !grads || !m || !v))) return SVLF_ERR_ARG;
    if (n == 0) return SVLF_OK;
    const double c1 = 1.0 / (1.0 - pow_step((double)beta1, step));
    const double c2 = 1.0 / (1.0 - pow_step((double)beta2, step));
    return launch_adam(params, grads, m, v, n, lr, beta1, beta2, eps, (float)c1, (float)c2, nullptr, bf16_shadow,
                       (cudaStream_t)stream);
}

extern "C" int svlf_adam_step_device(float *params, const float *grads, float *m, float *v, int64_t n,
                                     float lr, float beta1, float beta2, float eps, const int64_t *step,
                                     void *bf16_shadow, void *stream) {
    if (n < 0 || !step || (n > 0 && (!params || !grads || !m || !v))) return SVLF_ERR_ARG;
    if (n == 0) return SVLF_OK;
    return launch_adam(params, grads, m, v, n, lr, beta1, beta2, eps, 0.f, 0.f, step, bf16_shadow,
                       (cudaStream_t)stream);
}

extern "C" int svlf_step_advance(int64_t *step, void *stream) {
    if (!step) return SVLF_ERR_ARG;
    step_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(step);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}
