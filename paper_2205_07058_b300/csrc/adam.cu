// Adam (Kingma & Ba), the optimiser Sec. 4.5 trains with: one elementwise
// pass over the float32 parameters, bias-corrected, optionally refreshing a
// bfloat16 copy of the parameters that the renderer reads.
#include <cmath>

#include "svlf_internal.cuh"

namespace svlf {

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *__restrict__ shadow) {
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

extern "C" int svlf_adam_step(float *params, const float *grads, float *m, float *v, int64_t n,
                              float lr, float beta1, float beta2, float eps, int64_t step,
                              void *bf16_shadow, void *stream) {
    if (n < 0 || step < 1 || (n > 0 && (!params || !grads || !m || !v))) return SVLF_ERR_ARG;
    if (n == 0) return SVLF_OK;
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, (double)step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, (double)step));
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    prof_begin("adam", (cudaStream_t)stream);
    adam_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        params, grads, m, v, n, lr, beta1, beta2, eps, (float)c1, (float)c2,
        (__nv_bfloat16 *)bf16_shadow);
    prof_end((cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}
