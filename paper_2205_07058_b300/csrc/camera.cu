// Pinhole ray generation on the device (row a1's optional in-kernel ray
// generation): one thread per pixel writes its ray (origin, unit direction)
// in the layout svlf_render_rays reads.
#include "svlf_internal.cuh"

namespace svlf {

constexpr int kMaxCams = 64;  // cameras per launch (parameter space)

struct CamTable {
    svlf_camera cam[kMaxCams];
};

__global__ void pinhole_kernel(const __grid_constant__ CamTable C, int n_views, int width, int height,
                               float *__restrict__ rays) {
    const int64_t per_view = (int64_t)width * height;
    const int64_t n = per_view * n_views;
    const float sx = 2.0f / (float)width, sy = 2.0f / (float)height;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / per_view);
        const int64_t p = i - (int64_t)v * per_view;
        const int r = (int)(p / width), c = (int)(p - (int64_t)r * width);
        const svlf_camera &cm = C.cam[v];
        const float x = fmaf((float)c + 0.5f, sx, -1.0f) * cm.tan_half_fov;
        const float y = fmaf(-((float)r + 0.5f), sy, 1.0f) * cm.tan_half_fov;
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = fmaf(y, cm.up[a], fmaf(x, cm.right[a], cm.fwd[a]));
        const float inv = 1.0f / sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
        float2 *o = reinterpret_cast<float2 *>(rays + 6 * i);
        o[0] = make_float2(cm.eye[0], cm.eye[1]);
        o[1] = make_float2(cm.eye[2], d[0] * inv);
        o[2] = make_float2(d[1] * inv, d[2] * inv);
    }
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_pinhole_rays(const svlf_camera *cams, int n_views, int width, int height, float *rays_out,
                                 void *stream) {
    if (!cams || !rays_out || n_views < 1 || width < 1 || height < 1) return SVLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(rays_out) % 8) return SVLF_ERR_ARG;
    for (int v0 = 0; v0 < n_views; v0 += kMaxCams) {
        const int nv = n_views - v0 < kMaxCams ? n_views - v0 : kMaxCams;
        CamTable C;
        for (int i = 0; i < nv; ++i) C.cam[i] = cams[v0 + i];
        const int64_t n = (int64_t)width * height * nv;
        const int64_t blocks = (n + 255) / 256;
        const int64_t cap = (int64_t)num_sms() * 16;
        pinhole_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, (cudaStream_t)stream>>>(
            C, nv, width, height, rays_out + (int64_t)v0 * width * height * 6);
        if (cudaGetLastError() != cudaSuccess) return SVLF_ERR_CUDA;
    }
    return SVLF_OK;
}
