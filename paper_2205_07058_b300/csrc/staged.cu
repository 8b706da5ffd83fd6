// Staged training of the two-decoder form (Sec. 4.4, Eq. 4).
//
//  * Stage 1 ("voxel training", surface rendering): each ray with a known
//    surface depth D* is evaluated at one voxel, the leaf containing
//    x* = o + D* d. surface_samples_kernel finds it with a point lookup (the
//    dense parent index, then the brick mask) instead of a traversal, and
//    appends one sample per ray; the two decoders run on those samples, and
//    surface_loss_kernel forms Eq. 4,
//        L = (1/N) sum_v |c_v - c*|^2 + l_eta (eta_v - eta*)^2 + l_tau e^{-2 tau_v},
//    with eta* the within-voxel depth of x* on the ray's segment
//    (x* = eta* x1 + (1 - eta*) x2), and the gradients the two-decoder
//    backward consumes: dL/d(colour pre-activation), dL/d(tau_pre), and a
//    direct dL/d(eta) per sample.
//  * Stages 2-3 (volumetric): eta_term_kernel adds l_eta (eta_v - eta*)^2 / N
//    for each ray's surface voxel among its hits (the first hit whose
//    segment contains D*) after a two-decoder render, and records its direct
//    dL/d(eta) for the backward.
#include "svlf_internal.cuh"

namespace svlf {

// Rank of the leaf at finest cell c (0 <= c < 2^L), or -1 if the cell is empty.
__device__ __forceinline__ int leaf_of_cell(const OctreeView &T, const int c[3]) {
    if (T.empty) return -1;
    int node = 0;
    if (T.n_node_levels > 0) {
        const int ps = T.pgrid_shift;
        const uint32_t pidx = (uint32_t)(c[0] >> 3) | ((uint32_t)(c[1] >> 3) << ps) | ((uint32_t)(c[2] >> 3) << (2 * ps));
        const uint32_t pw = __ldg(&T.pgrid[pidx].x);
        const uint32_t m = pw >> 24;
        const int oct = ((c[0] >> 2) & 1) | (((c[1] >> 2) & 1) << 1) | (((c[2] >> 2) & 1) << 2);
        if (!((m >> oct) & 1u)) return -1;
        node = (int)(pw & 0xFFFFFFu) + __popc(m & ((1u << oct) - 1u));
    }
    if (node >= T.n_bricks) return -1;
    const uint4 b = __ldg(T.bricks + node);
    const uint64_t mask = (uint64_t)b.x | ((uint64_t)b.y << 32);
    const int bit = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2) | (((c[0] >> 1) & 1) << 3) |
                    (((c[1] >> 1) & 1) << 4) | (((c[2] >> 1) & 1) << 5);
    if (!((mask >> bit) & 1ull)) return -1;
    return (int)b.z + __popcll(mask & ((1ull << bit) - 1ull));
}

__device__ __forceinline__ float eta_target(float t_in, float t_out, float t_star) {
    return fminf(fmaxf((t_out - t_star) / (t_out - t_in), 0.f), 1.f);
}

// One sample per ray with a surface depth whose voxel is a leaf; appended with
// one atomic per warp. eta_gt[sample] = eta*.
__global__ void surface_samples_kernel(const __grid_constant__ SceneTable T, const float *__restrict__ depth_t,
                                       const float *__restrict__ mask, Sample *__restrict__ samples,
                                       float *__restrict__ eta_gt, unsigned int *__restrict__ counter) {
    const SceneDev &S = T.s[0];
    const OctreeView &tree = S.tree;
    const int n = 1 << tree.depth;
    const float fn = (float)n, h = ldexpf(1.0f, -tree.depth);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < S.n_rays; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = base + threadIdx.x;
        bool keep = false;
        int leaf = -1, cell[3] = {0, 0, 0};
        float t0 = 0.f, t1 = 0.f, eg = 0.f;
        if (r < S.n_rays) {
            const float ts = depth_t[r];
            const float m = mask ? mask[r] : 1.f;
            if (m > 0.f && isfinite(ts)) {
                const float2 *rp = reinterpret_cast<const float2 *>(S.rays + 6 * r);
                const float2 ra = __ldg(rp), rb = __ldg(rp + 1), rc = __ldg(rp + 2);
                const float o[3] = {ra.x, ra.y, rb.x};
                const float d[3] = {rb.y, rc.x, rc.y};
                for (int a = 0; a < 3; ++a)
                    cell[a] = min(max((int)floorf(fmaf(ts, d[a], o[a]) * fn), 0), n - 1);
                leaf = leaf_of_cell(tree, cell);
                if (leaf >= 0) {
                    t0 = 0.f;
                    t1 = INFINITY;
                    for (int a = 0; a < 3; ++a) {
                        if (d[a] == 0.f) continue;
                        const float lo = ((float)cell[a] * h - o[a]) / d[a];
                        const float hi = ((float)(cell[a] + 1) * h - o[a]) / d[a];
                        t0 = fmaxf(t0, fminf(lo, hi));
                        t1 = fminf(t1, fmaxf(lo, hi));
                    }
                    keep = t1 > t0;
                    eg = eta_target(t0, t1, ts);
                }
            }
        }
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, keep);
        unsigned int wbase = 0;
        if (lane == 0 && ballot) wbase = atomicAdd(counter + kCtrScene, (unsigned)__popc(ballot));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (keep) {
            const unsigned idx = wbase + __popc(ballot & ((1u << lane) - 1u));
            const uint32_t packed = (uint32_t)cell[0] | ((uint32_t)cell[1] << 10) | ((uint32_t)cell[2] << 20);
            samples[idx] = Sample{leaf, (int32_t)r, packed, 0.5f * (t0 + t1)};
            eta_gt[idx] = eg;
        }
    }
}

// Eq. 4 over the surface samples; deta holds eta* on entry and the direct
// dL/d(eta) on exit; w_dD is cleared (no depth term).
__global__ void surface_loss_kernel(const Sample *__restrict__ samples, const unsigned int *__restrict__ counter,
                                    const float4 *__restrict__ outputs, const float4 *__restrict__ aux,
                                    const float *__restrict__ rgb_t, int64_t n_rays, float lam_eta, float lam_tau,
                                    float4 *__restrict__ dout, float *__restrict__ deta, float *__restrict__ w_dD,
                                    unsigned int *__restrict__ max_abs_bits, double *__restrict__ loss_accum) {
    __shared__ double red[32];
    const unsigned int S = counter[kCtrScene];
    const float inv_n = 1.0f / (float)n_rays;
    double acc = 0.0;
    float gmax = 0.f;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        const float4 c = outputs[i];  // colour, tau
        const float4 a = aux[i];      // tau, eta, t_in, t_out
        const int r = samples[i].ray;
        const float e0 = c.x - rgb_t[3 * r], e1 = c.y - rgb_t[3 * r + 1], e2 = c.z - rgb_t[3 * r + 2];
        const float de = a.y - deta[i];
        const float et2 = expf(-2.f * a.x);
        acc += (double)(e0 * e0 + e1 * e1 + e2 * e2) + (double)lam_eta * de * de + (double)lam_tau * et2;
        float4 g;
        g.x = 2.f * e0 * inv_n * c.x * (1.f - c.x);
        g.y = 2.f * e1 * inv_n * c.y * (1.f - c.y);
        g.z = 2.f * e2 * inv_n * c.z * (1.f - c.z);
        g.w = a.x > 0.f ? -2.f * lam_tau * et2 * inv_n : 0.f;  // through tau = relu(tau_pre)
        dout[i] = g;
        deta[i] = 2.f * lam_eta * de * inv_n;
        w_dD[i] = 0.f;
        gmax = fmaxf(gmax, fmaxf(fmaxf(fabsf(g.x), fabsf(g.y)), fmaxf(fabsf(g.z), fabsf(g.w))));
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        gmax = fmaxf(gmax, __shfl_xor_sync(0xFFFFFFFFu, gmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = acc;
        if (gmax > 0.f) atomicMax(max_abs_bits, __float_as_uint(gmax));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss_accum, acc / (double)n_rays);
    }
}

// Stages 2-3: the eta term on each ray's first hit whose segment contains D*.
__global__ void eta_term_kernel(const __grid_constant__ SceneTable T, const int2 *__restrict__ ray_span,
                                const float4 *__restrict__ aux, const float *__restrict__ depth_t,
                                const float *__restrict__ mask, float lam_eta, float *__restrict__ deta,
                                double *__restrict__ loss_accum) {
    __shared__ double red[32];
    const SceneDev &S = T.s[0];
    const float inv_n = 1.0f / (float)S.n_rays;
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < S.n_rays;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float m = mask ? mask[r] : 1.f;
        const float ts = depth_t[r];
        if (!(m > 0.f) || !isfinite(ts)) continue;
        const int2 sp = ray_span[r];
        for (int j = 0; j < sp.y; ++j) {
            const float4 a = aux[sp.x + j];
            if (a.z <= ts && ts <= a.w && a.w > a.z) {
                const float de = a.y - eta_target(a.z, a.w, ts);
                acc += (double)lam_eta * de * de;
                deta[sp.x + j] = 2.f * lam_eta * de * inv_n;
                break;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss_accum, acc / (double)S.n_rays);
    }
}

static unsigned grid_of(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

int launch_surface_samples(const SceneTable &T, const float *depth_t, const float *mask, Sample *samples,
                           float *eta_gt, unsigned int *counter, cudaStream_t s) {
    prof_begin("surface_samples", s);
    surface_samples_kernel<<<grid_of(T.s[0].n_rays, 256), 256, 0, s>>>(T, depth_t, mask, samples, eta_gt, counter);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

int launch_surface_loss(const Sample *samples, const unsigned int *counter, const float4 *outputs,
                        const float4 *aux, const float *rgb_t, int64_t n_rays, float lam_eta, float lam_tau,
                        float4 *dout, float *deta, float *w_dD, unsigned int *max_abs_bits, double *loss_accum,
                        cudaStream_t s) {
    prof_begin("surface_loss", s);
    surface_loss_kernel<<<grid_of(n_rays, 256), 256, 0, s>>>(samples, counter, outputs, aux, rgb_t, n_rays, lam_eta,
                                                               lam_tau, dout, deta, w_dD, max_abs_bits, loss_accum);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

int launch_eta_term(const SceneTable &T, const int2 *ray_span, const float4 *aux, const float *depth_t,
                    const float *mask, float lam_eta, float *deta, double *loss_accum, cudaStream_t s) {
    prof_begin("eta_term", s);
    eta_term_kernel<<<grid_of(T.s[0].n_rays, 256), 256, 0, s>>>(T, ray_span, aux, depth_t, mask, lam_eta, deta,
                                                                  loss_accum);
    prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

}  // namespace svlf
