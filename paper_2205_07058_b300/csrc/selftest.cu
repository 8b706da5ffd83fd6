// Self-test of the tensor-core operand layouts: one 128 x N x K product
// D = A B^T through tcgen05.mma, with either operand in K-major or MN-major
// shared-memory layout, or with A in tensor memory (flags bit 5). Test aid
// for the descriptor conventions the network kernels rely on; not part of the
// rendering method.
#include "svlf_internal.cuh"
#include "tc_common.cuh"

namespace svlf {

__global__ void __launch_bounds__(128, 1) mma_selftest_kernel(const uint16_t *__restrict__ A,
                                                              const uint16_t *__restrict__ B,
                                                              float *__restrict__ D, int N, int K,
                                                              int a_mn, int b_mn, int bf16,
                                                              int flags) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    // flags: bit 0 swap the two descriptor byte offsets, bit 1 place B before A,
    // bit 2 / bit 3 start the B / A descriptor 16 bytes later, bit 5 A from
    // TMEM columns 256 .. 256 + K/2 (packed pairs) instead of shared memory
    const int swap = flags & 1;
    const bool a_tm = (flags & 32) != 0;
    const int gap = (flags >> 8) & 0xFFFF;  // bytes between the two staged operands
    uint8_t *sa = (flags & 2) ? smem + N * K * 2 + gap : smem;
    uint8_t *sb = (flags & 2) ? smem : smem + 128 * K * 2 + gap;
    const uint32_t adj_b = (flags & 4) ? 16u : 0u, adj_a = (flags & 8) ? 16u : 0u;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0 && (flags & 16)) D[0] = (float)tc::smem_u32(smem);
    for (int e = tid; e < 128 * K; e += 128) {
        const int m = e / K, k = e % K;
        const uint32_t off = a_mn ? tc::cm_offset(k, m, K) : tc::cm_offset(m, k, 128);
        *reinterpret_cast<uint16_t *>(sa + off) = A[e];
    }
    for (int e = tid; e < N * K; e += 128) {
        const int n = e / K, k = e % K;
        const uint32_t off = b_mn ? tc::cm_offset(k, n, K) : tc::cm_offset(n, k, N);
        *reinterpret_cast<uint16_t *>(sb + off) = B[e];
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&s_mbar), 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&s_tmem), 512);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (a_tm) {
        // row tid of A -> TMEM lane tid, elements (2j, 2j+1) in column 256 + j
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + 256u;
        for (int c = 0; c < K / 2; c += 32) {
            uint32_t v[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int j = c + e;
                v[e] = j < K / 2 ? (uint32_t)A[tid * K + 2 * j] | ((uint32_t)A[tid * K + 2 * j + 1] << 16) : 0u;
            }
            tc::tmem_st32(trow + (uint32_t)c, v);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(128, N, bf16, a_mn, b_mn);
        for (int k = 0; k < K; k += 16) {
            // (leading, stride) byte offsets: K-direction and M/N-direction core-matrix steps
            uint32_t la = a_mn ? 128u : 2048u, sa_ = a_mn ? (uint32_t)K * 16 : 128u;
            uint32_t lb = b_mn ? 128u : (uint32_t)N * 16, sb_ = b_mn ? (uint32_t)K * 16 : 128u;
            if (swap) {
                uint32_t t = la; la = sa_; sa_ = t;
                t = lb; lb = sb_; sb_ = t;
            }
            const uint64_t da = tc::sdesc(tc::smem_u32(sa) + adj_a + (k >> 3) * (a_mn ? 128 : 2048), la, sa_);
            const uint64_t db = tc::sdesc(tc::smem_u32(sb) + adj_b + (k >> 3) * (b_mn ? 128 : N * 16), lb, sb_);
            if (a_tm)
                tc::mma_f16_ta(tmem, tmem + 256u + (uint32_t)(k >> 1), db, idesc, k > 0 ? 1u : 0u);
            else
                tc::mma_f16(tmem, da, db, idesc, k > 0 ? 1u : 0u);
        }
        tc::mma_commit(tc::smem_u32(&s_mbar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&s_mbar), 0, 200000000ll);
    if (!ok && tid == 0) raise_status(SVLF_DEV_WAIT_TIMEOUT);
    tc::fence_after_sync();
    if (ok && !(flags & 16)) {
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < N; c += 32) {
            uint32_t v[32];
            tc::tmem_ld32_wait(trow + c, v);
            for (int e = 0; e < 32 && c + e < N; ++e) D[tid * N + c + e] = __uint_as_float(v[e]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_selftest_mma(const uint16_t *A, const uint16_t *B, float *D, int N, int K,
                                 int a_mn_major, int b_mn_major, int bf16, int flags,
                                 void *stream) {
    if (!A || !B || !D || N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16)
        return SVLF_ERR_ARG;
    if ((flags & 32) && a_mn_major) return SVLF_ERR_ARG;  // A in TMEM is K-major only
    // Generous on purpose: every read the descriptors can address stays inside
    // the allocation even if a layout were misread.
    const size_t need = (size_t)(128 + N) * K * 2 + ((flags >> 8) & 0xFFFF) + 128;
    const size_t smem = need > 200 * 1024 ? need : 200 * 1024;
    if (cudaFuncSetAttribute(mma_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return SVLF_ERR_CUDA;
    mma_selftest_kernel<<<1, 128, smem, (cudaStream_t)stream>>>(A, B, D, N, K, a_mn_major,
                                                                 b_mn_major, bf16, flags);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

// ---------------------------------------------------------------- FP32 FMA rate
namespace svlf {
__global__ void __launch_bounds__(256) ffma_kernel(float *__restrict__ out, int64_t iters, float a, float b) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    if (s == -1.2345f) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}
}  // namespace svlf

extern "C" int svlf_selftest_ffma(float *out, int blocks, int64_t iters, void *stream) {
    if (!out || blocks < 1 || iters < 1) return SVLF_ERR_ARG;
    svlf::ffma_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-4f);
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}

// ---------------------------------------------------------------- bounded waits
namespace svlf {
// One thread waits on an mbarrier (arrival count 1) that nothing arrives at
// unless `arrive` is set, giving up after `limit_cycles` SM clocks: the
// bounded wait every kernel of the library uses, and the status a kernel
// latches when a copy or an MMA it waits for does not complete. The kernel
// returns either way, so the context stays usable. out[0] = 1 if the phase
// completed, 0 if the wait gave up; out[1] = clocks spent waiting.
__global__ void __launch_bounds__(32) wait_selftest_kernel(long long limit_cycles, int arrive,
                                                           long long *__restrict__ out) {
    __shared__ __align__(8) uint64_t s_mbar;
    if (threadIdx.x != 0) return;
    const uint32_t mb = tc::smem_u32(&s_mbar);
    tc::mbar_init(mb, 1);
    tc::mbar_init_fence();
    if (arrive) tc::mbar_arrive(mb);
    const long long t0 = clock64();
    const bool ok = tc::mbar_wait(mb, 0, limit_cycles);
    const long long t1 = clock64();
    if (!ok) raise_status(SVLF_DEV_WAIT_TIMEOUT);
    out[0] = ok ? 1 : 0;
    out[1] = t1 - t0;
}
}  // namespace svlf

extern "C" int svlf_selftest_wait(int64_t limit_cycles, int arrive, int64_t *out, void *stream) {
    if (!out || limit_cycles < 1 || limit_cycles > (int64_t)4000000000ll) return SVLF_ERR_ARG;
    svlf::wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles, arrive ? 1 : 0,
                                                                    reinterpret_cast<long long *>(out));
    return cudaGetLastError() == cudaSuccess ? SVLF_OK : SVLF_ERR_CUDA;
}
