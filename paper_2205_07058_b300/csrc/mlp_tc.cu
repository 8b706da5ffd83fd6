// Tensor-core (tcgen05) network path. Placeholder until the kernels land.
#include "svlf_internal.cuh"
#include "mlp_common.cuh"

namespace svlf {
bool tc_supported(const MlpDims &md) { return false; }
size_t packed_tc_bytes(const MlpDims &md) { return 0; }
int launch_pack_tc(const MlpDims &, int, const float *, void *, cudaStream_t) { return SVLF_ERR_UNSUPPORTED; }
int launch_mlp_forward_tc(const MlpDims &, int, int, const void *, int, const void *, const float *,
                          const Workspace &, int64_t, cudaStream_t) { return SVLF_ERR_UNSUPPORTED; }
int launch_mlp_backward_tc(const MlpDims &, int, int, const void *, int, const void *,
                           const float *, const Workspace &, int64_t, float *, float *,
                           cudaStream_t) { return SVLF_ERR_UNSUPPORTED; }
}  // namespace svlf
