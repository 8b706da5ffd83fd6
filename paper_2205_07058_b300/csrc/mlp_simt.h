// Shape limits of the FP32 SIMT network kernels (mlp_simt.cu), checked
// before a call queues any work.
#pragma once

#include "mlp_common.cuh"

namespace svlf {

// The forward's shared memory fits: the whole packed network beside one
// 128-sample activation tile, or two activation tiles (each layer's W^T then
// staged or read through the cache).
bool f32_forward_fits(const MlpDims &md);

// The backward's shared memory fits: every layer's activations and two delta
// tiles for 64 samples (hidden width <= 128).
bool f32_backward_fits(const MlpDims &md);

}  // namespace svlf
