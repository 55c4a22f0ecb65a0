// nep_batch_launch.h -- launchers of the batched kernels (nep_batch.cu),
// called by the C ABI in nepzbl.cu.
#pragma once

#include <cuda_runtime.h>

#include "nep_device.cuh"

namespace nepk {
struct Batch;

// Launches k_batch for precision (0 = FP32, 1 = FP64), mode (0 forward,
// 1 backward, 2 loss + gradient), bt threads per CTA (64, 128 or 256; FP64
// uses 128) and grid CTAs, then the gradient reduction when mode != 0.
// Returns a cudaError_t.
cudaError_t launch_batch(int precision, int mode, int bt, int grid, const Model<float>& mf,
                         const Model<double>& md, const Batch& b, double* grad, cudaStream_t s);

// Resident CTAs per SM of the chosen variant.
int batch_blocks_per_sm(int precision, int mode, int bt);
}  // namespace nepk
