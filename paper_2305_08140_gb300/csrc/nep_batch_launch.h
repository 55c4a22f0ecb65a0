// nep_batch_launch.h -- launchers of the batched kernels (nep_batch.cu),
// called by the C ABI in nepzbl.cu.
#pragma once

#include <cuda_runtime.h>

#include "nep_device.cuh"

namespace nepk {
struct Batch;

// Launches k_batch for precision (0 = FP32, 1 = FP64), mode (0 forward,
// 1 backward, 2 loss + gradient, 3 neighbour lists only), bt threads per CTA
// (64, 128 or 256; FP64 uses 128) and grid CTAs, then the gradient reduction
// for modes 1 and 2.
// Returns a cudaError_t.
cudaError_t launch_batch(int precision, int mode, int bt, int grid, const Model<float>& mf,
                         const Model<double>& md, const Batch& b, double* grad, cudaStream_t s);

// Resident CTAs per SM of the chosen variant.
int batch_blocks_per_sm(int precision, int mode, int bt);

// Builds the n_pop models from thetas (device [n_pop][NP]) into `models`
// (device, n_pop * model_bytes(precision)) and runs the population forward
// over the batch (lists already built) into pout [n_pop][S][3].
// With several species the pair tables go to `tables` (device, n_pop * T^2 *
// CSTR values of the precision).
cudaError_t launch_population(int precision, int n_pop, const Model<float>& mf,
                              const Model<double>& md, const double* scaler,
                              const double* thetas, void* models, void* tables, const Batch& b,
                              double* pout, int grid, cudaStream_t s);

// Loss terms of every individual: losses [n_pop][6] (np parameters each).
cudaError_t launch_population_loss(int n_pop, const double* pout, const double* thetas, int S,
                                   long long ntot, double nv, double we, double wf, double wv,
                                   double l1, double l2, double* losses, int np, cudaStream_t s);

// SNES: candidates theta_k = mu + sigma s_k; utilities and the mu/sigma update.
cudaError_t launch_snes_sample(const double* mu, const double* sigma, const double* samples,
                               int n_pop, int np, double* thetas, cudaStream_t s);
cudaError_t launch_snes_update(double* mu, double* sigma, const double* samples,
                               const double* losses, double* util, int n_pop, int np,
                               double eta_mu, double eta_sigma, cudaStream_t s);

int population_blocks_per_sm(int precision);
size_t model_bytes(int precision);
}  // namespace nepk
