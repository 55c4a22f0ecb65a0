// nep_batch.cu -- instantiations and launchers of the batched kernels.
#include "nep_batch.cuh"
#include "nep_batch_launch.h"

namespace nepk {

template <typename R, int BT, bool MS>
static cudaError_t run(int mode, int grid, const Model<R>& P, const Batch& b, double* grad,
                       cudaStream_t s)
{
    switch (mode) {
    case MODE_FORWARD: k_batch<R, MODE_FORWARD, BT, MS><<<grid, BT, 0, s>>>(P, b); break;
    case MODE_BACKWARD: k_batch<R, MODE_BACKWARD, BT, MS><<<grid, BT, 0, s>>>(P, b); break;
    case MODE_LISTS: k_batch<R, MODE_LISTS, BT, false><<<grid, BT, 0, s>>>(P, b); break;
    default: k_batch<R, MODE_LOSS, BT, MS><<<grid, BT, 0, s>>>(P, b); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode == MODE_BACKWARD || mode == MODE_LOSS) {
        k_batch_grad_reduce<<<(b.np + 255) / 256, 256, 0, s>>>(b.gpart, b.S, b.np, grad);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_batch(int precision, int mode, int bt, int grid, const Model<float>& mf,
                         const Model<double>& md, const Batch& b, double* grad, cudaStream_t s)
{
    // several species: one configuration of 128 threads per CTA
    if (b.T > 1) {
        if (precision == 1) return run<double, 128, true>(mode, grid, md, b, grad, s);
        return run<float, 128, true>(mode, grid, mf, b, grad, s);
    }
    if (precision == 1) return run<double, 128, false>(mode, grid, md, b, grad, s);
    if (bt == 64) return run<float, 64, false>(mode, grid, mf, b, grad, s);
    if (bt == 256) return run<float, 256, false>(mode, grid, mf, b, grad, s);
    return run<float, 128, false>(mode, grid, mf, b, grad, s);
}

cudaError_t launch_population(int precision, int n_pop, const Model<float>& mf,
                              const Model<double>& md, const double* scaler,
                              const double* thetas, void* models, void* tables, const Batch& b,
                              double* pout, int grid, cudaStream_t s)
{
    const bool ms = b.T > 1;
    if (precision == 1) {
        k_build_models<double><<<n_pop, 256, 0, s>>>(md, scaler, thetas, (Model<double>*)models,
                                                    b.np, b.T, (double*)tables);
        if (ms)
            k_batch_pop<double, 128, true><<<grid, 128, 0, s>>>(
                (const Model<double>*)models, n_pop, b, pout, (const double*)tables);
        else
            k_batch_pop<double, 128, false><<<grid, 128, 0, s>>>(
                (const Model<double>*)models, n_pop, b, pout, nullptr);
    } else {
        k_build_models<float><<<n_pop, 256, 0, s>>>(mf, scaler, thetas, (Model<float>*)models,
                                                   b.np, b.T, (float*)tables);
        if (ms)
            k_batch_pop<float, 128, true><<<grid, 128, 0, s>>>(
                (const Model<float>*)models, n_pop, b, pout, (const float*)tables);
        else
            k_batch_pop<float, 128, false><<<grid, 128, 0, s>>>(
                (const Model<float>*)models, n_pop, b, pout, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_population_loss(int n_pop, const double* pout, const double* thetas, int S,
                                   long long ntot, double nv, double we, double wf, double wv,
                                   double l1, double l2, double* losses, int np, cudaStream_t s)
{
    k_pop_loss<256><<<n_pop, 256, 0, s>>>(pout, thetas, S, ntot, nv, we, wf, wv, l1, l2, losses,
                                          np);
    return cudaGetLastError();
}

cudaError_t launch_snes_sample(const double* mu, const double* sigma, const double* samples,
                               int n_pop, int np, double* thetas, cudaStream_t s)
{
    const long long n = (long long)n_pop * np;
    k_snes_sample<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mu, sigma, samples, n_pop, np,
                                                              thetas);
    return cudaGetLastError();
}

cudaError_t launch_snes_update(double* mu, double* sigma, const double* samples,
                               const double* losses, double* util, int n_pop, int np,
                               double eta_mu, double eta_sigma, cudaStream_t s)
{
    k_snes_utilities<<<1, 1024, 0, s>>>(losses, n_pop, util);
    k_snes_update<<<(np + 255) / 256, 256, 0, s>>>(mu, sigma, samples, util, n_pop, np, eta_mu,
                                                  eta_sigma);
    return cudaGetLastError();
}

int population_blocks_per_sm(int precision)
{
    int n = 0;
    cudaError_t e = precision == 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_pop<double, 128, false>, 128, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_pop<float, 128, false>, 128, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

size_t model_bytes(int precision)
{
    return precision == 1 ? sizeof(Model<double>) : sizeof(Model<float>);
}

template <typename K>
static int occ(K kernel, int bt)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, bt, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

int batch_blocks_per_sm(int precision, int mode, int bt)
{
    if (precision == 1) {
        if (mode == MODE_FORWARD) return occ(k_batch<double, MODE_FORWARD, 128, false>, 128);
        if (mode == MODE_BACKWARD) return occ(k_batch<double, MODE_BACKWARD, 128, false>, 128);
        return occ(k_batch<double, MODE_LOSS, 128, false>, 128);
    }
#define NEP_OCC(BT_)                                                            \
    if (bt == BT_) {                                                            \
        if (mode == MODE_FORWARD) return occ(k_batch<float, MODE_FORWARD, BT_, false>, BT_);   \
        if (mode == MODE_BACKWARD) return occ(k_batch<float, MODE_BACKWARD, BT_, false>, BT_); \
        return occ(k_batch<float, MODE_LOSS, BT_, false>, BT_);                       \
    }
    NEP_OCC(64)
    NEP_OCC(256)
#undef NEP_OCC
    if (mode == MODE_FORWARD) return occ(k_batch<float, MODE_FORWARD, 128, false>, 128);
    if (mode == MODE_BACKWARD) return occ(k_batch<float, MODE_BACKWARD, 128, false>, 128);
    return occ(k_batch<float, MODE_LOSS, 128, false>, 128);
}

}  // namespace nepk
