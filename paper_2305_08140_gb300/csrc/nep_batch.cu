// nep_batch.cu -- instantiations and launchers of the batched kernels.
#include "nep_batch.cuh"
#include "nep_batch_launch.h"

namespace nepk {

template <typename R, int BT>
static cudaError_t run(int mode, int grid, const Model<R>& P, const Batch& b, double* grad,
                       cudaStream_t s)
{
    switch (mode) {
    case MODE_FORWARD: k_batch<R, MODE_FORWARD, BT><<<grid, BT, 0, s>>>(P, b); break;
    case MODE_BACKWARD: k_batch<R, MODE_BACKWARD, BT><<<grid, BT, 0, s>>>(P, b); break;
    default: k_batch<R, MODE_LOSS, BT><<<grid, BT, 0, s>>>(P, b); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode != MODE_FORWARD) {
        k_batch_grad_reduce<<<(NP + 255) / 256, 256, 0, s>>>(b.gpart, b.S, grad);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_batch(int precision, int mode, int bt, int grid, const Model<float>& mf,
                         const Model<double>& md, const Batch& b, double* grad, cudaStream_t s)
{
    if (precision == 1) return run<double, 128>(mode, grid, md, b, grad, s);
    if (bt == 64) return run<float, 64>(mode, grid, mf, b, grad, s);
    if (bt == 256) return run<float, 256>(mode, grid, mf, b, grad, s);
    return run<float, 128>(mode, grid, mf, b, grad, s);
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
        if (mode == MODE_FORWARD) return occ(k_batch<double, MODE_FORWARD, 128>, 128);
        if (mode == MODE_BACKWARD) return occ(k_batch<double, MODE_BACKWARD, 128>, 128);
        return occ(k_batch<double, MODE_LOSS, 128>, 128);
    }
#define NEP_OCC(BT_)                                                            \
    if (bt == BT_) {                                                            \
        if (mode == MODE_FORWARD) return occ(k_batch<float, MODE_FORWARD, BT_>, BT_);   \
        if (mode == MODE_BACKWARD) return occ(k_batch<float, MODE_BACKWARD, BT_>, BT_); \
        return occ(k_batch<float, MODE_LOSS, BT_>, BT_);                       \
    }
    NEP_OCC(64)
    NEP_OCC(256)
#undef NEP_OCC
    if (mode == MODE_FORWARD) return occ(k_batch<float, MODE_FORWARD, 128>, 128);
    if (mode == MODE_BACKWARD) return occ(k_batch<float, MODE_BACKWARD, 128>, 128);
    return occ(k_batch<float, MODE_LOSS, 128>, 128);
}

}  // namespace nepk
