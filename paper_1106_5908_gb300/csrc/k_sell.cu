// Compiled configurations of the sorted row-slice kernel (plan family 5) and its
// relayout kernel: FP64 values and vectors, and FP32 storage with FP32 runs
// (every row at most 11 entries, so a lane's chain over a row is a run) or FP32
// runs of one block (4 slot rows) each folded into float-float.
#include "internal.h"
#include "sell_kernel.cuh"

namespace spmv {

bool sell_ops(int vk, int xk, int yk, int acc, SellOps *ops, int32_t max_row) {
    if (vk == kF64 && xk == kF64 && yk == kF64 && acc == kAccF64) {
        ops->launch = &SellKernel<double, double, double, AccF64>::launch;
        ops->ctas_for = &SellKernel<double, double, double, AccF64>::ctas_for;
        ops->launch_dot = nullptr;
        return true;
    }
    if (vk == kF32 && xk == kF32 && yk == kF32 && acc == kAccFF && max_row <= kFRMaxRun) {
        ops->launch = &SellKernel<float, float, float, AccFR>::launch;
        ops->ctas_for = &SellKernel<float, float, float, AccFR>::ctas_for;
        ops->launch_dot = &SellKernel<float, float, float, AccFR>::launch_dot;
        return true;
    }
    if (vk == kF32 && xk == kF32 && yk == kF32 && acc == kAccFF) {
        ops->launch = &SellKernel<float, float, float, AccFRF>::launch;
        ops->ctas_for = &SellKernel<float, float, float, AccFRF>::ctas_for;
        ops->launch_dot = &SellKernel<float, float, float, AccFRF>::launch_dot;
        return true;
    }
    return false;
}

cudaError_t launch_sell_mr(const SellParams &b, const double *X, double *Y, int64_t ldx, int64_t ldy, bool vec,
                           cudaStream_t s) {
    if (b.n_slices <= 0 || b.n_ctas <= 0) return cudaSuccess;
    const SellMrParams q{b, X, Y, ldx, ldy};
    if (vec) k_sell_mr<true><<<b.n_ctas, 256, 0, s>>>(q);
    else k_sell_mr<false><<<b.n_ctas, 256, 0, s>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_sell_relayout(const void *slices, const int32_t *srows, int32_t n_slices, const int32_t *rp,
                                 int vk, const void *val, const int32_t *col, void *vals_out, int32_t *cols_out,
                                 cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (static_cast<int64_t>(n_slices) * kSellC + 255) / 256;
    const int grid = static_cast<int>(want < 16LL * sms ? want : 16LL * sms);
    const int2 *d = static_cast<const int2 *>(slices);
    if (vk == kF64)
        k_sell_relayout<double><<<grid, 256, 0, s>>>(d, srows, n_slices, rp, static_cast<const double *>(val), col,
                                                     static_cast<double *>(vals_out), cols_out);
    else
        k_sell_relayout<float><<<grid, 256, 0, s>>>(d, srows, n_slices, rp, static_cast<const float *>(val), col,
                                                    static_cast<float *>(vals_out), cols_out);
    return cudaGetLastError();
}

}  // namespace spmv
