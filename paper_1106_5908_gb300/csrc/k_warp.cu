// Compiled configurations of the warp-chunk kernel (single right-hand side):
// FP64, FP32 storage with float-float or FP64 accumulation, the transposed apply
// of the reverse pass (values through a permutation) and the batched launch.
#include "pipe_kernel.cuh"
#include "warp_kernel.cuh"

namespace spmv {

bool warp_ops(int vk, int xk, int yk, int acc, int E, bool indirect, bool batched, WarpOps *ops) {
#define SPMV_W(VK_, VT_, YK_, YT_, ACCK_, ACC_, E_, IND_, BAT_)                                  \
    if (vk == VK_ && xk == VK_ && yk == YK_ && (VK_ == kF64 || acc == ACCK_) && E == E_ &&      \
        indirect == IND_ && batched == BAT_) {                                                   \
        ops->launch = &WarpKernel<E_, VT_, VT_, YT_, ACC_, IND_, BAT_>::launch;                  \
        return true;                                                                             \
    }
#define SPMV_P(VK_, VT_, YK_, YT_, ACCK_, ACC_, E_, IND_, BAT_)                                  \
    if (vk == VK_ && xk == VK_ && yk == YK_ && (VK_ == kF64 || acc == ACCK_) && E == E_ &&      \
        indirect == IND_ && batched == BAT_) {                                                   \
        ops->launch = &PipeKernel<E_, VT_, VT_, YT_, ACC_, IND_, BAT_>::launch;                  \
        return true;                                                                             \
    }
    SPMV_P(kF64, double, kF64, double, kAccF64, AccF64, 15, false, false)
    SPMV_P(kF64, double, kF64, double, kAccF64, AccF64, 7, false, false)
    SPMV_P(kF64, double, kF64, double, kAccF64, AccF64, 15, true, false)
    SPMV_P(kF64, double, kF64, double, kAccF64, AccF64, 15, false, true)
    SPMV_P(kF32, float, kF32, float, kAccFF, AccFF, 15, false, false)
    SPMV_P(kF32, float, kF64, double, kAccFF, AccFF, 15, false, false)
    SPMV_P(kF32, float, kF32, float, kAccF64, AccF64, 15, false, false)
    SPMV_P(kF32, float, kF64, double, kAccF64, AccF64, 15, false, false)
    SPMV_P(kF32, float, kF32, float, kAccFF, AccFF, 15, true, false)
    SPMV_P(kF32, float, kF32, float, kAccFF, AccFF, 15, false, true)
#undef SPMV_P
    SPMV_W(kF64, double, kF64, double, kAccF64, AccF64, 16, false, false)
    SPMV_W(kF64, double, kF64, double, kAccF64, AccF64, 8, false, false)
    SPMV_W(kF64, double, kF64, double, kAccF64, AccF64, 16, true, false)
    SPMV_W(kF64, double, kF64, double, kAccF64, AccF64, 16, false, true)
    SPMV_W(kF32, float, kF32, float, kAccFF, AccFF, 16, false, false)
    SPMV_W(kF32, float, kF64, double, kAccFF, AccFF, 16, false, false)
    SPMV_W(kF32, float, kF32, float, kAccF64, AccF64, 16, false, false)
    SPMV_W(kF32, float, kF64, double, kAccF64, AccF64, 16, false, false)
    SPMV_W(kF32, float, kF32, float, kAccFF, AccFF, 16, true, false)
    SPMV_W(kF32, float, kF32, float, kAccFF, AccFF, 16, false, true)
#undef SPMV_W
    return false;
}

}  // namespace spmv
