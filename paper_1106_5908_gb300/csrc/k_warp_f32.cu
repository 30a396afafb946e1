// Compiled configurations of the warp-chunk kernels for FP32-stored values and
// vectors, with float-float (FP32 pipe) or FP64-FMA accumulation.
#include "internal.h"
#include "pipe_kernel.cuh"
#include "warp_kernel.cuh"

namespace spmv {

bool warp_ops_f32(int yk, int acc, int E, bool indirect, bool batched, WarpOps *ops) {
#define SPMV_P(YK_, YT_, ACCK_, ACC_, E_, IND_, BAT_)                                   \
    if (yk == YK_ && acc == ACCK_ && E == E_ && indirect == IND_ && batched == BAT_) {  \
        ops->launch = &PipeKernel<E_, float, float, YT_, ACC_, IND_, BAT_>::launch;     \
        return true;                                                                    \
    }
#define SPMV_P3(YK_, YT_, ACCK_, ACC_, E_)                                                \
    if (yk == YK_ && acc == ACCK_ && E == E_ + 100 && !indirect && !batched) {          \
        ops->launch = &Pipe3Kernel<E_, float, float, YT_, ACC_, false, false>::launch;  \
        return true;                                                                    \
    }
    SPMV_P3(kF32, float, kAccFF, AccFF, 15)
    SPMV_P3(kF64, double, kAccFF, AccFF, 15)
    SPMV_P3(kF32, float, kAccF64, AccF64, 15)
    SPMV_P3(kF64, double, kAccF64, AccF64, 15)
#undef SPMV_P3
#define SPMV_W(YK_, YT_, ACCK_, ACC_, E_, IND_, BAT_)                                   \
    if (yk == YK_ && acc == ACCK_ && E == E_ && indirect == IND_ && batched == BAT_) {  \
        ops->launch = &WarpKernel<E_, float, float, YT_, ACC_, IND_, BAT_>::launch;     \
        return true;                                                                    \
    }
    SPMV_P(kF32, float, kAccFF, AccFF, 15, false, false)
    SPMV_P(kF32, float, kAccFF, AccFF, 7, false, false)
    SPMV_P(kF64, double, kAccFF, AccFF, 15, false, false)
    SPMV_P(kF64, double, kAccFF, AccFF, 7, false, false)
    SPMV_P(kF32, float, kAccF64, AccF64, 15, false, false)
    SPMV_P(kF32, float, kAccF64, AccF64, 7, false, false)
    SPMV_P(kF64, double, kAccF64, AccF64, 15, false, false)
    SPMV_P(kF64, double, kAccF64, AccF64, 7, false, false)
    SPMV_P(kF32, float, kAccFF, AccFF, 15, true, false)
    SPMV_P(kF32, float, kAccFF, AccFF, 7, true, false)
    SPMV_P(kF32, float, kAccFF, AccFF, 15, false, true)
    SPMV_P(kF32, float, kAccFF, AccFF, 7, false, true)
    SPMV_W(kF32, float, kAccFF, AccFF, 16, false, false)
    SPMV_W(kF64, double, kAccFF, AccFF, 16, false, false)
    SPMV_W(kF32, float, kAccF64, AccF64, 16, false, false)
    SPMV_W(kF64, double, kAccF64, AccF64, 16, false, false)
    SPMV_W(kF32, float, kAccFF, AccFF, 16, true, false)
    SPMV_W(kF32, float, kAccFF, AccFF, 16, false, true)
#undef SPMV_P
#undef SPMV_W
    return false;
}

}  // namespace spmv
