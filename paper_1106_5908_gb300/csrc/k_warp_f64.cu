// Compiled configurations of the warp-chunk kernels for FP64 values and
// vectors: the pipelined kernels (odd E; E + 100 three-stage) and the
// unpipelined one (E = 8, 16), for the plain product, the transposed apply of the
// reverse pass (values through a permutation) and the batched launch.
#include "internal.h"
#include "pipe_kernel.cuh"
#include "warp_kernel.cuh"

namespace spmv {

bool warp_ops_f64(int E, bool indirect, bool batched, WarpOps *ops) {
#define SPMV_P(E_, IND_, BAT_)                                                             \
    if (E == E_ && indirect == IND_ && batched == BAT_) {                                  \
        ops->launch = &PipeKernel<E_, double, double, double, AccF64, IND_, BAT_>::launch; \
        return true;                                                                       \
    }
#define SPMV_P3(E_, BAT_)                                                                   \
    if (E == E_ + 100 && !indirect && batched == BAT_) {                                   \
        ops->launch = &Pipe3Kernel<E_, double, double, double, AccF64, false, BAT_>::launch; \
        return true;                                                                       \
    }
    SPMV_P3(7, false)
    SPMV_P3(11, false)
    SPMV_P3(15, false)
#undef SPMV_P3
#define SPMV_W(E_, IND_, BAT_)                                                             \
    if (E == E_ && indirect == IND_ && batched == BAT_) {                                  \
        ops->launch = &WarpKernel<E_, double, double, double, AccF64, IND_, BAT_>::launch; \
        return true;                                                                       \
    }
    SPMV_P(15, false, false)
    SPMV_P(7, false, false)
    SPMV_P(15, true, false)
    SPMV_P(7, true, false)
    SPMV_P(15, false, true)
    SPMV_P(7, false, true)
    SPMV_W(16, false, false)
    SPMV_W(8, false, false)
    SPMV_W(16, true, false)
    SPMV_W(16, false, true)
#undef SPMV_P
#undef SPMV_W
    return false;
}

}  // namespace spmv
