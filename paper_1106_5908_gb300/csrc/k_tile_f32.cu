// Compiled configurations of the tile kernel for FP32-stored values and vectors.
// Products and row sums are carried in at least FP64-class precision, either by
// one FP64 FMA per entry (operands widened on the integer pipe) or by the exact
// float-float accumulator on the FP32 pipe.
#include "internal.h"
#include "tile_kernel.cuh"

namespace spmv {

namespace {
template <int R, int E, typename YT, typename ACC, bool IND, bool BAT>
TileOps ops32() {
    using K = TileKernel<256, R, E, 2, float, float, YT, ACC, IND, BAT>;
    return TileOps{&K::launch, &K::grid_limit, &K::cfg};
}
}  // namespace

bool tile_ops_f32(int xk, int yk, int acc, int R, int E, bool indirect, bool batched,
                  TileOps *ops) {
    if (xk != kF32) return false;
#define SPMV_F32_CASE(YK_, YT_, ACCK_, ACC_, R_, E_, IND_, BAT_)                          \
    if (yk == YK_ && acc == ACCK_ && R == R_ && E == E_ && indirect == IND_ &&            \
        batched == BAT_) {                                                                \
        *ops = ops32<R_, E_, YT_, ACC_, IND_, BAT_>();                                    \
        return true;                                                                      \
    }
    SPMV_F32_CASE(kF32, float, kAccFF, AccFF, 1, 15, false, false)
    SPMV_F32_CASE(kF32, float, kAccFF, AccFF, 1, 31, false, false)
    SPMV_F32_CASE(kF32, float, kAccF64, AccF64, 1, 15, false, false)
    SPMV_F32_CASE(kF64, double, kAccFF, AccFF, 1, 15, false, false)
    SPMV_F32_CASE(kF64, double, kAccF64, AccF64, 1, 15, false, false)
#undef SPMV_F32_CASE
    return false;
}

}  // namespace spmv
