// Compiled configurations of the tile kernel for FP64 values and vectors: the
// plain product (group width 1, plan family 2) and block vectors (group width
// 2..32).
#include "internal.h"
#include "tile_kernel.cuh"

namespace spmv {

namespace {
template <int R, int E, bool IND, bool BAT>
TileOps ops64() {
    using K = TileKernel<256, R, E, 2, double, double, double, AccF64, IND, BAT>;
    return TileOps{&K::launch, &K::grid_limit, &K::cfg};
}
}  // namespace

bool tile_ops_f64(int R, int E, bool indirect, bool batched, TileOps *ops) {
#define SPMV_F64_CASE(R_, E_, IND_, BAT_)                                   \
    if (R == R_ && E == E_ && indirect == IND_ && batched == BAT_) {        \
        *ops = ops64<R_, E_, IND_, BAT_>();                                 \
        return true;                                                        \
    }
    SPMV_F64_CASE(1, 7, false, false)
    SPMV_F64_CASE(1, 15, false, false)
    SPMV_F64_CASE(1, 31, false, false)
    SPMV_F64_CASE(2, 15, false, false)
    SPMV_F64_CASE(4, 15, false, false)
    SPMV_F64_CASE(8, 15, false, false)
    SPMV_F64_CASE(16, 15, false, false)
    SPMV_F64_CASE(32, 15, false, false)
#undef SPMV_F64_CASE
    return false;
}

}  // namespace spmv
