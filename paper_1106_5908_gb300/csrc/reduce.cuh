// Block sums and the last-block finish of the device reductions (CG dots and
// the dot product fused into the FP32 row-slice product): each block stores its
// partial, and the last block to finish (an atomic ticket, no waiting) sums the
// partials in block order and applies the scalar step, so the result is
// deterministic and no separate reduction launch is needed.
#pragma once
#include "cg.h"

namespace spmv {

__device__ __forceinline__ double block_sum(double v, double *s_red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? s_red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

__device__ __forceinline__ void apply_op(double t, double *sc, int op, int dst) {
    if (op == kOpStore) {
        sc[dst] = t;
    } else if (op == kOpAlpha) {  // t = p.q; a zero direction (converged) takes no step
        sc[kScPQ] = t;
        sc[kScAlpha] = (t != 0.0) ? sc[kScRho] / t : 0.0;
    } else if (op == kOpBeta) {   // t = r_new.r_new
        sc[kScBeta] = (sc[kScRho] != 0.0) ? t / sc[kScRho] : 0.0;
        sc[kScRho] = t;
    }
}

// t: the block's partial (valid in thread 0).  The last block sums all partials
// in block order, applies the step and re-arms the ticket.  Every thread of the
// block calls it.
__device__ __forceinline__ void finish(double t, const RedOut &o, double *s_red) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        o.partials[blockIdx.x] = t;
        __threadfence();
        s_last = (atomicAdd(o.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += blockDim.x) acc += __ldcg(o.partials + i);
    const double tot = block_sum(acc, s_red);
    if (threadIdx.x == 0) {
        apply_op(tot, o.sc, o.op, o.dst);
        *o.ticket = 0u;
    }
}

}  // namespace spmv
