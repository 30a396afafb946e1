// Vector kernels of the conjugate-gradient solvers: FP64-accumulated dot
// products with a deterministic two-stage reduction, fused CG updates in FP32
// (inner solver) and FP64 (outer residual, update, and the FP64 reference CG).
#include <algorithm>

#include "common.cuh"
#include "cg.h"

namespace spmv {

constexpr int kDotThreads = 256;

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

template <typename TA, typename TB>
__global__ void __launch_bounds__(kDotThreads) k_dot(const TA *__restrict__ a,
                                                     const TB *__restrict__ b, int64_t n,
                                                     double *__restrict__ partials) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        acc = fma(widen(a[i]), widen(b[i]), acc);
    const double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Sum the partials in a fixed order and apply the scalar step `op`.
__global__ void __launch_bounds__(kDotThreads) k_reduce(const double *__restrict__ partials,
                                                        int32_t np, double *sc, int op, int dst) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    const double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) {
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
}

// Inner (FP32) update: d += a*p, r -= a*q, partial sums of r.r (FP64 accumulate).
__global__ void __launch_bounds__(kDotThreads) k_update32(float *__restrict__ d,
                                                          float *__restrict__ r,
                                                          const float *__restrict__ p,
                                                          const float *__restrict__ q,
                                                          const double *__restrict__ sc, int64_t n,
                                                          double *__restrict__ partials) {
    __shared__ double s_red[32];
    const float a = __double2float_rn(sc[kScAlpha]);
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        d[i] = fmaf(a, p[i], d[i]);
        const float ri = fmaf(-a, q[i], r[i]);
        r[i] = ri;
        const double rw = widen(ri);
        acc = fma(rw, rw, acc);
    }
    const double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// FP64 update of the reference CG: x += a*p, r -= a*q, partial sums of r.r.
__global__ void __launch_bounds__(kDotThreads) k_update64(double *__restrict__ x,
                                                          double *__restrict__ r,
                                                          const double *__restrict__ p,
                                                          const double *__restrict__ q,
                                                          const double *__restrict__ sc, int64_t n,
                                                          double *__restrict__ partials) {
    __shared__ double s_red[32];
    const double a = sc[kScAlpha];
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_direction(T *__restrict__ p, const T *__restrict__ r,
                                                           const double *__restrict__ sc, int64_t n) {
    const T b = static_cast<T>(sc[kScBeta]);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = r[i] + b * p[i];
}

// r32 = FP32(s * r64)
__global__ void __launch_bounds__(kDotThreads) k_scale_to32(const double *__restrict__ r64,
                                                            float *__restrict__ r32, double s,
                                                            int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        r32[i] = __double2float_rn(s * r64[i]);
}

// x += s * d (FP64 update with the FP32 correction)
__global__ void __launch_bounds__(kDotThreads) k_axpy_64_32(double *__restrict__ x,
                                                            const float *__restrict__ d, double s,
                                                            int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[i] = fma(s, widen(d[i]), x[i]);
}

static int vec_grid(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kDotThreads - 1) / kDotThreads, 4LL * sms)));
}

int cg_partials_len() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 4 * sms;
}

cudaError_t cg_dot(const void *a, int ak, const void *b, int bk, int64_t n, double *partials,
                   double *sc, int op, int dst, cudaStream_t s) {
    const int grid = vec_grid(n);
    if (ak == kF64 && bk == kF64)
        k_dot<double, double><<<grid, kDotThreads, 0, s>>>(static_cast<const double *>(a), static_cast<const double *>(b), n, partials);
    else if (ak == kF32 && bk == kF32)
        k_dot<float, float><<<grid, kDotThreads, 0, s>>>(static_cast<const float *>(a), static_cast<const float *>(b), n, partials);
    else
        return cudaErrorInvalidValue;
    k_reduce<<<1, kDotThreads, 0, s>>>(partials, grid, sc, op, dst);
    return cudaGetLastError();
}

cudaError_t cg_update32(float *d, float *r, const float *p, const float *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s) {
    const int grid = vec_grid(n);
    k_update32<<<grid, kDotThreads, 0, s>>>(d, r, p, q, sc, n, partials);
    k_reduce<<<1, kDotThreads, 0, s>>>(partials, grid, sc, kOpBeta, 0);
    return cudaGetLastError();
}

cudaError_t cg_update64(double *x, double *r, const double *p, const double *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s) {
    const int grid = vec_grid(n);
    k_update64<<<grid, kDotThreads, 0, s>>>(x, r, p, q, sc, n, partials);
    k_reduce<<<1, kDotThreads, 0, s>>>(partials, grid, sc, kOpBeta, 0);
    return cudaGetLastError();
}

cudaError_t cg_direction(void *p, const void *r, int k, const double *sc, int64_t n, cudaStream_t s) {
    const int grid = vec_grid(n);
    if (k == kF32)
        k_direction<float><<<grid, kDotThreads, 0, s>>>(static_cast<float *>(p), static_cast<const float *>(r), sc, n);
    else
        k_direction<double><<<grid, kDotThreads, 0, s>>>(static_cast<double *>(p), static_cast<const double *>(r), sc, n);
    return cudaGetLastError();
}

cudaError_t cg_scale_to32(const double *r64, float *r32, double scale, int64_t n, cudaStream_t s) {
    k_scale_to32<<<vec_grid(n), kDotThreads, 0, s>>>(r64, r32, scale, n);
    return cudaGetLastError();
}

cudaError_t cg_axpy_64_32(double *x, const float *d, double scale, int64_t n, cudaStream_t s) {
    k_axpy_64_32<<<vec_grid(n), kDotThreads, 0, s>>>(x, d, scale, n);
    return cudaGetLastError();
}

}  // namespace spmv
