// Vector kernels of the conjugate-gradient solvers: dot products and fused CG
// updates in FP32 (inner solver) and FP64 (outer residual, update, and the FP64
// reference CG).  Reductions run on two blocks per SM; each block stores its
// partial sum and the last block to finish (an atomic ticket, no waiting) sums
// the partials in block order and applies the scalar step, so the result is
// deterministic and no separate reduction launch is needed.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "common.cuh"
#include "cg.h"
#include "reduce.cuh"

namespace spmv {

constexpr int kDotThreads = 256;

template <typename TA, typename TB>
__global__ void __launch_bounds__(kDotThreads) k_dot(const TA *__restrict__ a,
                                                     const TB *__restrict__ b, int64_t n,
                                                     const RedOut o) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        acc = fma(widen(a[i]), widen(b[i]), acc);
    finish(block_sum(acc, s_red), o, s_red);
}

// Vectorised variants for 16-byte aligned operands: four floats (or two
// doubles) per load and independent accumulators, so each thread keeps several
// loads in flight; the tail is handled element by element.  FP32 operands are
// accumulated as float-float pairs (exact products, two-sum), which keeps the
// FP64 pipe out of the loop; each thread's pairs are summed in FP64.
__global__ void __launch_bounds__(kDotThreads) k_dot_f32v(const float4 *__restrict__ a,
                                                          const float4 *__restrict__ b, int64_t n4,
                                                          const float *__restrict__ at,
                                                          const float *__restrict__ bt, int tail,
                                                          const RedOut o) {
    __shared__ double s_red[32];
    AccFF c0, c1, c2, c3;
    c0.zero(); c1.zero(); c2.zero(); c3.zero();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
#pragma unroll 4
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 u = __ldg(a + i), v = __ldg(b + i);
        c0.fma(u.x, v.x);
        c1.fma(u.y, v.y);
        c2.fma(u.z, v.z);
        c3.fma(u.w, v.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) c0.fma(at[threadIdx.x], bt[threadIdx.x]);
    double t = (c0.get() + c1.get()) + (c2.get() + c3.get());
    if (c0.poisoned() || c1.poisoned() || c2.poisoned() || c3.poisoned()) {
        // a product outside FP32's range: this thread's terms again with exact FP64 products
        t = 0.0;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 u = __ldg(a + i), v = __ldg(b + i);
            t = fma(widen(u.x), widen(v.x), t);
            t = fma(widen(u.y), widen(v.y), t);
            t = fma(widen(u.z), widen(v.z), t);
            t = fma(widen(u.w), widen(v.w), t);
        }
        if (blockIdx.x == 0 && threadIdx.x < tail) t = fma(widen(at[threadIdx.x]), widen(bt[threadIdx.x]), t);
    }
    finish(block_sum(t, s_red), o, s_red);
}

__global__ void __launch_bounds__(kDotThreads) k_dot_f64v(const double2 *__restrict__ a,
                                                          const double2 *__restrict__ b, int64_t n2,
                                                          const double *__restrict__ at,
                                                          const double *__restrict__ bt, int tail,
                                                          const RedOut o) {
    __shared__ double s_red[32];
    double c0 = 0.0, c1 = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
#pragma unroll 4
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n2; i += stride) {
        const double2 u = __ldg(a + i), v = __ldg(b + i);
        c0 = fma(u.x, v.x, c0);
        c1 = fma(u.y, v.y, c1);
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) c0 = fma(at[threadIdx.x], bt[threadIdx.x], c0);
    finish(block_sum(c0 + c1, s_red), o, s_red);
}

// Inner (FP32) update: d += a*p, r -= a*q, partial sums of r.r (FP64 accumulate).
__global__ void __launch_bounds__(kDotThreads) k_update32(float *__restrict__ d,
                                                          float *__restrict__ r,
                                                          const float *__restrict__ p,
                                                          const float *__restrict__ q,
                                                          const double *__restrict__ sc, int64_t n,
                                                          const RedOut o) {
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
    finish(block_sum(acc, s_red), o, s_red);
}

__global__ void __launch_bounds__(kDotThreads) k_update32v(float4 *__restrict__ d, float4 *__restrict__ r,
                                                           const float4 *__restrict__ p,
                                                           const float4 *__restrict__ q,
                                                           const double *__restrict__ sc, int64_t n4,
                                                           float *__restrict__ dt, float *__restrict__ rt,
                                                           const float *__restrict__ pt,
                                                           const float *__restrict__ qt, int tail,
                                                           const RedOut o) {
    __shared__ double s_red[32];
    const float a = __double2float_rn(sc[kScAlpha]);
    AccFF c0, c1, c2, c3;
    c0.zero(); c1.zero(); c2.zero(); c3.zero();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
#pragma unroll 2
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 pv = p[i], qv = q[i];
        float4 dv = d[i], rv = r[i];
        dv.x = fmaf(a, pv.x, dv.x); dv.y = fmaf(a, pv.y, dv.y);
        dv.z = fmaf(a, pv.z, dv.z); dv.w = fmaf(a, pv.w, dv.w);
        rv.x = fmaf(-a, qv.x, rv.x); rv.y = fmaf(-a, qv.y, rv.y);
        rv.z = fmaf(-a, qv.z, rv.z); rv.w = fmaf(-a, qv.w, rv.w);
        d[i] = dv;
        r[i] = rv;
        c0.fma(rv.x, rv.x);
        c1.fma(rv.y, rv.y);
        c2.fma(rv.z, rv.z);
        c3.fma(rv.w, rv.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) {
        const int j = threadIdx.x;
        dt[j] = fmaf(a, pt[j], dt[j]);
        const float ri = fmaf(-a, qt[j], rt[j]);
        rt[j] = ri;
        c0.fma(ri, ri);
    }
    double t = (c0.get() + c1.get()) + (c2.get() + c3.get());
    if (c0.poisoned() || c1.poisoned() || c2.poisoned() || c3.poisoned()) {
        // a square outside FP32's range: this thread's updated r again in FP64
        t = 0.0;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 rv = r[i];
            t = fma(widen(rv.x), widen(rv.x), t);
            t = fma(widen(rv.y), widen(rv.y), t);
            t = fma(widen(rv.z), widen(rv.z), t);
            t = fma(widen(rv.w), widen(rv.w), t);
        }
        if (blockIdx.x == 0 && threadIdx.x < tail) t = fma(widen(rt[threadIdx.x]), widen(rt[threadIdx.x]), t);
    }
    finish(block_sum(t, s_red), o, s_red);
}

__global__ void __launch_bounds__(kDotThreads) k_direction32v(float4 *__restrict__ p,
                                                              const float4 *__restrict__ r,
                                                              const double *__restrict__ sc, int64_t n4,
                                                              float *__restrict__ pt,
                                                              const float *__restrict__ rt, int tail) {
    const float b = static_cast<float>(sc[kScBeta]);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 rv = r[i];
        float4 pv = p[i];
        pv.x = fmaf(b, pv.x, rv.x); pv.y = fmaf(b, pv.y, rv.y);
        pv.z = fmaf(b, pv.z, rv.z); pv.w = fmaf(b, pv.w, rv.w);
        p[i] = pv;
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) pt[threadIdx.x] = fmaf(b, pt[threadIdx.x], rt[threadIdx.x]);
}

// FP64 update of the reference CG: x += a*p, r -= a*q, partial sums of r.r.
__global__ void __launch_bounds__(kDotThreads) k_update64(double *__restrict__ x,
                                                          double *__restrict__ r,
                                                          const double *__restrict__ p,
                                                          const double *__restrict__ q,
                                                          const double *__restrict__ sc, int64_t n,
                                                          const RedOut o) {
    __shared__ double s_red[32];
    const double a = sc[kScAlpha];
    double acc0 = 0.0, acc1 = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {  // two independent elements in flight
        const double p0 = p[i], q0 = q[i], x0 = x[i], r0 = r[i];
        const double p1 = p[i + stride], q1 = q[i + stride], x1 = x[i + stride], r1 = r[i + stride];
        x[i] = fma(a, p0, x0);
        x[i + stride] = fma(a, p1, x1);
        const double ri0 = fma(-a, q0, r0), ri1 = fma(-a, q1, r1);
        r[i] = ri0;
        r[i + stride] = ri1;
        acc0 = fma(ri0, ri0, acc0);
        acc1 = fma(ri1, ri1, acc1);
    }
    if (i < n) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        acc0 = fma(ri, ri, acc0);
    }
    finish(block_sum(acc0 + acc1, s_red), o, s_red);
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

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// elementwise kernels: up to 16 blocks per SM
static int vec_grid(int64_t n) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kDotThreads - 1) / kDotThreads,
                                                                   16LL * sm_count())));
}

// reductions: up to kRedBlocksPerSM blocks per SM (each block's FP64 tree work
// is paid once per block, so fewer, longer-running blocks)
constexpr int kRedBlocksPerSM = 2;
static int red_grid(int64_t n) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + kDotThreads - 1) / kDotThreads,
                                                                   int64_t(kRedBlocksPerSM) * sm_count())));
}

// partials (one per reduction block, room for 16 blocks per SM: the fused
// product's persistent launch) followed by the ticket word
int cg_partials_cap() { return 16 * sm_count(); }
int cg_partials_len() { return cg_partials_cap() + 2; }

RedOut cg_red_out(double *partials, double *sc, int op, int dst) {
    return RedOut{partials, reinterpret_cast<unsigned int *>(partials + cg_partials_cap()), sc, op, dst};
}
static RedOut red_out(double *partials, double *sc, int op, int dst) { return cg_red_out(partials, sc, op, dst); }

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cudaError_t cg_dot(const void *a, int ak, const void *b, int bk, int64_t n, double *partials,
                   double *sc, int op, int dst, cudaStream_t s) {
    const RedOut o = red_out(partials, sc, op, dst);
    if (ak == kF64 && bk == kF64) {
        const double *ad = static_cast<const double *>(a), *bd = static_cast<const double *>(b);
        if (aligned16(a) && aligned16(b)) {
            const int64_t n2 = n / 2;
            k_dot_f64v<<<red_grid(n2), kDotThreads, 0, s>>>(reinterpret_cast<const double2 *>(ad),
                                                            reinterpret_cast<const double2 *>(bd), n2,
                                                            ad + 2 * n2, bd + 2 * n2,
                                                            static_cast<int>(n - 2 * n2), o);
        } else {
            k_dot<double, double><<<red_grid(n), kDotThreads, 0, s>>>(ad, bd, n, o);
        }
    } else if (ak == kF32 && bk == kF32) {
        const float *af = static_cast<const float *>(a), *bf = static_cast<const float *>(b);
        if (aligned16(a) && aligned16(b)) {
            const int64_t n4 = n / 4;
            k_dot_f32v<<<red_grid(n4), kDotThreads, 0, s>>>(reinterpret_cast<const float4 *>(af),
                                                            reinterpret_cast<const float4 *>(bf), n4,
                                                            af + 4 * n4, bf + 4 * n4,
                                                            static_cast<int>(n - 4 * n4), o);
        } else {
            k_dot<float, float><<<red_grid(n), kDotThreads, 0, s>>>(af, bf, n, o);
        }
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t cg_update32(float *d, float *r, const float *p, const float *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s) {
    const RedOut o = red_out(partials, sc, kOpBeta, 0);
    if (aligned16(d) && aligned16(r) && aligned16(p) && aligned16(q)) {
        const int64_t n4 = n / 4;
        k_update32v<<<red_grid(n4), kDotThreads, 0, s>>>(
            reinterpret_cast<float4 *>(d), reinterpret_cast<float4 *>(r), reinterpret_cast<const float4 *>(p),
            reinterpret_cast<const float4 *>(q), sc, n4, d + 4 * n4, r + 4 * n4, p + 4 * n4, q + 4 * n4,
            static_cast<int>(n - 4 * n4), o);
    } else {
        k_update32<<<red_grid(n), kDotThreads, 0, s>>>(d, r, p, q, sc, n, o);
    }
    return cudaGetLastError();
}

cudaError_t cg_update64(double *x, double *r, const double *p, const double *q, int64_t n,
                        double *partials, double *sc, cudaStream_t s) {
    k_update64<<<red_grid(n), kDotThreads, 0, s>>>(x, r, p, q, sc, n, red_out(partials, sc, kOpBeta, 0));
    return cudaGetLastError();
}

cudaError_t cg_direction(void *p, const void *r, int k, const double *sc, int64_t n, cudaStream_t s) {
    const int grid = vec_grid(n);
    if (k == kF32 && aligned16(p) && aligned16(r)) {
        const int64_t n4 = n / 4;
        float *pf = static_cast<float *>(p);
        const float *rf = static_cast<const float *>(r);
        k_direction32v<<<vec_grid(n4), kDotThreads, 0, s>>>(reinterpret_cast<float4 *>(pf),
                                                            reinterpret_cast<const float4 *>(rf), sc, n4,
                                                            pf + 4 * n4, rf + 4 * n4,
                                                            static_cast<int>(n - 4 * n4));
    } else if (k == kF32)
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
