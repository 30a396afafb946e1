// Device helpers shared by the sm_103a kernels: TMA bulk copies into shared
// memory completed through an mbarrier, bounded waits, FP32->FP64 widening on the
// integer pipe, and the row-sum accumulators.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "types.h"

namespace spmv {

// ---------------------------------------------------------------------------
// mbarrier + cp.async.bulk (1-D bulk copy global -> shared, no tensor map)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from global
// memory into this CTA's shared memory; completion is signalled on `bar`.  The
// streamed operand is marked evict-first in L2 so it does not displace x.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// The suspend-time hint (ns) lets the hardware park the waiting warp until the
// phase completes instead of returning at once, so waiting warps do not take
// issue slots from the warps that compute.
constexpr uint32_t kTryWaitSuspendNs = 20000;

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(kTryWaitSuspendNs) : "memory");
    return ok;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete.  Gives up after limit_ns of wall
// time (checked every 64 polls), or after kWaitLimitIters polls should the timer
// not advance, and returns false; never spins forever.  A poll returns after at
// most kTryWaitSuspendNs, so the poll bound is at most ~80 s.
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr uint32_t kWaitLimitIters = 1u << 22;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < kWaitLimitIters; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Record a device error code in the handle's error word (first one wins).
__device__ __forceinline__ void set_error(int32_t *err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// FP32 -> FP64 widening without the FP64 pipe.  On GB300 the F2F.F64.F32
// conversion issues on the (narrow) FP64 unit, at the DFMA rate; here every
// input is widened with FP32/integer operations and no branch (a conditional
// hardware fallback would be if-converted and issued for every element):
//   normal:    exponent rebiased by 1023-127, 23-bit mantissa moved up 29 bits;
//   zero:      sign only;
//   inf/NaN:   exponent field 0x7ff, payload moved up 29 bits;
//   subnormal: scaled by 2^24 in FP32 (exact, the result is normal), widened as
//              a normal number, and the 24 taken off the FP64 exponent field.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double widen(float f) {
    const uint32_t a0 = __float_as_uint(f) & 0x7fffffffu;
    const bool sub = (a0 != 0u) && (a0 < 0x00800000u);
    const uint32_t u = __float_as_uint(sub ? f * 16777216.0f : f);
    const uint32_t a = u & 0x7fffffffu;
    const uint32_t bias = (a >= 0x7f800000u) ? 0x70000000u : (sub ? 0x38000000u - (24u << 20) : 0x38000000u);
    const uint32_t hi = (u & 0x80000000u) | (a ? (a >> 3) + bias : 0u);
    const uint32_t lo = u << 29;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
__device__ __forceinline__ double widen(double d) { return d; }

template <typename T> __device__ __forceinline__ T narrow(double d);
template <> __device__ __forceinline__ double narrow<double>(double d) { return d; }
template <> __device__ __forceinline__ float narrow<float>(double d) { return __double2float_rn(d); }

// ---------------------------------------------------------------------------
// Row-sum accumulators.  Each holds a partial row sum and supports:
//   zero(), fma(v, x) (acc += v*x), add(other), get() -> double.
// ---------------------------------------------------------------------------

// FP64 accumulation: exactly one DFMA per stored entry.
struct AccF64 {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    template <typename V, typename X>
    __device__ __forceinline__ void fma(V v, X x) { s = ::fma(widen(v), widen(x), s); }
    __device__ __forceinline__ void add(const AccF64 &o) { s += o.s; }
    __device__ __forceinline__ double get() const { return s; }
};

// Float-float accumulation on the FP32 pipe for FP32-stored operands (the Dot2
// scheme of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): each
// product of two floats is split exactly into ph + pl (FMA residual), ph is
// added to the running sum h by Knuth's two-sum, and the rounding error of that
// addition plus pl is collected in l.  The value is h + l; its error is about
// n^2 2^-48 sum |a_ij x_j| for n terms, far inside the FP32-storage tolerance,
// while using no FP64 instructions per entry.
//
// The scheme needs every product inside FP32's range.  Outside it the sum is
// marked untrustworthy ("poisoned": l is NaN) and the caller sums the row again
// with exact FP64 products (FP64 accumulation, the definition of this form):
//   * a nonzero product of magnitude below kFFTiny may have lost bits of its
//     exact split to FP32 underflow (the low part's last bit lies 47 binades
//     below the high part's leading one, and FP32 stops at 2^-149), or have
//     underflowed to zero altogether: fma() sets l to NaN for it;
//   * an overflow of a product or of the running sum makes the two-sum form
//     inf - inf, so l becomes NaN by itself, as it does for an infinite or NaN
//     operand.
// A poisoned row costs one FP64 pass over its entries; rows of ordinary
// magnitudes never take it.
constexpr float kFFTiny = 0x1p-100f;

struct AccFF {
    float h, l;
    __device__ __forceinline__ void zero() { h = 0.f; l = 0.f; }
    __device__ __forceinline__ void add_pair(float ph, float pl) {
        const float s = h + ph;
        const float bb = s - h;
        const float e = (h - (s - bb)) + (ph - bb);
        h = s;
        l = l + (e + pl);
    }
    __device__ __forceinline__ void fma(float v, float x) {
        const float ph = v * x;
        const float pl = fmaf(v, x, -ph);
        const bool tiny = fabsf(ph) < kFFTiny && v != 0.0f && x != 0.0f;
        add_pair(ph, tiny ? __int_as_float(0x7fffffff) : pl);
    }
    __device__ __forceinline__ void add(const AccFF &o) { add_pair(o.h, o.l); }
    __device__ __forceinline__ bool poisoned() const { return l != l; }
    __device__ __forceinline__ double get() const { return widen(h) + widen(l); }
};

// FP32 runs with float-float carries, for kernels whose lanes own at most
// kFRMaxRun consecutive entries of a row (the slot-major chunk kernel with
// E <= 11): the products of one lane's piece of a row are summed by plain FP32
// FMAs (recursive summation, error at most gamma_k sum |a_ij x_j| with k <= 11
// terms, gamma_k = k u / (1 - k u), u = 2^-24: 6.6e-7, inside the 1e-6 FP32-storage
// tolerance), and the pieces of a row cut by lane boundaries are combined by
// two-sum (float-float), whose error is of order u^2.  The bound assumes no
// partial sum underflows or overflows; a row whose final sum is not finite or
// below kFFTiny in magnitude (a sum that small can only come from terms that
// small, or from exact cancellation) is marked poisoned and summed again with
// FP64 products, as for AccFF.  Each entry costs one FP32 FMA instead of
// AccFF's ten-odd FP32 operations.
constexpr int kFRMaxRun = 11;
struct AccFR {
    float h, l;
    __device__ __forceinline__ void zero() { h = 0.f; l = 0.f; }
    __device__ __forceinline__ void fma(float v, float x) { h = fmaf(v, x, h); }
    __device__ __forceinline__ void add(const AccFR &o) {
        const float s = h + o.h;
        const float bb = s - h;
        const float e = (h - (s - bb)) + (o.h - bb);
        h = s;
        l = l + (e + o.l);
    }
    __device__ __forceinline__ bool poisoned() const {
        const float a = fabsf(h);
        return !(a >= kFFTiny && a <= 0x1.fffffep127f) || l != l;
    }
    __device__ __forceinline__ double get() const { return widen(h) + widen(l); }
};

// FP32 runs folded into float-float, for a lane that sums a whole row of any
// length in blocks of at most kFRMaxRun entries (the row-slice kernel): the
// block's products go into the run r by plain FP32 FMAs, and fold() adds r to
// the float-float total (h, l) by two-sum and clears it.  Error at most
// gamma_k sum |a_ij x_j| for blocks of k entries, plus order u^2 from the
// folds; the same range rule as AccFR (checked after the last fold).
struct AccFRF {
    float r, h, l;
    __device__ __forceinline__ void zero() { r = 0.f; h = 0.f; l = 0.f; }
    __device__ __forceinline__ void fma(float v, float x) { r = fmaf(v, x, r); }
    __device__ __forceinline__ void fold() {
        const float s = h + r;
        const float bb = s - h;
        const float e = (h - (s - bb)) + (r - bb);
        h = s;
        l = l + e;
        r = 0.f;
    }
    __device__ __forceinline__ bool poisoned() const {
        const float a = fabsf(h);
        return !(a >= kFFTiny && a <= 0x1.fffffep127f) || l != l || r != 0.f;
    }
    __device__ __forceinline__ double get() const { return widen(h) + widen(l) + widen(r); }
};

// Accumulator for work that is not cut into pieces of at most kFRMaxRun
// entries (whole rows per lane, long rows strided over a warp): AccFR and
// AccFRF fall back to AccFF there.
template <typename ACC> struct WholeRowAcc { using type = ACC; };
template <> struct WholeRowAcc<AccFR> { using type = AccFF; };
template <> struct WholeRowAcc<AccFRF> { using type = AccFF; };

// Ends a block of at most kFRMaxRun entries (AccFRF: fold the run; others: nothing).
template <typename ACC> __device__ __forceinline__ void end_run(ACC &) {}
template <> __device__ __forceinline__ void end_run<AccFRF>(AccFRF &a) { a.fold(); }

// Row r of m summed again with exact FP64 products of its (FP32-stored)
// operands, in CRS order: the fallback for a poisoned float-float row sum (see
// AccFF).  x[j] is read at x + j*ldx.
template <typename VT, bool INDIRECT, typename XT>
__device__ __forceinline__ double row_sum_exact(const MatRef m, int64_t r, const XT *__restrict__ x, int64_t ldx = 1) {
    double s = 0.0;
    const int kb = __ldg(m.rp + r), ke = __ldg(m.rp + r + 1);
    for (int k = kb; k < ke; ++k) {
        VT v;
        if constexpr (INDIRECT)
            v = __ldg(static_cast<const VT *>(m.vind) + __ldg(static_cast<const int32_t *>(m.vs) + k));
        else
            v = __ldg(static_cast<const VT *>(m.vs) + k);
        s = fma(widen(v), widen(__ldg(x + static_cast<int64_t>(__ldg(m.col + k)) * ldx)), s);
    }
    return s;
}

// The row sum of a finished accumulator: a poisoned float-float sum is summed
// again from the CRS arrays of m (row r, operand x); anything else as it is.
template <typename VT, bool INDIRECT, typename XT, typename ACC>
__device__ __forceinline__ double acc_value(const ACC &a, const MatRef &m, int64_t r, const XT *__restrict__ x) {
    if constexpr (std::is_same<ACC, AccFF>::value || std::is_same<ACC, AccFR>::value ||
                  std::is_same<ACC, AccFRF>::value) {
        if (a.poisoned()) return row_sum_exact<VT, INDIRECT>(m, r, x);
    }
    return a.get();
}

template <typename V, typename X> __device__ __forceinline__ X ldg_x(const X *p) { return __ldg(p); }

}  // namespace spmv
