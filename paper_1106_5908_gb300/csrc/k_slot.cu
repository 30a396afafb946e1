// Compiled configurations of the slot-major chunk kernel (plan family 4) and its
// relayout kernel: FP64 values and vectors, and FP32 storage with FP32 runs and
// float-float carries (E = 7, 9, 11: at most 11 entries of a row per lane) or
// float-float accumulation (E = 15).
#include "internal.h"
#include "slot_kernel.cuh"

namespace spmv {

bool slot_ops_batched(int vk, int acc, int E, SlotOps *ops) {
    if (vk == kF64 && acc == kAccF64 && E == 7) {
        ops->launch = &SlotKernel<7, double, double, double, AccF64, false, true>::launch;
        return true;
    }
    if (vk == kF64 && acc == kAccF64 && E == 9) {
        ops->launch = &SlotKernel<9, double, double, double, AccF64, false, true>::launch;
        return true;
    }
    if (vk == kF32 && acc == kAccFF && E == 7) {
        ops->launch = &SlotKernel<7, float, float, float, AccFR, false, true>::launch;
        return true;
    }
    if (vk == kF32 && acc == kAccFF && E == 9) {
        ops->launch = &SlotKernel<9, float, float, float, AccFR, false, true>::launch;
        return true;
    }
    return false;
}

bool slot_ops(int vk, int xk, int yk, int acc, int E, bool pre, SlotOps *ops) {
    if (pre) {
        // row-mapped products (the split's nonlocal part): FP64, E = 7 (E = 9
        // measured no faster there: split 230.9 against 229.4 us)
        if (vk == kF64 && xk == kF64 && yk == kF64 && acc == kAccF64 && E == 7) {
            ops->launch = &SlotKernel<7, double, double, double, AccF64, true>::launch;
            return true;
        }
        return false;
    }
#define SPMV_S(VK_, XK_, YK_, ACCK_, E_, VT_, XT_, YT_, ACC_)                                 \
    if (vk == VK_ && xk == XK_ && yk == YK_ && acc == ACCK_ && E == E_) {                     \
        ops->launch = &SlotKernel<E_, VT_, XT_, YT_, ACC_>::launch;                            \
        return true;                                                                          \
    }
    SPMV_S(kF64, kF64, kF64, kAccF64, 7, double, double, double, AccF64)
    SPMV_S(kF64, kF64, kF64, kAccF64, 9, double, double, double, AccF64)
    SPMV_S(kF64, kF64, kF64, kAccF64, 11, double, double, double, AccF64)
    SPMV_S(kF64, kF64, kF64, kAccF64, 15, double, double, double, AccF64)
    SPMV_S(kF32, kF32, kF32, kAccFF, 7, float, float, float, AccFR)
    SPMV_S(kF32, kF32, kF32, kAccFF, 9, float, float, float, AccFR)
    SPMV_S(kF32, kF32, kF32, kAccFF, 11, float, float, float, AccFR)
    SPMV_S(kF32, kF32, kF32, kAccFF, 15, float, float, float, AccFF)
#undef SPMV_S
    return false;
}

cudaError_t launch_slot_mixed(int vk, int acc, const SlotParams &p7, const SlotParams &p9, cudaStream_t s) {
    if (vk == kF64 && acc == kAccF64) return SlotKernelMixed<double, double, double, AccF64>::launch(p7, p9, s);
    if (vk == kF32 && acc == kAccFF) return SlotKernelMixed<float, float, float, AccFR>::launch(p7, p9, s);
    return cudaErrorInvalidValue;
}

bool slot_ops_tv(int vk, int xk, int yk, int acc, int E, SlotOps *ops) {
    if (vk == kF64 && xk == kF64 && yk == kF64 && acc == kAccF64) {
        if (E == 7) { ops->launch = &SlotKernelTV<7, double, double, double, AccF64>::launch; return true; }
        if (E == 9) { ops->launch = &SlotKernelTV<9, double, double, double, AccF64>::launch; return true; }
    }
    if (vk == kF32 && xk == kF32 && yk == kF32 && acc == kAccFF) {
        if (E == 9) { ops->launch = &SlotKernelTV<9, float, float, float, AccFF>::launch; return true; }
        if (E == 15) { ops->launch = &SlotKernelTV<15, float, float, float, AccFF>::launch; return true; }
    }
    return false;
}

cudaError_t launch_slot_relayout(const void *chunks, int E, int64_t n_slots, int vk, const void *val,
                                 const int32_t *col, void *vals_out, int32_t *cols_out, cudaStream_t s) {
    if (n_slots <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n_slots + 255) / 256;
    const int grid = static_cast<int>(want < 16LL * sms ? want : 16LL * sms);
    const ChunkDesc *d = static_cast<const ChunkDesc *>(chunks);
    if (vk == kF64)
        k_slot_relayout<double><<<grid, 256, 0, s>>>(d, E, n_slots, static_cast<const double *>(val), col,
                                                     static_cast<double *>(vals_out), cols_out);
    else
        k_slot_relayout<float><<<grid, 256, 0, s>>>(d, E, n_slots, static_cast<const float *>(val), col,
                                                    static_cast<float *>(vals_out), cols_out);
    return cudaGetLastError();
}

}  // namespace spmv
