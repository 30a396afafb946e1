// Internal declarations shared by the translation units of the library (not part
// of the public ABI in include/spmv.h): the compiled configurations of each
// kernel family and the launchers of the auxiliary kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "types.h"
#include "cg.h"

namespace spmv {

// One compiled configuration of the tile kernel.
struct TileOps {
    cudaError_t (*launch)(const KParams &, int grid, cudaStream_t);
    int (*grid_limit)();   // CTAs resident on the whole GPU (persistent grid)
    TileCfg (*cfg)();
};

// Look up a compiled configuration.  vk/xk/yk: value and vector kinds, acc:
// accumulator, R: group width (1 for a single vector, right-hand sides per group
// for block vectors), E: entries per segment, indirect: values read through a
// permutation (transposed apply), batched: per-tile matrix table.
bool tile_ops(int vk, int xk, int yk, int acc, int R, int E, bool indirect, bool batched,
              TileOps *ops);
bool tile_ops_f64(int R, int E, bool indirect, bool batched, TileOps *ops);
bool tile_ops_f32(int xk, int yk, int acc, int R, int E, bool indirect, bool batched,
                  TileOps *ops);

struct WarpParams;
// One compiled configuration of the warp-chunk kernel (single right-hand side).
struct WarpOps {
    cudaError_t (*launch)(const WarpParams &, int n_chunks, cudaStream_t);
};
bool warp_ops(int vk, int xk, int yk, int acc, int E, bool indirect, bool batched, WarpOps *ops);
bool warp_ops_f64(int E, bool indirect, bool batched, WarpOps *ops);
bool warp_ops_f32(int yk, int acc, int E, bool indirect, bool batched, WarpOps *ops);

struct SlotParams;
// One compiled configuration of the slot-major chunk kernel (plan family 4).
struct SlotOps {
    cudaError_t (*launch)(const SlotParams &, cudaStream_t);
};
// pre: the variant that loads each chunk's row map and old y before its chains
// (row-mapped products).
bool slot_ops(int vk, int xk, int yk, int acc, int E, bool pre, SlotOps *ops);
// The batched launch over two groups of members tuned apart (7 and 9 entries per
// lane, each group with its own slot-major copy): FP64, FP32 float-float.
cudaError_t launch_slot_mixed(int vk, int acc, const SlotParams &p7, const SlotParams &p9, cudaStream_t s);
// The variant whose values arrive by bulk copies into a shared-memory ring
// (plan family 6): FP64 E = 7, 9; FP32 float-float E = 9, 15.
bool slot_ops_tv(int vk, int xk, int yk, int acc, int E, SlotOps *ops);
// The batched variant (vectors of the value type): FP64, FP32 float-float; E = 7.
bool slot_ops_batched(int vk, int acc, int E, SlotOps *ops);
// Slot-major copies of the values (and, when cols_out is not null, the column
// indices) of the regular chunks in `chunks` (ChunkDesc[n_slots / (32E)]).
cudaError_t launch_slot_relayout(const void *chunks, int E, int64_t n_slots, int vk, const void *val,
                                 const int32_t *col, void *vals_out, int32_t *cols_out, cudaStream_t s);

struct SellParams;
// One compiled configuration of the sorted row-slice kernel (plan family 5):
// (F64, F64, F64) with FP64 FMAs and (F32, F32, F32) with float-float sums.
struct SellOps {
    cudaError_t (*launch)(const SellParams &, cudaStream_t);
    int (*ctas_for)(int32_t n_slices);  // CTAs a launch over n_slices uses
    // y = A x plus the dot x.y reduced into a CG reduction target (FP32
    // storage only; nullptr elsewhere)
    cudaError_t (*launch_dot)(const SellParams &, const RedOut &, cudaStream_t);
};
// max_row: the longest row of the matrix; FP32 storage with the default
// accumulator takes FP32 runs (AccFR) when no row exceeds 11 entries, else FP32
// runs of one block folded into float-float (AccFRF).
bool sell_ops(int vk, int xk, int yk, int acc, SellOps *ops, int32_t max_row = 0x7fffffff);
// Block vectors on the sorted row slices, 4 right-hand sides:
// Y[i*ldy + r] = alpha*sum_j a_ij X[j*ldx + r] + beta*Y[i*ldy + r], r = 0..3
// (b carries the slices, alpha and beta; its x and y are not used).  vec: X, Y,
// ldx and ldy allow 16-byte accesses.
cudaError_t launch_sell_mr(const SellParams &b, const double *X, double *Y, int64_t ldx, int64_t ldy, bool vec,
                           cudaStream_t s);
// Slot-major copies of the values (and, when cols_out is not null, the column
// indices) of the regular slices in `slices` (int2[n_slices]; srows: 32 rows per
// slice) from the CRS arrays rp, val, col.
cudaError_t launch_sell_relayout(const void *slices, const int32_t *srows, int32_t n_slices, const int32_t *rp,
                                 int vk, const void *val, const int32_t *col, void *vals_out, int32_t *cols_out,
                                 cudaStream_t s);

cudaError_t launch_rowvec(const KParams &p, const int32_t n_rows, int vk, int xk, int yk, int acc,
                          int T, cudaStream_t s);

// out[k] = val[perm[k]] for k < nnz (values of kind vk: FP64 or FP32).
cudaError_t launch_permute(const void *val, const int32_t *perm, void *out, int64_t nnz, int vk, cudaStream_t s);
// Device-side CRS check; sets *bad to 1 on any violation.
cudaError_t launch_validate(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                            int32_t *bad, cudaStream_t s);
// One warp waits on an mbarrier nothing completes, for limit_ns, then records
// kDevErrTimeout in *err.
cudaError_t launch_wait_timeout(uint64_t limit_ns, int32_t *err, cudaStream_t s);
// Halo gather: halo[h] = x[map[h]].
cudaError_t launch_gather(const double *x, const int32_t *map, double *halo, int64_t n,
                          cudaStream_t s);

// grad_val over the warp chunks of A (ChunkDesc table + row-start bitmasks with
// mwp words per chunk): chunks of kGradValE entries per lane, mwp = kGradValWords
// (other tables are rejected with cudaErrorInvalidValue).
constexpr int kGradValE = 7;
constexpr int kGradValWords = 8;
cudaError_t launch_grad_val_chunks(const int32_t *rp, const int32_t *col, const void *chunks,
                                   const uint32_t *masks, int mwp, int32_t n_chunks, int vk,
                                   const void *g, const void *x, double alpha, void *grad_val,
                                   cudaStream_t s);

// Transposed structure: counts, exclusive scan, fill, per-row ordering.
cudaError_t launch_transpose(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp,
                             const int32_t *col, int32_t *rowT, int32_t *colT, int32_t *perm,
                             int32_t *work, cudaStream_t s);

// Transposed structure into caller buffers with the fixed device work array
// (no allocation); n_cols <= transpose_noalloc_max_cols().
cudaError_t launch_transpose_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                     const int32_t *col, int32_t *rowT, int32_t *colT, int32_t *perm,
                                     cudaStream_t s);
int64_t transpose_noalloc_max_cols();

// Value conversion (FP64 <-> FP32), n entries.
cudaError_t launch_convert(const void *src, int sk, void *dst, int dk, int64_t n, cudaStream_t s);

// Vector kernels of the CG solvers (see cg.cu).
cudaError_t launch_fill(void *p, int k, double v, int64_t n, cudaStream_t s);

}  // namespace spmv
