// Types and constants the kernels share (operand descriptors, padding, kinds):
// the definitions device code is compiled from.  The host-side declarations of
// the compiled configurations and launchers are in internal.h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spmv {

// A tile is a run of whole rows [r0, r1) whose entries [k0, k1) are staged in
// shared memory together.  A tile with one row and more entries than a tile
// holds ("long row") is reduced by the whole CTA straight from global memory.
// mat indexes the matrix table of a batched launch (0 otherwise).
struct alignas(32) TileDesc {
    int32_t r0, r1, k0, k1;
    int32_t mat, pad0, pad1, pad2;
};

// Operands of one matrix.  The tile kernel streams two per-entry arrays through
// shared memory: `col` (the gather index into x) and `vs` (the values, or, for
// the transposed apply, the permutation into `vind` that holds the values).
struct MatRef {
    const int32_t *rp;    // row_ptr, padded (see kRowPad)
    const int32_t *col;   // per-entry gather index, padded (see kEntryPad)
    const void *vs;       // per-entry values (VT) or permutation (int32)
    const void *vind;     // values read through the permutation, or nullptr
    const void *x;        // dense input, element (j, r) at x[j*ldx + r]
    void *y;              // dense output, element (i, r) at y[i*ldy + r]
    const int32_t *rmap;  // optional: output row of each stored row (nullptr = identity)
};

struct KParams {
    MatRef m;                 // the matrix of a single launch
    const MatRef *mats;       // per-matrix table of a batched launch
    const TileDesc *tiles;
    int32_t n_tiles;
    int32_t rhs_count;        // right-hand sides handled by this launch (<= group width)
    int64_t ldx, ldy;
    double alpha, beta;
    int32_t *err;             // device error word
};

// Arrays handed to the tile kernel are padded so the 16-byte aligned bulk copies
// may read a few entries past the logical end.
constexpr int kEntryPad = 16;
constexpr int kRowPad = 16;

// Device error codes written into the error word.
constexpr int32_t kDevErrTimeout = 1;

// Kernel configuration chosen per matrix by the autotuner.
enum ValKind : int32_t { kF64 = 0, kF32 = 1 };
enum AccKind : int32_t { kAccF64 = 0, kAccFF = 1 };

struct TileCfg {
    int32_t E;        // entries per thread segment (odd)
    int32_t threads;  // CTA size
    int32_t rowcap;   // rows per tile cap
    int32_t cap;      // entries per tile = (threads / group) * E
};

}  // namespace spmv
