// The warp-chunk CRS kernel (single right-hand side).
//
// Listing 1 (Sect. 1.2) sums val(j)*B(col_idx(j)) over the entries of each row.
// On GB300 the FP64 FMA rate (about 1.2 TFLOP/s) is close to what an HBM-rate
// spMVM needs, so the kernel keeps every lane of every FP64 FMA busy and adds no
// per-entry FP64 work, and it keeps enough loads in flight to cover HBM and L2
// latency without shared-memory staging or CTA barriers:
//
//   * The matrix is cut (once, on the host) into chunks of whole rows whose
//     entries fit in 32*E slots counted from the 16-byte aligned start below the
//     chunk's first entry.  Each chunk carries a bitmask with one bit per slot,
//     set where a row starts.  One warp processes one chunk.
//   * Lane l owns the E consecutive slots [16-byte base + l*E, ... + E).  It loads
//     its values and column indices with 128-bit loads, then issues its E x
//     gathers before any arithmetic, so E gathers per lane are in flight.
//   * One FMA chain per lane runs over its slots; at a set bit the running row
//     sum is final (stored to a per-warp row buffer in shared memory) unless the
//     row began in an earlier lane.  A row cut by lane boundaries is combined in
//     lane order through shuffles (one FP64 add per crossing), so results are
//     deterministic.  Finished rows leave the row buffer row-contiguously with
//     the alpha/beta update.
//   * Chunks that contain empty rows take a row-per-lane path; a row too long for
//     a chunk forms its own chunk reduced by the whole warp.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace spmv {

// Chunk descriptor: rows [r0, r1), entries [k0, k1), flags in the top bits of r1.
struct alignas(16) ChunkDesc {
    int32_t k0, k1, r0, r1f;
};
constexpr int32_t kChunkLong = 1 << 30;   // one row longer than a chunk
constexpr int32_t kChunkEmpty = 1 << 29;  // chunk contains empty rows
constexpr int32_t kChunkRowMask = (1 << 29) - 1;
constexpr int kWarpRowCap = 96;           // rows per chunk (per-warp row buffer)

struct WarpParams {
    MatRef m;
    const MatRef *mats;           // batched: per-chunk matrix table (index in cmat)
    const ChunkDesc *chunks;
    const uint32_t *masks;        // (32*E/32) words per chunk
    const int32_t *cmat;          // batched: matrix of each chunk
    int32_t n_chunks;
    double alpha, beta;
    int32_t *err;
};

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec4<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec4<int32_t> { using type = int4; static constexpr int N = 4; };

// Load E consecutive elements starting at a 16-byte aligned address with 128-bit
// loads; groups of 4 elements past `valid` (count from p) are not read.
template <int E, typename T>
__device__ __forceinline__ void load_run(const T *__restrict__ p, int valid, T (&out)[E]) {
    using V = typename Vec4<T>::type;
    constexpr int N = Vec4<T>::N;
#pragma unroll
    for (int g = 0; g < E / N; ++g) {
        V v{};
        if (g * N < valid) v = __ldg(reinterpret_cast<const V *>(p) + g);
        if constexpr (N == 2) {
            out[g * 2] = reinterpret_cast<T *>(&v)[0];
            out[g * 2 + 1] = reinterpret_cast<T *>(&v)[1];
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) out[g * 4 + q] = reinterpret_cast<T *>(&v)[q];
        }
    }
}

template <typename YT>
__device__ __forceinline__ void store_row(YT *__restrict__ y, int64_t row, double v, double alpha,
                                          double beta, bool plain, const int32_t *rmap) {
    if (rmap) row = __ldg(rmap + row);
    double out;
    if (plain) out = v;
    else if (beta == 0.0) out = alpha * v;
    else out = fma(alpha, v, beta * widen(y[row]));
    y[row] = narrow<YT>(out);
}

// Store the finished row sum of stored row `row` of m (output row through
// m.rmap).  A float-float sum bound for an FP32 y with alpha = 1, beta = 0 is
// rounded to float directly (h + l on the FP32 pipe); a poisoned one is summed
// again in FP64; every other case goes through FP64.
template <typename VT, bool INDIRECT, typename XT, typename YT, typename ACC>
__device__ __forceinline__ void store_acc(const MatRef &m, const XT *__restrict__ x, YT *__restrict__ y,
                                          int64_t row, const ACC &a, double alpha, double beta, bool plain) {
    if constexpr (std::is_same<ACC, AccFF>::value || std::is_same<ACC, AccFR>::value) {
        if (a.poisoned()) {
            store_row(y, row, row_sum_exact<VT, INDIRECT>(m, row, x), alpha, beta, plain, m.rmap);
            return;
        }
        if constexpr (std::is_same<YT, float>::value) {
            if (plain) {
                y[m.rmap ? __ldg(m.rmap + row) : row] = a.h + a.l;
                return;
            }
        }
    }
    store_row(y, row, a.get(), alpha, beta, plain, m.rmap);
}

// Form of the update y = alpha*v + beta*y, decided once per launch so that no
// FP64 comparison or multiply by 1 runs per row: kEpiPlain y = v; kEpiScale
// y = alpha*v; kEpiAdd y = v + y (alpha = beta = 1, as in the nonlocal part of
// the split product); kEpiGeneral y = fma(alpha, v, beta*y).
constexpr int kEpiPlain = 0, kEpiScale = 1, kEpiAdd = 2, kEpiGeneral = 3;
__host__ __device__ __forceinline__ int epi_mode(double alpha, double beta) {
    if (beta == 0.0) return alpha == 1.0 ? kEpiPlain : kEpiScale;
    return (alpha == 1.0 && beta == 1.0) ? kEpiAdd : kEpiGeneral;
}

// Row epilogue of a regular chunk (at most kWarpRowCap rows, lane l owns rows
// l, l+32, l+64): the output index of each row (through rmap) and, when beta is
// nonzero, its old y value are loaded before the FMA chains run, so that their
// latency overlaps the chains instead of following them.
template <typename YT>
struct RowEpilogue {
    static constexpr int K = kWarpRowCap / 32;
    int64_t dst[K];
    double old[K];
    __device__ __forceinline__ void prefetch(const YT *__restrict__ y, const int32_t *__restrict__ rmap, int r0,
                                             int nrows, bool need_old, int lane) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = lane + 32 * k;
            dst[k] = r0 + q;
            if (rmap && q < nrows) dst[k] = __ldg(rmap + r0 + q);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = lane + 32 * k;
            old[k] = 0.0;
            if (need_old && q < nrows) old[k] = widen(y[dst[k]]);
        }
    }
    template <typename ACC>
    __device__ __forceinline__ void store(YT *__restrict__ y, const ACC *srow, int nrows, double alpha,
                                          double beta, int mode, int lane) const {
        static_assert(std::is_same<ACC, AccF64>::value, "row-mapped products accumulate in FP64");
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = lane + 32 * k;
            if (q >= nrows) break;
            const double v = srow[q].get();
            double out;
            if (mode == kEpiPlain) out = v;
            else if (mode == kEpiScale) out = alpha * v;
            else if (mode == kEpiAdd) out = v + old[k];
            else out = fma(alpha, v, beta * old[k]);
            y[dst[k]] = narrow<YT>(out);
        }
    }
};

__device__ __forceinline__ AccF64 shfl_up_acc(const AccF64 &a, int d) {
    AccF64 b;
    b.s = __shfl_up_sync(0xffffffffu, a.s, d);
    return b;
}
__device__ __forceinline__ AccFF shfl_up_acc(const AccFF &a, int d) {
    AccFF b;
    b.h = __shfl_up_sync(0xffffffffu, a.h, d);
    b.l = __shfl_up_sync(0xffffffffu, a.l, d);
    return b;
}
__device__ __forceinline__ AccFR shfl_up_acc(const AccFR &a, int d) {
    AccFR b;
    b.h = __shfl_up_sync(0xffffffffu, a.h, d);
    b.l = __shfl_up_sync(0xffffffffu, a.l, d);
    return b;
}
__device__ __forceinline__ AccF64 shfl_xor_acc2(const AccF64 &a, int d) {
    AccF64 b;
    b.s = __shfl_xor_sync(0xffffffffu, a.s, d);
    return b;
}
__device__ __forceinline__ AccFF shfl_xor_acc2(const AccFF &a, int d) {
    AccFF b;
    b.h = __shfl_xor_sync(0xffffffffu, a.h, d);
    b.l = __shfl_xor_sync(0xffffffffu, a.l, d);
    return b;
}

// A row too long for a chunk: lanes stride the row, then a butterfly reduction.
template <typename VT, typename XT, typename YT, typename ACC, bool INDIRECT>
__device__ __forceinline__ void long_row(const MatRef &m, const ChunkDesc &d, const XT *__restrict__ x,
                                         YT *__restrict__ y, double alpha, double beta, bool plain,
                                         int lane) {
    typename WholeRowAcc<ACC>::type acc;
    acc.zero();
    for (int k = d.k0 + lane; k < d.k1; k += 32) {
        const XT xv = __ldg(x + __ldg(m.col + k));
        if constexpr (INDIRECT)
            acc.fma(__ldg(static_cast<const VT *>(m.vind) + __ldg(static_cast<const int32_t *>(m.vs) + k)), xv);
        else
            acc.fma(__ldg(static_cast<const VT *>(m.vs) + k), xv);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc.add(shfl_xor_acc2(acc, o));
    if (lane == 0) store_acc<VT, INDIRECT>(m, x, y, d.r0, acc, alpha, beta, plain);
}

// A chunk with empty rows: one row per lane straight from global memory.
template <typename VT, typename XT, typename YT, typename ACC, bool INDIRECT>
__device__ __forceinline__ void rows_per_lane(const MatRef &m, int r0, int r1, const XT *__restrict__ x,
                                              YT *__restrict__ y, double alpha, double beta, bool plain,
                                              int lane) {
    for (int r = r0 + lane; r < r1; r += 32) {
        typename WholeRowAcc<ACC>::type acc;
        acc.zero();
        const int kb = __ldg(m.rp + r), ke = __ldg(m.rp + r + 1);
        for (int k = kb; k < ke; ++k) {
            const XT xv = __ldg(x + __ldg(m.col + k));
            if constexpr (INDIRECT)
                acc.fma(__ldg(static_cast<const VT *>(m.vind) + __ldg(static_cast<const int32_t *>(m.vs) + k)), xv);
            else
                acc.fma(__ldg(static_cast<const VT *>(m.vs) + k), xv);
        }
        store_acc<VT, INDIRECT>(m, x, y, r, acc, alpha, beta, plain);
    }
}

// One lane's share of a regular chunk.  vals/xv hold the lane's E slots (zero in
// slots outside [lo, hi)); bit e of mbits is set where a row starts in slot e;
// `ends` says whether the lane's last row ends with its slots.  The FMA chain
// restarts at every row start (a register select, no branch); a row that starts
// and ends in this lane is in the row buffer once its last slot is done (FP64:
// stored at that slot only; float-float: stored after every slot).  The part of
// the first row that started in an earlier lane is combined in lane order with
// the carries of those lanes (one add per crossing) and stored by the lane where
// the row ends.
// `pre` is the number of rows starting in the chunk before this lane's slots.
template <int E, typename VT, typename XT, typename ACC>
__device__ __forceinline__ void chunk_lane_pre(const VT (&vals)[E], const XT (&xv)[E], uint32_t mbits,
                                               int lo, int hi, bool ends, int pre, int r0, ACC *srow,
                                               int lane, int chain = -1) {
    const bool active = lo < hi;
    const bool starts_first = active && ((mbits >> lo) & 1u);
    int row = r0 + pre + (starts_first ? 1 : 0) - 1;  // row of slot lo
    const int first_row = row;
    const uint32_t flush = active ? (mbits & ~(1u << lo)) : 0u;
    // slots in [lo, hi) after which a row ends: the next slot starts one, or the
    // slot is the lane's last and `ends`
    const uint32_t span = active ? ((hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u)) : 0u;
    const uint32_t endm = ((mbits >> 1) | ((active && ends) ? (1u << (hi - 1)) : 0u)) & span;
    // FP64 and FP32-run sums store at row ends only (fewer shared-memory
    // wavefronts for a kernel bound by L1TEX and the FP64 pipe: C2 150.4 ->
    // 149.9 us, E = 11 163.8 -> 156.5 us); the float-float kernels, bound by
    // instruction issue, store after every slot once the row has started (the
    // row-end test costs them 3-6 %), so the last store of a row is its full sum
    constexpr bool kRowEndStores = !std::is_same<ACC, AccFF>::value;
    static_assert(!std::is_same<ACC, AccFR>::value || E <= kFRMaxRun, "FP32 runs of at most kFRMaxRun entries");
    // per-slot decisions as bit masks, formed once: capm = the slot before which
    // the piece of a row begun in an earlier lane ends (the first row start
    // after slot lo, unless slot lo starts one); startm = the slots at and
    // after the first row start of the lane; storem = the slots whose running
    // sum is stored
    const uint32_t low = flush & (0u - flush);
    const uint32_t capm = starts_first ? 0u : low;
    const uint32_t startm = starts_first ? span : (low ? (span & ~(low - 1u)) : 0u);
    const uint32_t storem = kRowEndStores ? (endm & startm) : startm;
    const bool started = startm != 0u;  // a row starts in the lane's slots
    ACC acc;
    acc.zero();
    ACC pend;
    pend.zero();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool b = (flush >> e) & 1u;
        if ((capm >> e) & 1u) pend = acc;
        if (b) acc.zero();
        row += b ? 1 : 0;
        acc.fma(vals[e], xv[e]);
        if ((storem >> e) & 1u) srow[row - r0] = acc;
    }
    bool has_pend = capm != 0u;
    if (active && !started && ends) {
        pend = acc;
        has_pend = true;
    }
    const bool carry = active && !ends;
    const bool through = carry && !started;  // the lane's slots lie inside one row
    ACC tot = pend;
    if (chain >= 0) {
        // chain: how many earlier lanes' sums this lane adds (from the host: 1 +
        // the through lanes just before it, 0 without a pending piece); the
        // warp runs the longest chain, with no vote per step
        const int longest = __reduce_max_sync(0xffffffffu, chain);
        for (int dist = 1; dist <= longest; ++dist) {
            const ACC c = shfl_up_acc(acc, dist);
            if (dist <= chain) {
                ACC t2 = c;
                t2.add(tot);
                tot = t2;
            }
        }
    } else {
        int dist = 1;
        bool need = has_pend;
        while (__any_sync(0xffffffffu, need)) {
            const ACC c = shfl_up_acc(acc, dist);
            const bool cthrough = __shfl_up_sync(0xffffffffu, through, dist);
            if (need) {
                ACC t2 = c;
                t2.add(tot);
                tot = t2;
                need = cthrough;
            }
            ++dist;
        }
    }
    if (has_pend) srow[first_row - r0] = tot;
}

// As chunk_lane_pre, with `pre` from a shuffle scan of the lanes' row-start counts.
template <int E, typename VT, typename XT, typename ACC>
__device__ __forceinline__ void chunk_lane(const VT (&vals)[E], const XT (&xv)[E], uint32_t mbits,
                                           int lo, int hi, bool ends, int r0, ACC *srow, int lane,
                                           int chain = -1) {
    const int cnt = __popc(mbits);
    int pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += t;
    }
    pre -= cnt;
    chunk_lane_pre<E, VT, XT, ACC>(vals, xv, mbits, lo, hi, ends, pre, r0, srow, lane, chain);
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
__global__ void __launch_bounds__(256) k_warp(const WarpParams p) {
    static_assert(E == 8 || E == 16, "E is 8 or 16");
    constexpr int SLOTS = 32 * E;
    constexpr int MW = SLOTS / 32;  // mask words per chunk
    using VS = typename std::conditional<INDIRECT, int32_t, VT>::type;
    static_assert(sizeof(ACC) == 8, "row buffer entries are 8 bytes");
    __shared__ ACC s_rows[8][kWarpRowCap];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t w = static_cast<int64_t>(blockIdx.x) * 8 + wib;
    if (w >= p.n_chunks) return;
    const ChunkDesc d = p.chunks[w];
    MatRef m;
    if constexpr (BATCHED) m = p.mats[p.cmat[w]];
    else m = p.m;
    const XT *__restrict__ x = static_cast<const XT *>(m.x);
    YT *__restrict__ y = static_cast<YT *>(m.y);
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);
    const int r0 = d.r0;
    const int r1 = d.r1f & kChunkRowMask;

    if (d.r1f & kChunkLong) {
        long_row<VT, XT, YT, ACC, INDIRECT>(m, d, x, y, alpha, beta, plain, lane);
        return;
    }
    if (d.r1f & kChunkEmpty) {
        rows_per_lane<VT, XT, YT, ACC, INDIRECT>(m, r0, r1, x, y, alpha, beta, plain, lane);
        return;
    }

    // ---- regular chunk -----------------------------------------------------
    const int base = d.k0 & ~3;
    const int seg = base + lane * E;
    const int lo = max(0, d.k0 - seg);          // first valid slot of the lane
    const int hi = min(E, d.k1 - seg);          // one past the last valid slot
    uint32_t mbits;
    if constexpr (E == 16) {
        const uint32_t word = __ldg(p.masks + w * MW + (lane >> 1));
        mbits = (word >> ((lane & 1) * 16)) & 0xffffu;
    } else {
        const uint32_t word = __ldg(p.masks + w * MW + (lane >> 2));
        mbits = (word >> ((lane & 3) * 8)) & 0xffu;
    }
    VS vv[E];
    int32_t cc[E];
    XT xv[E];
    load_run<E>(static_cast<const VS *>(m.vs) + seg, hi, vv);
    load_run<E>(m.col + seg, hi, cc);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        xv[e] = XT(0);
        if (e >= lo && e < hi) xv[e] = __ldg(x + cc[e]);
    }
    VT vals[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        vals[e] = VT(0);
        if (e >= lo && e < hi) {
            if constexpr (INDIRECT) vals[e] = __ldg(static_cast<const VT *>(m.vind) + vv[e]);
            else vals[e] = vv[e];
        }
    }
    const uint32_t next_bits = __shfl_down_sync(0xffffffffu, mbits, 1);
    const bool ends = (seg + E >= d.k1) || (lane < 31 && (next_bits & 1u));
    ACC *srow = s_rows[wib];
    chunk_lane<E, VT, XT, ACC>(vals, xv, mbits, lo, hi, ends, r0, srow, lane);
    __syncwarp();
    for (int i = lane; i < r1 - r0; i += 32) store_acc<VT, INDIRECT>(m, x, y, r0 + i, srow[i], alpha, beta, plain);
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
struct WarpKernel {
    static cudaError_t launch(const WarpParams &p, int n_chunks, cudaStream_t s) {
        if (n_chunks <= 0) return cudaSuccess;
        const int grid = (n_chunks + 7) / 8;
        k_warp<E, VT, XT, YT, ACC, INDIRECT, BATCHED><<<grid, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
};
}  // namespace spmv
