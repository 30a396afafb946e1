// Slot-major warp-chunk kernel (plan family 4).
//
// Same chunking (whole rows, at most 32*E entries and kWarpRowCap rows per
// chunk), row-start bits, per-lane FMA chains and lane-order carries as the
// staged chunk kernels, with a different home for the streamed operands: the
// values and column indices of each regular chunk are stored once in slot-major
// order, entry k0 + l*E + e of the chunk at [chunk][e][l].  The e-th load of a
// warp therefore reads 32 consecutive elements (one coalesced access), nothing
// is staged in shared memory, and the streamed loads bypass L1 (evict-first in
// L2), which leaves the whole L1 to the x gathers.  A warp keeps the next
// chunk's gathers and values and the chunk after's column indices in flight in
// registers while its FMA chains run.
#pragma once
#include "warp_kernel.cuh"

namespace spmv {

// Lane word of a regular chunk: bit e (e < E <= 15) = a row starts at slot
// l*E + e; bits 16-22 = rows starting in the chunk before the lane's slots; bit
// 23 = the lane's last slot ends a row or the chunk.  All follow from the row
// starts, so they are set once on the host and the kernel needs no cross-lane
// scan for them.
constexpr int kSlotPreShift = 16;
constexpr uint32_t kSlotPreMask = 0x7fu;
constexpr uint32_t kSlotEnds = 1u << 23;
// bits 24-28: the lane's carry chain, how many earlier lanes' sums it adds (1
// + the lanes just before it that lie inside one row, 0 when its first slot
// starts a row or it holds no entries)
constexpr int kSlotChainShift = 24;
constexpr uint32_t kSlotChainMask = 0x1fu;

struct SlotParams {
    const ChunkDesc *chunks;
    const uint32_t *lmask;  // 32 words per chunk (kSlotPre*, kSlotEnds below)
    const void *vals;       // n_chunks * 32E values, slot-major (zero in padding)
    const int32_t *cols;    // n_chunks * 32E column indices, slot-major (zero in padding)
    MatRef m;               // the CRS itself (long and empty-row chunks), x, y, row map
    const MatRef *mats;     // batched: the matrix table (index in cmat per chunk)
    const int32_t *cmat;
    int32_t n_chunks;
    double alpha, beta;
    int32_t *err;           // device error word (the staged variant's bounded waits)
};

__device__ __forceinline__ double ld_stream(const double *p, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Whether a configuration takes the lanes' row counts from a shuffle scan
// instead of the packed lane words: only FP64 with E = 9 (150.1 against
// 152.5 us on the Hamiltonian-like matrix; the packed words win elsewhere, e.g.
// E = 11 154 against 169 us, the split's nonlocal part 256 against 262 us).
template <int E, typename VT, bool PRE>
struct kSlotScan {
    static constexpr bool value = std::is_same<VT, double>::value && E == 9 && !PRE;
};

// PRE: the row epilogue's operands (row map, old y) are loaded before the FMA
// chains (row-mapped products: the nonlocal part of the split form).
// BATCHED: chunks of many matrices in one launch; chunk c belongs to matrix
// cmat[c] of the table mats (its own x, y and CRS arrays).
// The persistent loop of one warp over chunks c, c + nwarps, ... of p (srow:
// the warp's row buffer).
template <int E, typename VT, typename XT, typename YT, typename ACC, bool PRE, bool BATCHED>
__device__ __forceinline__ void slot_loop(const SlotParams &p, ACC *srow, int c, int nwarps) {
    constexpr int SL = 32 * E;
    const int lane = threadIdx.x & 31;
    const int n = p.n_chunks;
    if (c >= n) return;
    const uint64_t pol = l2_evict_first_policy();
    const VT *__restrict__ vals = static_cast<const VT *>(p.vals);
    const double alpha = p.alpha, beta = p.beta;
    auto mat_of = [&](int cc) -> MatRef {
        if constexpr (BATCHED) return p.mats[p.cmat[cc]];
        else return p.m;
    };
    const bool plain = (alpha == 1.0 && beta == 0.0);
    const int emode = epi_mode(alpha, beta);

    auto regular = [](const ChunkDesc &d) { return (d.r1f & (kChunkLong | kChunkEmpty)) == 0; };
    auto hi_of = [&](const ChunkDesc &d) { return max(0, min(E, d.k1 - d.k0 - lane * E)); };
    auto load_cols = [&](int cc, int32_t (&cl)[E]) {
        const int32_t *b = p.cols + static_cast<int64_t>(cc) * SL + lane;
#pragma unroll
        for (int e = 0; e < E; ++e) cl[e] = ld_stream(b + e * 32, pol);
    };
    auto load_vals = [&](int cc, VT (&v)[E]) {
        const VT *b = vals + static_cast<int64_t>(cc) * SL + lane;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ld_stream(b + e * 32, pol);
    };
    auto xptr_of = [&](int cc) -> const XT * {
        if constexpr (BATCHED) return static_cast<const XT *>(p.mats[__ldg(p.cmat + cc)].x);
        else return static_cast<const XT *>(p.m.x);
    };
    auto gather = [&](const XT *__restrict__ x, const ChunkDesc &d, const int32_t (&cl)[E], XT (&xv)[E]) {
        const int hi = regular(d) ? hi_of(d) : 0;
#pragma unroll
        for (int e = 0; e < E; ++e) xv[e] = (e < hi) ? __ldg(x + cl[e]) : XT(0);
    };
    auto load_desc = [&](int cc) {
        const int4 q = __ldg(reinterpret_cast<const int4 *>(p.chunks) + cc);
        return ChunkDesc{q.x, q.y, q.z, q.w};
    };

    // chunk c: descriptor, row starts, gathers, values; chunk c + nwarps:
    // descriptor, row starts, column indices
    ChunkDesc dc = load_desc(c);
    uint32_t mc = __ldg(p.lmask + static_cast<int64_t>(c) * 32 + lane);
    XT xc[E];
    VT vc[E];
    {
        int32_t cl[E];
        load_cols(c, cl);
        gather(xptr_of(c), dc, cl, xc);
        load_vals(c, vc);
    }
    ChunkDesc dn{};
    uint32_t mn = 0;
    const XT *xpn = nullptr;
    int32_t cn[E];
#pragma unroll
    for (int e = 0; e < E; ++e) cn[e] = 0;
    if (c + nwarps < n) {
        xpn = xptr_of(c + nwarps);
        dn = load_desc(c + nwarps);
        mn = __ldg(p.lmask + static_cast<int64_t>(c + nwarps) * 32 + lane);
        load_cols(c + nwarps, cn);
    }

    for (; c < n; c += nwarps) {
        const int c1 = c + nwarps, c2 = c + 2 * nwarps;
        // chunk c1: gathers and values; chunk c2: descriptor, row starts, columns
        XT xn[E];
        VT vn[E];
        if (c1 < n) {
            gather(xpn, dn, cn, xn);
            load_vals(c1, vn);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                xn[e] = XT(0);
                vn[e] = VT(0);
            }
        }
        ChunkDesc d2{};
        uint32_t m2 = 0;
        const XT *xp2 = nullptr;
        int32_t c2l[E];
        if (c2 < n) {
            xp2 = xptr_of(c2);
            d2 = load_desc(c2);
            m2 = __ldg(p.lmask + static_cast<int64_t>(c2) * 32 + lane);
            load_cols(c2, c2l);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) c2l[e] = 0;
        }
        // ---- chunk c ---------------------------------------------------------
        const MatRef m = mat_of(c);
        const XT *__restrict__ x = static_cast<const XT *>(m.x);
        YT *__restrict__ y = static_cast<YT *>(m.y);
        const int r0 = dc.r0;
        const int r1 = dc.r1f & kChunkRowMask;
        if (dc.r1f & kChunkLong) {
            long_row<VT, XT, YT, ACC, false>(m, dc, x, y, alpha, beta, plain, lane);
        } else if (dc.r1f & kChunkEmpty) {
            rows_per_lane<VT, XT, YT, ACC, false>(m, r0, r1, x, y, alpha, beta, plain, lane);
        } else {
            RowEpilogue<YT> epi;
            if constexpr (PRE) epi.prefetch(y, m.rmap, r0, r1 - r0, emode >= kEpiAdd, lane);
            const int hi = hi_of(dc);
            const uint32_t mbits = mc & ((1u << E) - 1u);
            if constexpr (kSlotScan<E, VT, PRE>::value) {
                const uint32_t next_bits = __shfl_down_sync(0xffffffffu, mbits, 1);
                const bool ends = (lane * E + E >= dc.k1 - dc.k0) || (lane < 31 && (next_bits & 1u));
                chunk_lane<E, VT, XT, ACC>(vc, xc, mbits, 0, hi, ends, r0, srow, lane,
                                           static_cast<int>((mc >> kSlotChainShift) & kSlotChainMask));
            } else {
                chunk_lane_pre<E, VT, XT, ACC>(vc, xc, mbits, 0, hi, (mc & kSlotEnds) != 0u,
                                               static_cast<int>((mc >> kSlotPreShift) & kSlotPreMask), r0,
                                               srow, lane,
                                               static_cast<int>((mc >> kSlotChainShift) & kSlotChainMask));
            }
            __syncwarp();
            if constexpr (PRE) {
                epi.store(y, srow, r1 - r0, alpha, beta, emode, lane);
            } else {
                for (int q = lane; q < r1 - r0; q += 32)
                    store_acc<VT, false>(m, x, y, r0 + q, srow[q], alpha, beta, plain);
            }
        }
        __syncwarp();  // the row buffer is free again
        dc = dn;
        mc = mn;
        dn = d2;
        mn = m2;
        xpn = xp2;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            xc[e] = xn[e];
            vc[e] = vn[e];
            cn[e] = c2l[e];
        }
    }
}

// CTAs per SM the register allocation must allow: FP64 with up to 11 entries
// per lane two (16 warps per SM, at most 128 registers; left free, the
// compiler takes 146-156 and halves the warps); FP32 storage with up to 9,
// single matrix, three (at most 80 registers, no spills: 134 against 138 us on
// the Hamiltonian-like matrix); the FP32 batch as the compiler chooses (held to
// 80 it spills: 256 matrices 0.85 against 0.655 ms).
template <int E, typename VT, bool BATCHED>
constexpr int slot_min_ctas() {
    return sizeof(VT) == 8 ? (E <= 11 ? 2 : 1) : ((E <= 9 && !BATCHED) ? 3 : ((E <= 11 && !BATCHED) ? 2 : 1));
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool PRE = false, bool BATCHED = false>
__global__ void __launch_bounds__(256, (slot_min_ctas<E, VT, BATCHED>())) k_slot(const SlotParams p) {
    static_assert(sizeof(ACC) == 8, "row buffer entries are 8 bytes");
    __shared__ ACC s_rows[8][kWarpRowCap];
    const int wib = threadIdx.x >> 5;
    slot_loop<E, VT, XT, YT, ACC, PRE, BATCHED>(p, s_rows[wib], blockIdx.x * 8 + wib, gridDim.x * 8);
}

// A batch whose members were tuned apart: the chunks of the members given 7
// entries per lane (p7, their own slot-major copy) and those given 9 (p9), one
// after the other in the same persistent launch (every warp takes its share of
// each group).
template <typename VT, typename XT, typename YT, typename ACC>
__global__ void __launch_bounds__(256, (slot_min_ctas<9, VT, true>())) k_slot_mixed(const SlotParams p7, const SlotParams p9) {
    static_assert(sizeof(ACC) == 8, "row buffer entries are 8 bytes");
    __shared__ ACC s_rows[8][kWarpRowCap];
    const int wib = threadIdx.x >> 5;
    slot_loop<7, VT, XT, YT, ACC, false, true>(p7, s_rows[wib], blockIdx.x * 8 + wib, gridDim.x * 8);
    __syncwarp();
    slot_loop<9, VT, XT, YT, ACC, false, true>(p9, s_rows[wib], blockIdx.x * 8 + wib, gridDim.x * 8);
}

template <typename VT, typename XT, typename YT, typename ACC>
struct SlotKernelMixed {
    static cudaError_t launch(const SlotParams &p7, const SlotParams &p9, cudaStream_t s) {
        static int cached = -1, cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached < 0 || cached_dev != dev) {
            int per_sm = 0, sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_slot_mixed<VT, XT, YT, ACC>, 256, 0) !=
                cudaSuccess)
                return cudaErrorInvalidConfiguration;
            cached = per_sm * sms;
            cached_dev = dev;
        }
        const int n = p7.n_chunks > p9.n_chunks ? p7.n_chunks : p9.n_chunks;
        if (n <= 0) return cudaSuccess;
        const int want = (n + 7) / 8;
        k_slot_mixed<VT, XT, YT, ACC><<<want < cached ? want : cached, 256, 0, s>>>(p7, p9);
        return cudaGetLastError();
    }
};

// Staged-values variant (TV).  The values of each chunk (32E contiguous
// elements of the slot-major copy) arrive by one 1-D bulk copy (cp.async.bulk,
// evict-first in L2) into a two-stage ring per warp in shared memory, requested
// two chunks before they are used; the column indices and the x gathers stay
// plain loads one and two chunks ahead, as above.  What this changes: the
// streamed values no longer pass through L1's miss handling, which on the
// Hamiltonian-like matrix limits the kernel (about one missed sector per cycle
// per SM, shared by the streamed operands and the gathers of far columns), and
// the values no longer occupy registers while they are in flight.  Every wait
// on a stage is bounded (mbar_wait_bounded); on a timeout the warp records
// kDevErrTimeout, waits (bounded) for its other stage and leaves.
template <int E, typename VT, typename XT, typename YT, typename ACC>
__global__ void __launch_bounds__(256, 2) k_slot_tv(const SlotParams p) {
    constexpr int SL = 32 * E;
    constexpr uint32_t kStageBytes = SL * sizeof(VT);
    static_assert(kStageBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
    static_assert(sizeof(ACC) == 8, "row buffer entries are 8 bytes");
    __shared__ ACC s_rows[8][kWarpRowCap];
    __shared__ __align__(128) VT s_vals[8][2][SL];
    __shared__ __align__(8) uint64_t s_bar[8][2];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * 8;
    const int n = p.n_chunks;
    int c = blockIdx.x * 8 + wib;
    if (lane == 0) {
        mbar_init(&s_bar[wib][0], 1);
        mbar_init(&s_bar[wib][1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (c >= n) return;
    ACC *srow = s_rows[wib];
    const uint64_t pol = l2_evict_first_policy();
    const VT *__restrict__ vals = static_cast<const VT *>(p.vals);
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);
    const XT *__restrict__ x = static_cast<const XT *>(p.m.x);
    YT *__restrict__ y = static_cast<YT *>(p.m.y);
    const MatRef m = p.m;

    auto regular = [](const ChunkDesc &d) { return (d.r1f & (kChunkLong | kChunkEmpty)) == 0; };
    auto hi_of = [&](const ChunkDesc &d) { return max(0, min(E, d.k1 - d.k0 - lane * E)); };
    auto load_cols = [&](int cc, int32_t (&cl)[E]) {
        const int32_t *b = p.cols + static_cast<int64_t>(cc) * SL + lane;
#pragma unroll
        for (int e = 0; e < E; ++e) cl[e] = ld_stream(b + e * 32, pol);
    };
    auto gather = [&](const ChunkDesc &d, const int32_t (&cl)[E], XT (&xv)[E]) {
        const int hi = regular(d) ? hi_of(d) : 0;
#pragma unroll
        for (int e = 0; e < E; ++e) xv[e] = (e < hi) ? __ldg(x + cl[e]) : XT(0);
    };
    auto load_desc = [&](int cc) {
        const int4 q = __ldg(reinterpret_cast<const int4 *>(p.chunks) + cc);
        return ChunkDesc{q.x, q.y, q.z, q.w};
    };
    // lane 0 requests the values of chunk cc into stage st (every lane has
    // finished reading that stage: the caller synchronises the warp first)
    auto request = [&](int cc, int st) {
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[wib][st], kStageBytes);
            bulk_g2s(&s_vals[wib][st][0], vals + static_cast<int64_t>(cc) * SL, kStageBytes, &s_bar[wib][st], pol);
        }
    };
    uint32_t phase = 0;  // bit st: parity of the next completion of stage st

    request(c, 0);
    if (c + nwarps < n) request(c + nwarps, 1);
    ChunkDesc dc = load_desc(c);
    uint32_t mc = __ldg(p.lmask + static_cast<int64_t>(c) * 32 + lane);
    XT xc[E];
    {
        int32_t cl[E];
        load_cols(c, cl);
        gather(dc, cl, xc);
    }
    ChunkDesc dn{};
    uint32_t mn = 0;
    int32_t cn[E];
#pragma unroll
    for (int e = 0; e < E; ++e) cn[e] = 0;
    if (c + nwarps < n) {
        dn = load_desc(c + nwarps);
        mn = __ldg(p.lmask + static_cast<int64_t>(c + nwarps) * 32 + lane);
        load_cols(c + nwarps, cn);
    }

    for (int it = 0; c < n; c += nwarps, ++it) {
        const int st = it & 1;
        const int c1 = c + nwarps, c2 = c + 2 * nwarps;
        // chunk c1: gathers; chunk c2: descriptor, row starts, columns
        XT xn[E];
        if (c1 < n) {
            gather(dn, cn, xn);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) xn[e] = XT(0);
        }
        ChunkDesc d2{};
        uint32_t m2 = 0;
        int32_t c2l[E];
        if (c2 < n) {
            d2 = load_desc(c2);
            m2 = __ldg(p.lmask + static_cast<int64_t>(c2) * 32 + lane);
            load_cols(c2, c2l);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) c2l[e] = 0;
        }
        // ---- chunk c: its values from stage st --------------------------------
        const bool ok = mbar_wait_bounded(&s_bar[wib][st], (phase >> st) & 1u);
        phase ^= 1u << st;
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) set_error(p.err, kDevErrTimeout);
            if (c1 < n) (void)mbar_wait_bounded(&s_bar[wib][st ^ 1], (phase >> (st ^ 1)) & 1u);
            return;
        }
        VT vc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) vc[e] = s_vals[wib][st][e * 32 + lane];
        __syncwarp();
        if (c2 < n) request(c2, st);
        const int r0 = dc.r0;
        const int r1 = dc.r1f & kChunkRowMask;
        if (dc.r1f & kChunkLong) {
            long_row<VT, XT, YT, ACC, false>(m, dc, x, y, alpha, beta, plain, lane);
        } else if (dc.r1f & kChunkEmpty) {
            rows_per_lane<VT, XT, YT, ACC, false>(m, r0, r1, x, y, alpha, beta, plain, lane);
        } else {
            const int hi = hi_of(dc);
            const uint32_t mbits = mc & ((1u << E) - 1u);
            chunk_lane_pre<E, VT, XT, ACC>(vc, xc, mbits, 0, hi, (mc & kSlotEnds) != 0u,
                                           static_cast<int>((mc >> kSlotPreShift) & kSlotPreMask), r0, srow, lane);
            __syncwarp();
            for (int q = lane; q < r1 - r0; q += 32)
                store_acc<VT, false>(m, x, y, r0 + q, srow[q], alpha, beta, plain);
        }
        __syncwarp();  // the row buffer is free again
        dc = dn;
        mc = mn;
        dn = d2;
        mn = m2;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            xc[e] = xn[e];
            cn[e] = c2l[e];
        }
    }
}

template <int E, typename VT, typename XT, typename YT, typename ACC>
struct SlotKernelTV {
    static int grid_limit() {
        static int cached = -1;
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_slot_tv<E, VT, XT, YT, ACC>, 256, 0) !=
            cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    static cudaError_t launch(const SlotParams &p, cudaStream_t s) {
        if (p.n_chunks <= 0) return cudaSuccess;
        const int lim = grid_limit();
        if (lim <= 0) return cudaErrorInvalidConfiguration;
        const int want = (p.n_chunks + 7) / 8;
        k_slot_tv<E, VT, XT, YT, ACC><<<want < lim ? want : lim, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
};

// Slot-major copies of a CRS: slot t = chunk*32E + e*32 + l holds entry
// k0 + l*E + e of the chunk when the chunk is regular and the entry belongs to
// it, else zero.  cols_out may be null (values only, after new values).
template <typename VT>
__global__ void __launch_bounds__(256) k_slot_relayout(const ChunkDesc *__restrict__ chunks, int E,
                                                       int64_t n_slots, const VT *__restrict__ val,
                                                       const int32_t *__restrict__ col, VT *__restrict__ vals_out,
                                                       int32_t *__restrict__ cols_out) {
    const int64_t SL = 32LL * E;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n_slots; t += stride) {
        const int64_t cc = t / SL;
        const int r = static_cast<int>(t - cc * SL);
        const int e = r >> 5, l = r & 31;
        const ChunkDesc d = chunks[cc];
        const int64_t k = static_cast<int64_t>(d.k0) + static_cast<int64_t>(l) * E + e;
        const bool ok = ((d.r1f & (kChunkLong | kChunkEmpty)) == 0) && k < d.k1;
        vals_out[t] = ok ? val[k] : VT(0);
        if (cols_out) cols_out[t] = ok ? col[k] : 0;
    }
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool PRE = false, bool BATCHED = false>
struct SlotKernel {
    static int grid_limit() {
        static int cached = -1;
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_slot<E, VT, XT, YT, ACC, PRE, BATCHED>, 256, 0) !=
            cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    static cudaError_t launch(const SlotParams &p, cudaStream_t s) {
        if (p.n_chunks <= 0) return cudaSuccess;
        const int lim = grid_limit();
        if (lim <= 0) return cudaErrorInvalidConfiguration;
        const int want = (p.n_chunks + 7) / 8;
        k_slot<E, VT, XT, YT, ACC, PRE, BATCHED><<<want < lim ? want : lim, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
};

}  // namespace spmv
