// The pipelined warp-chunk CRS kernel (single right-hand side).
//
// Same chunking, row bitmasks, per-lane FMA chains and lane-order carries as the
// warp-chunk kernel, but each warp is persistent and streams its chunks through a
// private two-stage shared-memory ring filled by cp.async.bulk (1-D TMA, 16-byte
// aligned, evict-first in L2): while a warp gathers x and runs the FMA chains of
// one chunk, the values, column indices and row bitmask of its next chunk are in
// flight.  Warps never wait for each other (no CTA barrier); each stage has its
// own mbarrier.  E is odd so lanes reading shared memory at stride E use
// distinct banks.
#pragma once
#include <type_traits>

#include "warp_kernel.cuh"

namespace spmv {

template <int E, typename VS>
struct PipeLayout {
    static constexpr int SLOTS = 32 * E;
    static constexpr int SL = SLOTS + 8;                 // alignment slack
    static constexpr int MWP = ((E + 3) / 4) * 4;        // mask words per chunk (16-byte rows)
    static constexpr size_t al(size_t v) { return (v + 15) & ~size_t(15); }
    static constexpr size_t off_vs = 0;
    static constexpr size_t off_col = off_vs + al(sizeof(VS) * SL);
    static constexpr size_t off_mask = off_col + al(4 * SL);
    static constexpr size_t off_desc = off_mask + al(4 * MWP);
    static constexpr size_t stage = off_desc + 16;
    static constexpr size_t off_rows = 2 * stage;
    static constexpr size_t off_bar = off_rows + 8 * kWarpRowCap;
    static constexpr size_t warp_bytes = al(off_bar + 16);
    static constexpr size_t block_bytes = 8 * warp_bytes;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
__global__ void __launch_bounds__(256) k_pipe(const WarpParams p) {
    static_assert(E % 2 == 1, "odd E: conflict-free strided shared-memory reads");
    using VS = typename std::conditional<INDIRECT, int32_t, VT>::type;
    using L = PipeLayout<E, VS>;
    extern __shared__ __align__(128) unsigned char smem[];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *ws = smem + wib * L::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ws + L::off_bar);
    ACC *srow = reinterpret_cast<ACC *>(ws + L::off_rows);
    const int nwarps = gridDim.x * 8;
    int c = blockIdx.x * 8 + wib;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (c >= p.n_chunks) return;

    uint64_t policy = 0;
    if (lane == 0) policy = l2_evict_first_policy();
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);

    auto is_regular = [](const ChunkDesc &d) { return (d.r1f & (kChunkLong | kChunkEmpty)) == 0; };
    // Lane 0: publish chunk cc's descriptor in stage s and start its copies.
    auto issue = [&](int cc, const ChunkDesc &d, int s) {
        unsigned char *st = ws + s * L::stage;
        *reinterpret_cast<ChunkDesc *>(st + L::off_desc) = d;
        if (is_regular(d)) {
            MatRef m;
            if constexpr (BATCHED) m = p.mats[p.cmat[cc]];
            else m = p.m;
            const int base = d.k0 & ~3;
            const int n = ((d.k1 - base) + 3) & ~3;
            const uint32_t bv = static_cast<uint32_t>(n * sizeof(VS));
            const uint32_t bc = static_cast<uint32_t>(n * 4);
            const uint32_t bm = static_cast<uint32_t>(L::MWP * 4);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[s], bv + bc + bm);
            bulk_g2s(st + L::off_vs, static_cast<const VS *>(m.vs) + base, bv, &bar[s], policy);
            bulk_g2s(st + L::off_col, m.col + base, bc, &bar[s], policy);
            bulk_g2s(st + L::off_mask, p.masks + static_cast<int64_t>(cc) * L::MWP, bm, &bar[s], policy);
        } else {
            mbar_arrive(&bar[s]);
        }
    };

    ChunkDesc dnext{};
    if (lane == 0) {
        const ChunkDesc d0 = p.chunks[c];
        issue(c, d0, 0);
        if (c + nwarps < p.n_chunks) dnext = p.chunks[c + nwarps];
    }
    uint32_t phase = 0;
    for (int i = 0; c < p.n_chunks; c += nwarps, ++i) {
        const int s = i & 1;
        const int cn = c + nwarps;
        if (lane == 0 && cn < p.n_chunks) {
            issue(cn, dnext, s ^ 1);
            if (cn + nwarps < p.n_chunks) dnext = p.chunks[cn + nwarps];
        }
        bool ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
        phase ^= 1u << s;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) {
                set_error(p.err, kDevErrTimeout);
                if (cn < p.n_chunks) (void)mbar_wait_bounded(&bar[s ^ 1], (phase >> (s ^ 1)) & 1u);
            }
            return;
        }
        unsigned char *st = ws + s * L::stage;
        const ChunkDesc d = *reinterpret_cast<const ChunkDesc *>(st + L::off_desc);
        MatRef m;
        if constexpr (BATCHED) m = p.mats[p.cmat[c]];
        else m = p.m;
        const XT *__restrict__ x = static_cast<const XT *>(m.x);
        YT *__restrict__ y = static_cast<YT *>(m.y);
        const int r0 = d.r0;
        const int r1 = d.r1f & kChunkRowMask;

        if (d.r1f & kChunkLong) {
            long_row<VT, XT, YT, ACC, INDIRECT>(m, d, x, y, alpha, beta, plain, lane);
        } else if (d.r1f & kChunkEmpty) {
            rows_per_lane<VT, XT, YT, ACC, INDIRECT>(m, r0, r1, x, y, alpha, beta, plain, lane);
        } else {
            const VS *sv = reinterpret_cast<const VS *>(st + L::off_vs);
            const int32_t *sc = reinterpret_cast<const int32_t *>(st + L::off_col);
            const uint32_t *smk = reinterpret_cast<const uint32_t *>(st + L::off_mask);
            const int base = d.k0 & ~3;
            const int off = lane * E;              // first slot of the lane
            const int lo = max(0, d.k0 - base - off);
            const int hi = min(E, d.k1 - base - off);
            const int w0 = off >> 5, sh = off & 31;
            const uint64_t win = (static_cast<uint64_t>(smk[w0 + 1]) << 32) | smk[w0];
            const uint32_t mbits = static_cast<uint32_t>(win >> sh) & ((1u << E) - 1u);
            XT xv[E];
            VT vals[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                xv[e] = XT(0);
                if (e >= lo && e < hi) xv[e] = __ldg(x + sc[off + e]);
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                vals[e] = VT(0);
                if (e >= lo && e < hi) {
                    if constexpr (INDIRECT) vals[e] = __ldg(static_cast<const VT *>(m.vind) + sv[off + e]);
                    else vals[e] = sv[off + e];
                }
            }
            const uint32_t next_bits = __shfl_down_sync(0xffffffffu, mbits, 1);
            const bool ends = (base + off + E >= d.k1) || (lane < 31 && (next_bits & 1u));
            chunk_lane<E, VT, XT, ACC>(vals, xv, mbits, lo, hi, ends, r0, srow, lane);
            __syncwarp();
            for (int q = lane; q < r1 - r0; q += 32)
                store_acc<VT, INDIRECT>(m, x, y, r0 + q, srow[q], alpha, beta, plain);
        }
        // every lane is done with stage s (and the row buffer) before lane 0
        // refills it at the next iteration
        __syncwarp();
    }
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
struct PipeKernel {
    using VS = typename std::conditional<INDIRECT, int32_t, VT>::type;
    using L = PipeLayout<E, VS>;
    static constexpr auto fn = k_pipe<E, VT, XT, YT, ACC, INDIRECT, BATCHED>;
    static int grid_limit() {
        static int cached = -1;
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(L::block_bytes)) != cudaSuccess)
            return 0;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, L::block_bytes) != cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    static cudaError_t launch(const WarpParams &p, int n_chunks, cudaStream_t s) {
        if (n_chunks <= 0) return cudaSuccess;
        const int lim = grid_limit();
        if (lim <= 0) return cudaErrorInvalidConfiguration;
        const int want = (n_chunks + 7) / 8;
        fn<<<want < lim ? want : lim, 256, L::block_bytes, s>>>(p);
        return cudaGetLastError();
    }
};

}  // namespace spmv

namespace spmv {

// Three-stage variant: the x gathers of chunk i+1 are issued before the FMA
// chains of chunk i, so one warp keeps its next chunk's L2 gathers in flight
// while its FP64 chain runs; chunk i+2 is being copied meanwhile.
template <int E, typename VS, int WPB>
struct Pipe3Layout {
    static constexpr int SLOTS = 32 * E;
    static constexpr int SL = SLOTS + 4;
    static constexpr int MWP = ((E + 3) / 4) * 4;
    static constexpr size_t al(size_t v) { return (v + 15) & ~size_t(15); }
    static constexpr size_t off_vs = 0;
    static constexpr size_t off_col = off_vs + al(sizeof(VS) * SL);
    static constexpr size_t off_mask = off_col + al(4 * SL);
    static constexpr size_t off_desc = off_mask + al(4 * MWP);
    static constexpr size_t stage = off_desc + 16;
    static constexpr size_t off_rows = 3 * stage;
    static constexpr size_t off_bar = off_rows + 8 * kWarpRowCap;
    static constexpr size_t warp_bytes = al(off_bar + 24);
    static constexpr size_t block_bytes = WPB * warp_bytes;
    // resident blocks per SM that shared memory allows (227 KB usable)
    static constexpr int min_blocks = (232448 / (block_bytes + 1024)) < 1 ? 1
                                      : ((232448 / (block_bytes + 1024)) > 4 ? 4 : (232448 / (block_bytes + 1024)));
};

// warps per block of the three-stage kernel (fewer resident warps leave more of
// the SM's 256 KB to L1, which holds the x lines near columns reuse)
template <int E> struct Pipe3Warps { static constexpr int value = 8; };

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
__global__ void __launch_bounds__(32 * Pipe3Warps<E>::value, Pipe3Layout<E, VT, Pipe3Warps<E>::value>::min_blocks)
k_pipe3(const WarpParams p) {
    static_assert(E % 2 == 1, "odd E: conflict-free strided shared-memory reads");
    static_assert(!INDIRECT, "values read from the staged copy");
    using VS = VT;
    constexpr int WPB = Pipe3Warps<E>::value;
    using L = Pipe3Layout<E, VS, WPB>;
    extern __shared__ __align__(128) unsigned char smem[];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *ws = smem + wib * L::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ws + L::off_bar);
    ACC *srow = reinterpret_cast<ACC *>(ws + L::off_rows);
    const int nwarps = gridDim.x * WPB;
    const int c0 = blockIdx.x * WPB + wib;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (c0 >= p.n_chunks) return;

    uint64_t policy = 0;
    if (lane == 0) policy = l2_evict_first_policy();
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);
    auto is_regular = [](const ChunkDesc &d) { return (d.r1f & (kChunkLong | kChunkEmpty)) == 0; };
    auto mat_of = [&](int cc) -> MatRef {
        if constexpr (BATCHED) return p.mats[p.cmat[cc]];
        else return p.m;
    };
    auto issue = [&](int cc, const ChunkDesc &d, int s) {
        unsigned char *st = ws + s * L::stage;
        *reinterpret_cast<ChunkDesc *>(st + L::off_desc) = d;
        if (is_regular(d)) {
            const MatRef m = mat_of(cc);
            const int base = d.k0 & ~3;
            const int n = ((d.k1 - base) + 3) & ~3;
            const uint32_t bv = static_cast<uint32_t>(n * sizeof(VS));
            const uint32_t bc = static_cast<uint32_t>(n * 4);
            const uint32_t bm = static_cast<uint32_t>(L::MWP * 4);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[s], bv + bc + bm);
            bulk_g2s(st + L::off_vs, static_cast<const VS *>(m.vs) + base, bv, &bar[s], policy);
            bulk_g2s(st + L::off_col, m.col + base, bc, &bar[s], policy);
            bulk_g2s(st + L::off_mask, p.masks + static_cast<int64_t>(cc) * L::MWP, bm, &bar[s], policy);
        } else {
            mbar_arrive(&bar[s]);
        }
    };
    uint32_t phase = 0;  // bit s: parity of the next completion of stage s
    auto wait_stage = [&](int s) -> bool {
        bool ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
        phase ^= 1u << s;
        return __all_sync(0xffffffffu, ok);
    };
    // gathers of the chunk staged in s (regular chunks only)
    auto gather = [&](int cc, int s, XT (&xv)[E]) {
        const unsigned char *st = ws + s * L::stage;
        const ChunkDesc d = *reinterpret_cast<const ChunkDesc *>(st + L::off_desc);
#pragma unroll
        for (int e = 0; e < E; ++e) xv[e] = XT(0);
        if (!is_regular(d)) return;
        const MatRef m = mat_of(cc);
        const XT *__restrict__ x = static_cast<const XT *>(m.x);
        const int32_t *sc = reinterpret_cast<const int32_t *>(st + L::off_col);
        const int base = d.k0 & ~3;
        const int off = lane * E;
        const int lo = max(0, d.k0 - base - off);
        const int hi = min(E, d.k1 - base - off);
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (e >= lo && e < hi) xv[e] = __ldg(x + sc[off + e]);
    };

    // prologue: chunks c0 and c0+nwarps in flight, gathers of c0 issued
    ChunkDesc dnext{};
    if (lane == 0) {
        issue(c0, p.chunks[c0], 0);
        if (c0 + nwarps < p.n_chunks) {
            issue(c0 + nwarps, p.chunks[c0 + nwarps], 1);
            if (c0 + 2 * nwarps < p.n_chunks) dnext = p.chunks[c0 + 2 * nwarps];
        }
    }
    XT xcur[E];
    if (!wait_stage(0)) {
        if (lane == 0) set_error(p.err, kDevErrTimeout);
        return;
    }
    gather(c0, 0, xcur);

    int s = 0;
    for (int c = c0; c < p.n_chunks; c += nwarps) {
        const int c1 = c + nwarps, c2 = c + 2 * nwarps;
        const int s1 = (s + 1) % 3, s2 = (s + 2) % 3;
        if (lane == 0 && c2 < p.n_chunks) {
            issue(c2, dnext, s2);
            if (c2 + nwarps < p.n_chunks) dnext = p.chunks[c2 + nwarps];
        }
        XT xnext[E];
#pragma unroll
        for (int e = 0; e < E; ++e) xnext[e] = XT(0);
        if (c1 < p.n_chunks) {
            if (!wait_stage(s1)) {
                if (lane == 0) set_error(p.err, kDevErrTimeout);
                return;
            }
            gather(c1, s1, xnext);
        }
        // ---- chunk c (staged in s, gathers in xcur) --------------------------
        const unsigned char *st = ws + s * L::stage;
        const ChunkDesc d = *reinterpret_cast<const ChunkDesc *>(st + L::off_desc);
        const MatRef m = mat_of(c);
        const XT *__restrict__ x = static_cast<const XT *>(m.x);
        YT *__restrict__ y = static_cast<YT *>(m.y);
        const int r0 = d.r0;
        const int r1 = d.r1f & kChunkRowMask;
        if (d.r1f & kChunkLong) {
            long_row<VT, XT, YT, ACC, false>(m, d, x, y, alpha, beta, plain, lane);
        } else if (d.r1f & kChunkEmpty) {
            rows_per_lane<VT, XT, YT, ACC, false>(m, r0, r1, x, y, alpha, beta, plain, lane);
        } else {
            const VS *sv = reinterpret_cast<const VS *>(st + L::off_vs);
            const uint32_t *smk = reinterpret_cast<const uint32_t *>(st + L::off_mask);
            const int base = d.k0 & ~3;
            const int off = lane * E;
            const int lo = max(0, d.k0 - base - off);
            const int hi = min(E, d.k1 - base - off);
            const int w0 = off >> 5, sh = off & 31;
            const uint64_t win = (static_cast<uint64_t>(smk[w0 + 1]) << 32) | smk[w0];
            const uint32_t mbits = static_cast<uint32_t>(win >> sh) & ((1u << E) - 1u);
            VT vals[E];
#pragma unroll
            for (int e = 0; e < E; ++e) vals[e] = (e >= lo && e < hi) ? sv[off + e] : VT(0);
            const uint32_t next_bits = __shfl_down_sync(0xffffffffu, mbits, 1);
            const bool ends = (base + off + E >= d.k1) || (lane < 31 && (next_bits & 1u));
            chunk_lane<E, VT, XT, ACC>(vals, xcur, mbits, lo, hi, ends, r0, srow, lane);
            __syncwarp();
            for (int q = lane; q < r1 - r0; q += 32) store_acc<VT, INDIRECT>(m, x, y, r0 + q, srow[q], alpha, beta, plain);
        }
        __syncwarp();  // stage s and the row buffer are free again
#pragma unroll
        for (int e = 0; e < E; ++e) xcur[e] = xnext[e];
        s = s1;
    }
}

template <int E, typename VT, typename XT, typename YT, typename ACC, bool INDIRECT, bool BATCHED>
struct Pipe3Kernel {
    static constexpr int WPB = Pipe3Warps<E>::value;
    using L = Pipe3Layout<E, VT, WPB>;
    static constexpr auto fn = k_pipe3<E, VT, XT, YT, ACC, INDIRECT, BATCHED>;
    static int grid_limit() {
        static int cached = -1;
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(L::block_bytes)) != cudaSuccess)
            return 0;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * WPB, L::block_bytes) != cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    static cudaError_t launch(const WarpParams &p, int n_chunks, cudaStream_t s) {
        if (n_chunks <= 0) return cudaSuccess;
        const int lim = grid_limit();
        if (lim <= 0) return cudaErrorInvalidConfiguration;
        const int want = (n_chunks + WPB - 1) / WPB;
        fn<<<want < lim ? want : lim, 32 * WPB, L::block_bytes, s>>>(p);
        return cudaGetLastError();
    }
};

}  // namespace spmv
