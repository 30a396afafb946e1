// The nnz-split CRS tile kernel.
//
// Listing 1 (Sect. 1.2) sums val(j)*B(col_idx(j)) over the entries of each row.
// GB300 executes FP64 FMAs at about 1/57 of the FP32 rate, so an FP64 spMVM is
// bounded by the FP64 pipe almost as tightly as by HBM: the kernel is built so
// every warp-wide FMA does useful work on all 32 lanes and no other FP64
// instruction is issued per entry.
//
//   * The matrix is cut into tiles of whole rows with at most CAP entries (built
//     once on the host from row_ptr).  A persistent CTA walks its tiles; one
//     thread streams each tile's col_idx, values and row_ptr slice into shared
//     memory with cp.async.bulk (16-byte aligned 1-D TMA copies, evict-first in
//     L2 so x stays resident), double-buffered on two mbarriers.
//   * Inside a tile, group g of R lanes (R = 1 for one vector, R right-hand sides
//     for block vectors) owns the E consecutive entries [g*E, g*E+E): it gathers
//     its E x values first (E loads in flight per lane), then runs one FMA chain,
//     restarting at each row start.  Rows that start and end inside a segment are
//     final; a row cut by segment ends leaves a "carry" (the part before the cut)
//     and a "pending" part, combined after a barrier in segment order, so the
//     result is deterministic.  E is odd, so lanes reading shared memory at stride
//     E hit distinct banks.
//   * Row results collect in shared memory and are written to y row-contiguous
//     with the alpha/beta update, one store per row and right-hand side.
//   * A row longer than a tile forms its own tile, reduced by the whole CTA from
//     global memory in fixed order.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace spmv {

__host__ __device__ constexpr int rowcap_for(int cap) {
    return ((cap / 4 + 31) / 32) * 32 < 32 ? 32 : ((cap / 4 + 31) / 32) * 32;
}

template <int NT, int R, int E, int STAGES, typename VS, typename ACC>
struct TileLayout {
    static constexpr int G = NT / R;
    static constexpr int CAP = G * E;
    static constexpr int ROWCAP = rowcap_for(CAP);
    static constexpr int NPAD = CAP + 8;
    static constexpr int RPAD = ROWCAP + 8;
    static constexpr size_t al(size_t v) { return (v + 127) & ~size_t(127); }
    static constexpr size_t sz_vs = al(sizeof(VS) * NPAD);
    static constexpr size_t sz_col = al(4 * NPAD);
    static constexpr size_t sz_rp = al(4 * RPAD);
    static constexpr size_t off_vs = 0;
    static constexpr size_t off_col = off_vs + STAGES * sz_vs;
    static constexpr size_t off_rp = off_col + STAGES * sz_col;
    static constexpr size_t off_y = off_rp + STAGES * sz_rp;
    static constexpr size_t off_carry = off_y + al(sizeof(double) * ROWCAP * R);
    static constexpr size_t off_crow = off_carry + al(sizeof(ACC) * G * R);
    static constexpr size_t off_bar = off_crow + al(sizeof(int32_t) * G);
    static constexpr size_t bytes = off_bar + 128;
};

template <typename T> __device__ __forceinline__ T ld_nc(const T *p) { return __ldg(p); }

template <int NT, int R, int E, int STAGES, typename VT, typename XT, typename YT, typename ACC,
          bool INDIRECT, bool BATCHED>
__global__ void __launch_bounds__(NT) k_tile(const KParams p) {
    static_assert(E % 2 == 1, "E must be odd (bank-conflict-free strided reads)");
    static_assert(NT % R == 0 && (R & (R - 1)) == 0, "R must be a power of two dividing NT");
    static_assert(STAGES == 2, "two-stage ring");
    using VS = typename std::conditional<INDIRECT, int32_t, VT>::type;
    using L = TileLayout<NT, R, E, STAGES, VS, ACC>;
    constexpr int G = L::G;
    constexpr int CAP = L::CAP;

    extern __shared__ __align__(128) unsigned char smem[];
    VS *s_vs = reinterpret_cast<VS *>(smem + L::off_vs);
    int32_t *s_col = reinterpret_cast<int32_t *>(smem + L::off_col);
    int32_t *s_rp = reinterpret_cast<int32_t *>(smem + L::off_rp);
    double *s_y = reinterpret_cast<double *>(smem + L::off_y);
    ACC *s_carry = reinterpret_cast<ACC *>(smem + L::off_carry);
    int32_t *s_crow = reinterpret_cast<int32_t *>(smem + L::off_crow);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + L::off_bar);
    volatile int32_t *s_abort = reinterpret_cast<volatile int32_t *>(smem + L::off_bar + 64);
    constexpr int VS_STRIDE = static_cast<int>(L::sz_vs / sizeof(VS));
    constexpr int COL_STRIDE = static_cast<int>(L::sz_col / sizeof(int32_t));
    constexpr int RP_STRIDE = static_cast<int>(L::sz_rp / sizeof(int32_t));

    const int tid = threadIdx.x;
    const int g = tid / R;
    const int r = tid % R;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&s_bar[s], 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    for (int i = tid; i < L::ROWCAP * R; i += NT) s_y[i] = 0.0;
    __syncthreads();

    int t = blockIdx.x;
    if (t >= p.n_tiles) return;

    const TileDesc *tiles = p.tiles;
    const int stride = gridDim.x;
    uint64_t policy = 0;
    if (tid == 0) policy = l2_evict_first_policy();

    auto is_long = [](const TileDesc &d) { return d.k1 - d.k0 > CAP; };
    auto mat_of = [&](const TileDesc &d) -> MatRef {
        if constexpr (BATCHED) return p.mats[d.mat];
        else return p.m;
    };
    // Producer: stage the entries, the values (or permutation) and the row_ptr
    // slice of tile d into stage s.  Ranges are widened to 16-byte boundaries.
    auto issue = [&](const TileDesc &d, int s) {
        const MatRef m = mat_of(d);
        const int k0a = d.k0 & ~3;
        int k1a = (d.k1 + 3) & ~3;
        if (k1a < k0a + 4) k1a = k0a + 4;
        const int r0a = d.r0 & ~3;
        const int r1a = (d.r1 + 1 + 3) & ~3;
        const uint32_t bv = static_cast<uint32_t>((k1a - k0a) * sizeof(VS));
        const uint32_t bc = static_cast<uint32_t>((k1a - k0a) * 4);
        const uint32_t br = static_cast<uint32_t>((r1a - r0a) * 4);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[s], bv + bc + br);
        bulk_g2s(s_vs + s * VS_STRIDE, static_cast<const VS *>(m.vs) + k0a, bv, &s_bar[s], policy);
        bulk_g2s(s_col + s * COL_STRIDE, m.col + k0a, bc, &s_bar[s], policy);
        bulk_g2s(s_rp + s * RP_STRIDE, m.rp + r0a, br, &s_bar[s], policy);
    };

    TileDesc d = tiles[t];
    TileDesc dn;
    dn.r0 = dn.r1 = dn.k0 = dn.k1 = 0;
    dn.mat = 0;
    if (t + stride < p.n_tiles) dn = tiles[t + stride];
    if (tid == 0 && !is_long(d)) issue(d, 0);

    uint32_t phase = 0;  // bit s: parity of the next completion of stage s
    const double alpha = p.alpha, beta = p.beta;
    const bool plain_store = (alpha == 1.0 && beta == 0.0);

    for (int i = 0; t < p.n_tiles; t += stride, ++i) {
        const int s = i & 1;
        const int tn = t + stride;
        TileDesc dnn;
        dnn.r0 = dnn.r1 = dnn.k0 = dnn.k1 = 0;
        dnn.mat = 0;
        if (tn + stride < p.n_tiles) dnn = tiles[tn + stride];
        // The other stage was last read before the previous tile's final barrier.
        if (tid == 0 && tn < p.n_tiles && !is_long(dn)) issue(dn, s ^ 1);

        const MatRef m = mat_of(d);
        const XT *__restrict__ x = static_cast<const XT *>(m.x);
        YT *__restrict__ y = static_cast<YT *>(m.y);
        const int r0 = d.r0, r1 = d.r1, k0 = d.k0;
        const int nt = d.k1 - d.k0;

        if (!is_long(d)) {
            const bool ok = mbar_wait_bounded(&s_bar[s], (phase >> s) & 1u);
            phase ^= (1u << s);
            if (!ok) {
                *s_abort = 1;
                set_error(p.err, kDevErrTimeout);
            }
            __syncthreads();
            if (*s_abort) {
                // Drain the copy issued for the next tile, then leave.
                if (tid == 0 && tn < p.n_tiles && !is_long(dn))
                    (void)mbar_wait_bounded(&s_bar[s ^ 1], (phase >> (s ^ 1)) & 1u);
                return;
            }

            const VS *sv = s_vs + s * VS_STRIDE + (k0 - (k0 & ~3));
            const int32_t *sc = s_col + s * COL_STRIDE + (k0 - (k0 & ~3));
            const int32_t *srp = s_rp + s * RP_STRIDE - (r0 & ~3);  // srp[row] = row_ptr[row]

            // ---- phase A: one FMA chain per segment --------------------------
            const int jb = g * E;
            bool has_pend = false;
            int pend_row = 0;
            ACC pend;
            pend.zero();
            if (jb < nt) {
                const int je = min(jb + E, nt);
                const int kk = k0 + jb;
                int lo = r0, hi = r1 - 1;  // largest row with row_ptr[row] <= kk
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (srp[mid] <= kk) lo = mid;
                    else hi = mid - 1;
                }
                int row = lo;
                int next = srp[row + 1];
                bool started = (srp[row] == kk);

                XT xv[E];
                const bool lane_ok = (r < p.rhs_count);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    xv[e] = XT(0);
                    if (jb + e < je && lane_ok)
                        xv[e] = ld_nc(x + static_cast<int64_t>(sc[jb + e]) * p.ldx + r);
                }
                ACC acc;
                acc.zero();
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (jb + e < je) {
                        const int k = kk + e;
                        if (k == next) {
                            if (started) s_y[(row - r0) * R + r] = acc.get();
                            else { has_pend = true; pend_row = row; pend = acc; }
                            acc.zero();
                            do { ++row; next = srp[row + 1]; } while (next == k);
                            started = true;
                        }
                        if constexpr (INDIRECT)
                            acc.fma(ld_nc(static_cast<const VT *>(m.vind) + sv[jb + e]), xv[e]);
                        else
                            acc.fma(sv[jb + e], xv[e]);
                    }
                }
                if (next == k0 + je) {  // the last row ends with the segment
                    if (started) s_y[(row - r0) * R + r] = acc.get();
                    else { has_pend = true; pend_row = row; pend = acc; }
                    if (r == 0) s_crow[g] = -1;
                } else {
                    s_carry[g * R + r] = acc;
                    if (r == 0) s_crow[g] = row;
                }
            } else if (r == 0) {
                s_crow[g] = -1;
            }
            __syncthreads();

            // ---- phase B: rows cut by segment ends, combined in segment order --
            if (has_pend) {
                int q = g - 1;
                while (q >= 0 && s_crow[q] == pend_row) --q;
                ACC tot = s_carry[(q + 1) * R + r];
                for (int u = q + 2; u < g; ++u) tot.add(s_carry[u * R + r]);
                tot.add(pend);
                s_y[(pend_row - r0) * R + r] = tot.get();
            }
            __syncthreads();

            // ---- phase C: y = alpha*(A x) + beta*y, row-contiguous -------------
            const int nrows = r1 - r0;
            for (int idx = tid; idx < nrows * R; idx += NT) {
                const int i_r = idx / R;
                const int rr = idx % R;
                double v = s_y[idx];
                s_y[idx] = 0.0;
                if constexpr (std::is_same<ACC, AccFF>::value) {
                    // a poisoned float-float sum arrives as NaN: sum the row again in FP64
                    if (v != v && rr < p.rhs_count) v = row_sum_exact<VT, INDIRECT>(m, r0 + i_r, x + rr, p.ldx);
                }
                if (rr < p.rhs_count) {
                    YT *yp = y + static_cast<int64_t>(r0 + i_r) * p.ldy + rr;
                    double out;
                    if (plain_store) out = v;
                    else if (beta == 0.0) out = alpha * v;
                    else out = fma(alpha, v, beta * widen(*yp));
                    *yp = narrow<YT>(out);
                }
            }
            // The next iteration's first barrier (after its wait) orders these
            // shared-memory writes before the next tile's phase A.
        } else {
            // ---- long row: the whole CTA reduces row r0 from global memory -----
            ACC acc;
            acc.zero();
            const bool lane_ok = (r < p.rhs_count);
            if (lane_ok) {
                for (int k = d.k0 + g; k < d.k1; k += G) {
                    const int c = ld_nc(m.col + k);
                    const XT xv = ld_nc(x + static_cast<int64_t>(c) * p.ldx + r);
                    if constexpr (INDIRECT)
                        acc.fma(ld_nc(static_cast<const VT *>(m.vind) + ld_nc(static_cast<const int32_t *>(m.vs) + k)), xv);
                    else
                        acc.fma(ld_nc(static_cast<const VT *>(m.vs) + k), xv);
                }
            }
            __syncthreads();  // s_carry may still be read by the previous tile's phase B
            s_carry[g * R + r] = acc;
            __syncthreads();
            if (g == 0 && lane_ok) {
                ACC tot = s_carry[r];
                for (int u = 1; u < G; ++u) tot.add(s_carry[u * R + r]);
                double v = tot.get();
                if constexpr (std::is_same<ACC, AccFF>::value) {
                    if (tot.poisoned()) v = row_sum_exact<VT, INDIRECT>(m, r0, x + r, p.ldx);
                }
                YT *yp = y + static_cast<int64_t>(r0) * p.ldy + r;
                double out;
                if (plain_store) out = v;
                else if (beta == 0.0) out = alpha * v;
                else out = fma(alpha, v, beta * widen(*yp));
                *yp = narrow<YT>(out);
            }
            __syncthreads();
        }
        d = dn;
        dn = dnn;
    }
}

template <int NT, int R, int E, int STAGES, typename VT, typename XT, typename YT, typename ACC,
          bool INDIRECT, bool BATCHED>
struct TileKernel {
    using VS = typename std::conditional<INDIRECT, int32_t, VT>::type;
    using L = TileLayout<NT, R, E, STAGES, VS, ACC>;
    static constexpr auto fn = k_tile<NT, R, E, STAGES, VT, XT, YT, ACC, INDIRECT, BATCHED>;

    static cudaError_t prepare() {
        static bool done = false;  // attribute set once per process and device set
        static int dev = -1;
        int cur = 0;
        cudaGetDevice(&cur);
        if (done && dev == cur) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(L::bytes));
        if (e == cudaSuccess) { done = true; dev = cur; }
        return e;
    }
    static int grid_limit() {
        static int cached = -1;  // resident CTAs on the whole GPU, computed once
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        if (prepare() != cudaSuccess) return 0;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, L::bytes) != cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    static cudaError_t launch(const KParams &p, int grid, cudaStream_t s) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if (grid <= 0) return cudaSuccess;
        fn<<<grid, NT, L::bytes, s>>>(p);
        return cudaGetLastError();
    }
    static TileCfg cfg() { return TileCfg{E, NT, L::ROWCAP, L::CAP}; }
};

}  // namespace spmv
