// Sorted row-slice kernel (plan family 5).
//
// The rows of each window of `sigma` consecutive rows are ordered by length
// (longest first) and cut into slices of kSellC = 64 rows; lane l of a warp owns
// rows l and l + 32 of a slice from their first entries to their last, so a row
// sum is one FMA chain in one lane: no row-start bits, no carries between lanes
// and no row buffer, and each lane runs two independent chains (one chain per
// lane leaves the FP64 pipe waiting on its own results).  Entry j of the slice's
// row h*32 + l is stored at slot (off + j)*64 + h*32 + l (the slice's width w is
// its longest row; shorter rows are padded with value 0 and column -1), so every
// load of a warp reads 32 consecutive elements.  Sorting inside windows keeps
// the padding small (equal-length rows share slices) while the rows of a slice
// stay close together in x and y.  This is the SELL-C-sigma layout of Kreutzer,
// Hager, Wellein, Fehske and Bishop (SIAM J. Sci. Comput. 36(5), 2014) with
// C = 64, built as a derived copy of the CRS arrays.
//
// CTA b owns the slices [cstart[b], cstart[b+1]), a contiguous range chosen on
// the host so that every CTA gets the same number of slots (a fixed
// round-robin over windows sorted by length would hand some warps the widest
// slices of every window); its 8 warps take the range's slices in turn, so the
// CTA works on one or two windows at a time and their x entries stay in L1.  A
// warp walks its slices in blocks of kSellU slot rows.  The values and gathers
// of the next block and the column indices of the block after it are in flight
// in registers while the current block's FMAs run (two register sets in turn).
// A block shorter than kSellU holds its entries at the end of the register
// arrays (the loads before it read the preceding slot rows, which exist because
// the arrays start with kSellU rows of padding, and their columns are masked)
// and enters the FMA sequence part-way, so every FMA issued belongs to a stored
// slot.
#pragma once
#include "slot_kernel.cuh"
#include "reduce.cuh"

namespace spmv {

constexpr int kSellK = 2;            // rows per lane
constexpr int kSellC = 32 * kSellK;  // rows per slice
constexpr int kSellU = 4;            // slot rows per block

struct SellParams {
    const int2 *slices;    // per slice: x = first slot row (>= kSellU), y = width w; y < 0: long row x (CRS)
    const int32_t *srows;  // kSellC per slice: the row of each lane and half (-1: none)
    const int32_t *cstart; // n_ctas + 1: the first slice of each CTA
    const void *vals;      // slot-major values (0 in padding)
    const int32_t *cols;   // slot-major column indices (-1 in padding)
    MatRef m;              // the CRS itself (long rows), x, y
    int32_t n_slices;
    int32_t n_ctas;        // CTAs of the launch
    double alpha, beta;
};

// For i = 0 .. cnt-1 and both rows h of the lane, in that order:
// acc[h] += v[U-cnt+i][h] * xv[U-cnt+i][h].  A jump into an unrolled sequence
// (cnt is the same in all lanes), so no FMA is issued for an empty register.
template <typename ACC, typename VT, typename XT>
__device__ __forceinline__ void sell_fma_tail(ACC (&acc)[kSellK], const VT (&v)[kSellU][kSellK],
                                              const XT (&xv)[kSellU][kSellK], int cnt) {
    static_assert(kSellU == 4 && kSellK == 2, "the jump table below is written for 4 slot rows of 2 rows");
    switch (cnt) {
        case 4:
            acc[0].fma(v[0][0], xv[0][0]);
            acc[1].fma(v[0][1], xv[0][1]);
            [[fallthrough]];
        case 3:
            acc[0].fma(v[1][0], xv[1][0]);
            acc[1].fma(v[1][1], xv[1][1]);
            [[fallthrough]];
        case 2:
            acc[0].fma(v[2][0], xv[2][0]);
            acc[1].fma(v[2][1], xv[2][1]);
            [[fallthrough]];
        case 1:
            acc[0].fma(v[3][0], xv[3][0]);
            acc[1].fma(v[3][1], xv[3][1]);
            [[fallthrough]];
        default:
            break;
    }
}

// Final store of stored row `row` of m; `old` is y[row] widened, loaded ahead
// (read only when beta is nonzero).  A poisoned float-float sum is summed again
// in FP64 from the CRS arrays of m.
template <typename VT, typename XT, typename YT, typename ACC>
__device__ __forceinline__ YT sell_store(const MatRef &m, const XT *__restrict__ x, YT *__restrict__ y, int row,
                                         const ACC &a, double alpha, double beta, bool plain, double old) {
    if constexpr ((std::is_same<ACC, AccFF>::value || std::is_same<ACC, AccFR>::value ||
                   std::is_same<ACC, AccFRF>::value) &&
                  std::is_same<YT, float>::value) {
        if (plain && !a.poisoned()) {
            const float out = a.h + a.l;
            y[row] = out;
            return out;
        }
    }
    const double v = acc_value<VT, false>(a, m, row, x);
    double out;
    if (plain) out = v;
    else if (beta == 0.0) out = alpha * v;
    else out = fma(alpha, v, beta * old);
    const YT yo = narrow<YT>(out);
    y[row] = yo;
    return yo;
}

// Gather of x through L1, issued where it stands in the source (the compiler may
// not move it next to its use, which would leave no time for its latency).
__device__ __forceinline__ double ld_gather(const double *p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_gather(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// The walk of one warp over its CTA's slices.  DOT: also dsum += x[r] * y[r]
// (exact products of the stored values, FP64 sums) for every row r the warp
// stores (the p.q of a CG step, with x = p and y = q).
template <typename VT, typename XT, typename YT, typename ACC, bool DOT>
__device__ __forceinline__ void sell_walk(const SellParams &p, double &dsum) {
    constexpr int U = kSellU, K = kSellK, C = kSellC;
    const int lane = threadIdx.x & 31;
    if (static_cast<int>(blockIdx.x) >= p.n_ctas) return;
    const int s0 = __ldg(p.cstart + blockIdx.x) + (threadIdx.x >> 5);
    const int n = __ldg(p.cstart + blockIdx.x + 1);  // end of this CTA's slices
    if (s0 >= n) return;
    const uint64_t pol = l2_evict_first_policy();
    const VT *__restrict__ vals = static_cast<const VT *>(p.vals);
    const int32_t *__restrict__ cols = p.cols;
    const XT *__restrict__ x = static_cast<const XT *>(p.m.x);
    YT *__restrict__ y = static_cast<YT *>(p.m.y);
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);
    const bool read_y = !plain && beta != 0.0;

    // block cursor: slice s (descriptor off, w) and the block's first slot row j0
    struct Cur {
        int s, off, w, j0;
    };
    auto slice_of = [&](int s) { return s < n ? __ldg(p.slices + s) : make_int2(0, 0); };
    auto cnt_of = [](const Cur &c) { return max(0, min(U, c.w - c.j0)); };
    auto last_of = [](const Cur &c) { return c.j0 + U >= c.w; };
    // next block of the warp; dnext is the descriptor of slice c.s + 8
    auto advance = [&](Cur &c, int2 &dnext) {
        if (!last_of(c)) {
            c.j0 += U;
            return;
        }
        c.s += 8;
        c.off = dnext.x;
        c.w = dnext.y;
        c.j0 = 0;
        dnext = slice_of(c.s + 8);
    };
    // Element of register row 0 of the block (a block of cnt slot rows starts at
    // register row U - cnt; the slot rows before it exist, see above).  Blocks
    // without slots (long rows, past the end) read the leading padding rows.
    // The loads are unconditional and nothing inspects their results until the
    // block is used (a select on a fresh column index would wait for it).
    auto base_of = [&](const Cur &c) {
        const int cnt = c.s < n ? cnt_of(c) : 0;
        return cnt > 0 ? (static_cast<int64_t>(c.off) + c.j0 - (U - cnt)) * C + lane : static_cast<int64_t>(lane);
    };
    auto load_cols = [&](const Cur &c, int32_t (&cl)[U][K]) {
        const int32_t *b = cols + base_of(c);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < K; ++h) cl[u][h] = ld_stream(b + u * C + h * 32, pol);
    };
    auto load_vals = [&](const Cur &c, VT (&v)[U][K]) {
        const VT *b = vals + base_of(c);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < K; ++h) v[u][h] = ld_stream(b + u * C + h * 32, pol);
    };
    // gathers of the block's slots (register rows U - cnt .. U - 1, stored columns)
    auto gather = [&](const Cur &c, const int32_t (&cl)[U][K], XT (&xv)[U][K]) {
        const int cnt = c.s < n ? cnt_of(c) : 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < K; ++h)
                xv[u][h] = (u >= U - cnt && cl[u][h] >= 0) ? ld_gather(x + cl[u][h]) : XT(0);
    };
    // the output rows of the lane, for the last block of a regular slice
    auto rows_of = [&](const Cur &c, int (&r)[K]) {
        const bool ok = c.s < n && c.w >= 0 && last_of(c);
#pragma unroll
        for (int h = 0; h < K; ++h) r[h] = ok ? __ldg(p.srows + static_cast<int64_t>(c.s) * C + h * 32 + lane) : -1;
    };

    // cursors: a (FMAs now), b (gathers and values in flight), c (columns in flight)
    Cur ca{s0, 0, 0, 0};
    {
        const int2 d = slice_of(s0);
        ca.off = d.x;
        ca.w = d.y;
    }
    int2 dnext = slice_of(s0 + 8);
    Cur cb = ca;
    advance(cb, dnext);
    Cur cc = cb;
    advance(cc, dnext);

    // Two register sets used in turn: set P holds block a (values, gathers,
    // output rows, old y) and receives block c's column indices and rows once
    // block a no longer needs them; set Q holds block b.  Nothing is copied
    // between the sets, so no register still waiting for its load is read
    // before the FMAs that need it.
    struct Set {
        VT v[U][K];
        XT x[U][K];
        int32_t c[U][K];
        int r[K];
        double y[K];
    };
    Set S0, S1;
    rows_of(ca, S0.r);
    load_cols(ca, S0.c);
    gather(ca, S0.c, S0.x);
    load_vals(ca, S0.v);
#pragma unroll
    for (int h = 0; h < K; ++h) S0.y[h] = 0.0;
    if (read_y) {
#pragma unroll
        for (int h = 0; h < K; ++h)
            if (S0.r[h] >= 0) S0.y[h] = widen(y[S0.r[h]]);
    }
    load_cols(cb, S1.c);
    rows_of(cb, S1.r);

    ACC acc[K];
#pragma unroll
    for (int h = 0; h < K; ++h) acc[h].zero();
    auto step = [&](Set &P, Set &Q) {
        // block b: gathers, values, old y (into Q); block c: columns (into P)
        gather(cb, Q.c, Q.x);
        load_vals(cb, Q.v);
        if (read_y) {
#pragma unroll
            for (int h = 0; h < K; ++h) Q.y[h] = (Q.r[h] >= 0) ? widen(y[Q.r[h]]) : 0.0;
        }
        load_cols(cc, P.c);
        // ---- block a ----------------------------------------------------------
        if (ca.w < 0) {
            const int row = ca.off;
            const ChunkDesc d{__ldg(p.m.rp + row), __ldg(p.m.rp + row + 1), row, (row + 1) | kChunkLong};
            long_row<VT, XT, YT, ACC, false>(p.m, d, x, y, alpha, beta, plain, lane);
            if constexpr (DOT) {
                if (lane == 0) dsum = fma(widen(x[row]), widen(y[row]), dsum);  // lane 0 stored it
            }
        } else {
            sell_fma_tail(acc, P.v, P.x, cnt_of(ca));
#pragma unroll
            for (int h = 0; h < K; ++h) end_run(acc[h]);
            if (last_of(ca)) {
#pragma unroll
                for (int h = 0; h < K; ++h) {
                    if (P.r[h] >= 0) {
                        const YT q = sell_store<VT>(p.m, x, y, P.r[h], acc[h], alpha, beta, plain, P.y[h]);
                        if constexpr (DOT) dsum = fma(widen(x[P.r[h]]), widen(q), dsum);
                    }
                    acc[h].zero();
                }
            }
        }
        rows_of(cc, P.r);
        ca = cb;
        cb = cc;
        advance(cc, dnext);
    };
    while (ca.s < n) {
        step(S0, S1);
        if (ca.s >= n) break;
        step(S1, S0);
    }
}

template <typename VT, typename XT, typename YT, typename ACC, bool DOT = false>
__global__ void __launch_bounds__(256) k_sell(const SellParams p, const RedOut o) {
    double dsum = 0.0;
    sell_walk<VT, XT, YT, ACC, DOT>(p, dsum);
    if constexpr (DOT) {
        __shared__ double s_red[32];
        finish(block_sum(dsum, s_red), o, s_red);
    }
}

// ---------------------------------------------------------------------------
// Block vectors on the same slices: Y[:, c0:c0+4] = alpha*A*X[:, c0:c0+4] +
// beta*Y[:, c0:c0+4] for row-major X (leading dimension ldx) and Y (ldy).  Each
// lane keeps 2 rows x 4 right-hand sides = 8 independent FMA chains and walks
// its slices one slot row at a time; a slot's four x values are one 32-byte
// sector (two 16-byte loads when VEC).  FP64 only.
// ---------------------------------------------------------------------------
constexpr int kSellR = 4;  // right-hand sides per pass

struct SellMrParams {
    SellParams b;   // slices, rows, copies, CRS (long rows), n_slices, cstart, alpha, beta
    const double *X;
    double *Y;
    int64_t ldx, ldy;
};

__device__ __forceinline__ double2 ld_gather2(const double *p) {
    double2 v;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// A row too long for a slice, for 4 right-hand sides: lanes stride the row, then
// a butterfly reduction of each sum.
template <bool VEC>
__device__ __forceinline__ void long_row_mr(const SellMrParams &q, int row, double alpha, double beta, bool plain,
                                            int lane) {
    const int32_t *__restrict__ col = q.b.m.col;
    const double *__restrict__ val = static_cast<const double *>(q.b.m.vs);
    const int k0 = __ldg(q.b.m.rp + row), k1 = __ldg(q.b.m.rp + row + 1);
    double acc[kSellR];
#pragma unroll
    for (int r = 0; r < kSellR; ++r) acc[r] = 0.0;
    for (int k = k0 + lane; k < k1; k += 32) {
        const double v = __ldg(val + k);
        const double *xp = q.X + static_cast<int64_t>(__ldg(col + k)) * q.ldx;
#pragma unroll
        for (int r = 0; r < kSellR; ++r) acc[r] = fma(v, __ldg(xp + r), acc[r]);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
        for (int r = 0; r < kSellR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (lane == 0) {
        double *yp = q.Y + static_cast<int64_t>(row) * q.ldy;
#pragma unroll
        for (int r = 0; r < kSellR; ++r)
            yp[r] = plain ? acc[r] : (beta == 0.0 ? alpha * acc[r] : fma(alpha, acc[r], beta * yp[r]));
    }
}

template <bool VEC>
__global__ void __launch_bounds__(256, 2) k_sell_mr(const SellMrParams q) {
    constexpr int K = kSellK, C = kSellC, R = kSellR;
    const SellParams &p = q.b;
    const int lane = threadIdx.x & 31;
    if (static_cast<int>(blockIdx.x) >= p.n_ctas) return;
    const int s0 = __ldg(p.cstart + blockIdx.x) + (threadIdx.x >> 5);
    const int n = __ldg(p.cstart + blockIdx.x + 1);
    if (s0 >= n) return;
    const uint64_t pol = l2_evict_first_policy();
    const double *__restrict__ vals = static_cast<const double *>(p.vals);
    const int32_t *__restrict__ cols = p.cols;
    const double *__restrict__ X = q.X;
    double *__restrict__ Y = q.Y;
    const int64_t ldx = q.ldx, ldy = q.ldy;
    const double alpha = p.alpha, beta = p.beta;
    const bool plain = (alpha == 1.0 && beta == 0.0);

    // cursor: slice s (descriptor off, w) and its slot row j (one per step)
    struct Cur {
        int s, off, w, j;
    };
    auto slice_of = [&](int s) { return s < n ? __ldg(p.slices + s) : make_int2(0, 0); };
    auto has_slot = [&](const Cur &c) { return c.s < n && c.j < c.w; };
    auto last_of = [](const Cur &c) { return c.j + 1 >= c.w; };
    auto advance = [&](Cur &c, int2 &dnext) {
        if (!last_of(c)) {
            c.j += 1;
            return;
        }
        c.s += 8;
        c.off = dnext.x;
        c.w = dnext.y;
        c.j = 0;
        dnext = slice_of(c.s + 8);
    };
    // steps without a slot (long rows, empty slices, past the end) read the
    // leading padding row; nothing inspects the loaded columns before the gather
    auto base_of = [&](const Cur &c) {
        return has_slot(c) ? (static_cast<int64_t>(c.off) + c.j) * C + lane : static_cast<int64_t>(lane);
    };
    struct Set {
        double v[K];
        double x[K][R];
        int32_t c[K];
        int r[K];
    };
    auto load_cols = [&](const Cur &c, Set &S) {
        const int32_t *b = cols + base_of(c);
#pragma unroll
        for (int h = 0; h < K; ++h) S.c[h] = ld_stream(b + h * 32, pol);
    };
    auto load_vals = [&](const Cur &c, Set &S) {
        const double *b = vals + base_of(c);
#pragma unroll
        for (int h = 0; h < K; ++h) S.v[h] = ld_stream(b + h * 32, pol);
    };
    auto gather = [&](const Cur &c, Set &S) {
        const bool ok = has_slot(c);
#pragma unroll
        for (int h = 0; h < K; ++h) {
            if (ok && S.c[h] >= 0) {
                const double *xp = X + static_cast<int64_t>(S.c[h]) * ldx;
                if constexpr (VEC) {
                    const double2 a = ld_gather2(xp), b2 = ld_gather2(xp + 2);
                    S.x[h][0] = a.x;
                    S.x[h][1] = a.y;
                    S.x[h][2] = b2.x;
                    S.x[h][3] = b2.y;
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) S.x[h][r] = ld_gather(xp + r);
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) S.x[h][r] = 0.0;
            }
        }
    };
    auto rows_of = [&](const Cur &c, Set &S) {
        const bool ok = c.s < n && c.w >= 0 && last_of(c);
#pragma unroll
        for (int h = 0; h < K; ++h) S.r[h] = ok ? __ldg(p.srows + static_cast<int64_t>(c.s) * C + h * 32 + lane) : -1;
    };

    Cur ca{s0, 0, 0, 0};
    {
        const int2 d = slice_of(s0);
        ca.off = d.x;
        ca.w = d.y;
    }
    int2 dnext = slice_of(s0 + 8);
    Cur cb = ca;
    advance(cb, dnext);
    Cur cc = cb;
    advance(cc, dnext);

    Set S0, S1;
    rows_of(ca, S0);
    load_cols(ca, S0);
    gather(ca, S0);
    load_vals(ca, S0);
    load_cols(cb, S1);
    rows_of(cb, S1);

    double acc[K][R];
#pragma unroll
    for (int h = 0; h < K; ++h)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[h][r] = 0.0;
    auto step = [&](Set &P, Set &Q) {
        gather(cb, Q);
        load_vals(cb, Q);
        load_cols(cc, P);
        if (ca.w < 0) {
            long_row_mr<VEC>(q, ca.off, alpha, beta, plain, lane);
        } else {
            if (has_slot(ca)) {
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int h = 0; h < K; ++h) acc[h][r] = fma(P.v[h], P.x[h][r], acc[h][r]);
            }
            if (last_of(ca)) {
#pragma unroll
                for (int h = 0; h < K; ++h) {
                    if (P.r[h] >= 0) {
                        double *yp = Y + static_cast<int64_t>(P.r[h]) * ldy;
                        double o[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const double a = acc[h][r];
                            o[r] = plain ? a : (beta == 0.0 ? alpha * a : fma(alpha, a, beta * yp[r]));
                        }
                        if constexpr (VEC) {
                            reinterpret_cast<double2 *>(yp)[0] = make_double2(o[0], o[1]);
                            reinterpret_cast<double2 *>(yp)[1] = make_double2(o[2], o[3]);
                        } else {
#pragma unroll
                            for (int r = 0; r < R; ++r) yp[r] = o[r];
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[h][r] = 0.0;
                }
            }
        }
        rows_of(cc, P);
        ca = cb;
        cb = cc;
        advance(cc, dnext);
    };
    while (ca.s < n) {
        step(S0, S1);
        if (ca.s >= n) break;
        step(S1, S0);
    }
}

// Slot-major copy of the regular slices: row h*32 + l of slice s, holding row
// r, has entry rp[r] + j at slot (off + j)*64 + h*32 + l for j < len(r), value 0
// and column -1 after it.  cols_out may be null (values only, after new values).
template <typename VT>
__global__ void __launch_bounds__(256) k_sell_relayout(const int2 *__restrict__ slices,
                                                       const int32_t *__restrict__ srows, int32_t n_slices,
                                                       const int32_t *__restrict__ rp, const VT *__restrict__ val,
                                                       const int32_t *__restrict__ col, VT *__restrict__ vals_out,
                                                       int32_t *__restrict__ cols_out) {
    const int64_t total = static_cast<int64_t>(n_slices) * kSellC;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int2 d = slices[t / kSellC];
        if (d.y <= 0) continue;
        const int hl = static_cast<int>(t % kSellC);
        const int32_t row = srows[t];
        const int32_t k0 = row >= 0 ? rp[row] : 0;
        const int32_t len = row >= 0 ? rp[row + 1] - k0 : 0;
        for (int j = 0; j < d.y; ++j) {
            const int64_t slot = (static_cast<int64_t>(d.x) + j) * kSellC + hl;
            const bool ok = j < len;
            vals_out[slot] = ok ? val[k0 + j] : VT(0);
            if (cols_out) cols_out[slot] = ok ? col[k0 + j] : -1;
        }
    }
}

template <typename VT, typename XT, typename YT, typename ACC>
struct SellKernel {
    static int grid_limit() {
        static int cached = -1;
        static int cached_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (cached >= 0 && cached_dev == dev) return cached;
        int per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sell<VT, XT, YT, ACC, false>, 256, 0) !=
            cudaSuccess)
            return 0;
        cached = per_sm * sms;
        cached_dev = dev;
        return cached;
    }
    // CTAs of a launch over n_slices slices: up to the resident limit, with at
    // least 8 slices each
    static int ctas_for(int32_t n_slices) {
        const int lim = grid_limit();
        if (lim <= 0) return 0;
        const int64_t want = (static_cast<int64_t>(n_slices) + 7) / 8;
        return static_cast<int>(want < lim ? want : lim);
    }
    static cudaError_t launch(const SellParams &p, cudaStream_t s) {
        if (p.n_slices <= 0 || p.n_ctas <= 0) return cudaSuccess;
        k_sell<VT, XT, YT, ACC, false><<<p.n_ctas, 256, 0, s>>>(p, RedOut{});
        return cudaGetLastError();
    }
    // y = A x with the dot x.y reduced into o (the CG step's p.q); needs at least
    // one slice and at most cg_partials_cap() CTAs
    static cudaError_t launch_dot(const SellParams &p, const RedOut &o, cudaStream_t s) {
        if (p.n_slices <= 0 || p.n_ctas <= 0 || p.n_ctas > cg_partials_cap()) return cudaErrorInvalidValue;
        k_sell<VT, XT, YT, ACC, true><<<p.n_ctas, 256, 0, s>>>(p, o);
        return cudaGetLastError();
    }
};

}  // namespace spmv
