// Auxiliary kernels: the row-vector CRS kernel (T lanes per row, shuffle
// reduction), the halo gather of the split form, the per-entry gradient of the
// reverse pass, the on-device transposed-CRS build and value conversions.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "common.cuh"
#include "slot_kernel.cuh"

namespace spmv {

// ---------------------------------------------------------------------------
// Row-vector kernel: T consecutive lanes share one row of Listing 1, each lane
// running an FMA chain over every T-th entry, then a butterfly shuffle reduce.
// Used for matrices whose rows are long and uniform, and as the tuner's
// alternative to the tile kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ AccF64 shfl_xor_acc(const AccF64 &a, int o, unsigned mask) {
    AccF64 b;
    b.s = __shfl_xor_sync(mask, a.s, o);
    return b;
}
__device__ __forceinline__ AccFF shfl_xor_acc(const AccFF &a, int o, unsigned mask) {
    AccFF b;
    b.h = __shfl_xor_sync(mask, a.h, o);
    b.l = __shfl_xor_sync(mask, a.l, o);
    return b;
}

template <int T, typename VT, typename XT, typename YT, typename ACC>
__global__ void __launch_bounds__(256) k_rowvec(const KParams p, int32_t n_rows) {
    const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t row = gt / T;
    const int lane = threadIdx.x % T;
    const unsigned base = (threadIdx.x & 31u) & ~static_cast<unsigned>(T - 1);
    const unsigned mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << base);
    if (row >= n_rows) return;  // whole T-lane groups leave together
    const int32_t *rp = p.m.rp;
    const int32_t *col = p.m.col;
    const VT *val = static_cast<const VT *>(p.m.vs);
    const XT *x = static_cast<const XT *>(p.m.x);
    YT *y = static_cast<YT *>(p.m.y);
    ACC acc;
    acc.zero();
    const int kb = __ldg(rp + row), ke = __ldg(rp + row + 1);
    for (int k = kb + lane; k < ke; k += T) acc.fma(__ldg(val + k), __ldg(x + __ldg(col + k)));
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) acc.add(shfl_xor_acc(acc, o, mask));
    if (lane == 0) {
        const double v = acc_value<VT, false>(acc, p.m, row, x);
        double out;
        if (p.alpha == 1.0 && p.beta == 0.0) out = v;
        else if (p.beta == 0.0) out = p.alpha * v;
        else out = fma(p.alpha, v, p.beta * widen(y[row]));
        y[row] = narrow<YT>(out);
    }
}

template <int T, typename VT, typename XT, typename YT, typename ACC>
static cudaError_t rowvec_launch(const KParams &p, int32_t n_rows, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const int64_t threads = static_cast<int64_t>(n_rows) * T;
    const int grid = static_cast<int>((threads + 255) / 256);
    k_rowvec<T, VT, XT, YT, ACC><<<grid, 256, 0, s>>>(p, n_rows);
    return cudaGetLastError();
}

cudaError_t launch_rowvec(const KParams &p, const int32_t n_rows, int vk, int xk, int yk, int acc,
                          int T, cudaStream_t s) {
#define SPMV_RV(T_)                                                                       \
    if (T == T_) {                                                                        \
        if (vk == kF64 && xk == kF64 && yk == kF64)                                       \
            return rowvec_launch<T_, double, double, double, AccF64>(p, n_rows, s);       \
        if (vk == kF32 && xk == kF32 && yk == kF32 && acc == kAccFF)                      \
            return rowvec_launch<T_, float, float, float, AccFF>(p, n_rows, s);           \
        if (vk == kF32 && xk == kF32 && yk == kF64 && acc == kAccFF)                      \
            return rowvec_launch<T_, float, float, double, AccFF>(p, n_rows, s);          \
        if (vk == kF32 && xk == kF32 && yk == kF32 && acc == kAccF64)                     \
            return rowvec_launch<T_, float, float, float, AccF64>(p, n_rows, s);          \
        if (vk == kF32 && xk == kF32 && yk == kF64 && acc == kAccF64)                     \
            return rowvec_launch<T_, float, float, double, AccF64>(p, n_rows, s);         \
        return cudaErrorInvalidValue;                                                     \
    }
    SPMV_RV(1)
    SPMV_RV(2)
    SPMV_RV(4)
    SPMV_RV(8)
    SPMV_RV(16)
    SPMV_RV(32)
#undef SPMV_RV
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Halo gather (the stand-in for the MPI exchange of Sect. 3.1-3.5): every
// nonlocal column a block needs is copied into the contiguous halo buffer.
// ---------------------------------------------------------------------------
// halo[h] = x[map[h]]: each thread takes four entries a blockDim apart per
// step, so four map loads and then four x gathers are in flight at once.  (The
// halo stored evict-last in L2 and read back evict-first by the nonlocal part:
// split 248.7 against 232-235 us, dropped.)
__global__ void __launch_bounds__(256) k_gather(const double *__restrict__ x,
                                                const int32_t *__restrict__ map,
                                                double *__restrict__ halo, int64_t n) {
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * 4;
    for (int64_t h0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * 4 + threadIdx.x; h0 < n; h0 += step) {
        int32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t h = h0 + static_cast<int64_t>(u) * blockDim.x;
            c[u] = (h < n) ? __ldg(map + h) : -1;
        }
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (c[u] >= 0) ? __ldg(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t h = h0 + static_cast<int64_t>(u) * blockDim.x;
            if (h < n) halo[h] = v[u];
        }
    }
}

// out[k] = val[perm[k]]: coalesced permutation and output, four gathers per
// thread in flight.
template <typename VT>
__global__ void __launch_bounds__(256) k_permute(const VT *__restrict__ val, const int32_t *__restrict__ perm,
                                                 VT *__restrict__ out, int64_t n) {
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * 4;
    for (int64_t k0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * 4 + threadIdx.x; k0 < n; k0 += step) {
        int32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + static_cast<int64_t>(u) * blockDim.x;
            c[u] = (k < n) ? __ldg(perm + k) : -1;
        }
        VT v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (c[u] >= 0) ? __ldg(val + c[u]) : VT(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + static_cast<int64_t>(u) * blockDim.x;
            if (k < n) out[k] = v[u];
        }
    }
}

cudaError_t launch_permute(const void *val, const int32_t *perm, void *out, int64_t nnz, int vk, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (nnz + 1023) / 1024;
    const int grid = static_cast<int>(want < 8LL * sms ? want : 8LL * sms);
    if (vk == kF64)
        k_permute<double><<<grid, 256, 0, s>>>(static_cast<const double *>(val), perm, static_cast<double *>(out), nnz);
    else
        k_permute<float><<<grid, 256, 0, s>>>(static_cast<const float *>(val), perm, static_cast<float *>(out), nnz);
    return cudaGetLastError();
}

cudaError_t launch_gather(const double *x, const int32_t *map, double *halo, int64_t n,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (n + 1023) / 1024;
    int grid = static_cast<int>(want < 8LL * sms ? want : 8LL * sms);
    k_gather<<<grid, 256, 0, s>>>(x, map, halo, n);
    return cudaGetLastError();
}

// grad_val over the warp chunks of A: lanes take 32 consecutive entries at a
// time (coalesced column loads and gradient stores); the row of each entry is the
// chunk's first row plus the row starts (bits of the chunk's bitmask) up to it.
// Persistent warps walk the chunks c, c + nw, ...: the row-start words and
// column indices of the next chunk (and the descriptors of the two after it) are
// in flight while the current chunk's gathers and stores run, so a warp does not
// wait on one whole load chain per chunk (27-point 128^3 pattern: 163 us; one
// chunk per warp 176-181 us with DRAM 47 % busy; two chunks ahead, at 104
// registers, 366 us; register copies between iterations instead of two sets
// used in turn, 406 us).  MW: mask words per chunk (chunks of at most 32*MW slots).
template <typename VT, int MW>
__global__ void __launch_bounds__(256) k_grad_val_pipe(const int32_t *__restrict__ rp,
                                                       const int32_t *__restrict__ col,
                                                       const ChunkDesc *__restrict__ chunks,
                                                       const uint32_t *__restrict__ masks, int32_t n_chunks,
                                                       const VT *__restrict__ g, const VT *__restrict__ x,
                                                       double alpha, VT *__restrict__ gv) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * 8;
    int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= n_chunks) return;
    const uint64_t pol = l2_evict_first_policy();
    const bool scaled = (alpha != 1.0);
    const VT a = static_cast<VT>(alpha);
    const uint32_t below = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
    auto regular = [](const ChunkDesc &d) { return (d.r1f & (kChunkLong | kChunkEmpty)) == 0; };
    auto load_desc = [&](int cc) {
        if (cc >= n_chunks) return ChunkDesc{0, 0, 0, kChunkEmpty};
        const int4 q = __ldg(reinterpret_cast<const int4 *>(chunks) + cc);
        return ChunkDesc{q.x, q.y, q.z, q.w};
    };
    // row-start words and column indices of a regular chunk (-1: no entry)
    auto load_body = [&](int cc, const ChunkDesc &d, uint32_t (&wds)[MW], int32_t (&cl)[MW]) {
        const bool ok = cc < n_chunks && regular(d);
        const int base = d.k0 & ~3;
#pragma unroll
        for (int wd = 0; wd < MW; ++wd) {
            const int k = base + 32 * wd + lane;
            wds[wd] = ok ? __ldg(masks + static_cast<int64_t>(cc) * MW + wd) : 0u;
            cl[wd] = (ok && k >= d.k0 && k < d.k1) ? ld_stream(col + k, pol) : -1;
        }
    };

    // chunk c's gathers, products and stores (its words and columns loaded one
    // chunk earlier)
    auto process = [&](const ChunkDesc &d, const uint32_t (&wds)[MW], const int32_t (&cl)[MW]) {
        const int r0 = d.r0;
        const int r1 = d.r1f & kChunkRowMask;
        if (d.r1f & kChunkLong) {
            const VT gr = scaled ? static_cast<VT>(a * __ldg(g + r0)) : __ldg(g + r0);
            for (int k = d.k0 + lane; k < d.k1; k += 32) gv[k] = gr * __ldg(x + __ldg(col + k));
        } else if (d.r1f & kChunkEmpty) {
            for (int r = r0 + lane; r < r1; r += 32) {
                const VT gr = scaled ? static_cast<VT>(a * __ldg(g + r)) : __ldg(g + r);
                const int kb = __ldg(rp + r), ke = __ldg(rp + r + 1);
                for (int k = kb; k < ke; ++k) gv[k] = gr * __ldg(x + __ldg(col + k));
            }
        } else {
            const int base = d.k0 & ~3;
            VT xv[MW], gr[MW];
            int rows_before = 0;  // row starts in the chunk's earlier words
#pragma unroll
            for (int wd = 0; wd < MW; ++wd) {
                const int row = r0 + rows_before + __popc(wds[wd] & below) - 1;
                xv[wd] = VT(0);
                gr[wd] = VT(0);
                if (cl[wd] >= 0) {
                    xv[wd] = __ldg(x + cl[wd]);
                    gr[wd] = __ldg(g + row);
                }
                rows_before += __popc(wds[wd]);
            }
#pragma unroll
            for (int wd = 0; wd < MW; ++wd) {
                if (cl[wd] >= 0) {
                    const VT gg = scaled ? static_cast<VT>(a * gr[wd]) : gr[wd];
                    gv[base + 32 * wd + lane] = gg * xv[wd];
                }
            }
        }
    };
    // Two sets of words and columns used in turn (no register copies, so no
    // copy waits on a load still in flight): while one chunk is processed the
    // next one's words and columns arrive in the other set.
    struct Body {
        ChunkDesc d;
        uint32_t w[MW];
        int32_t c[MW];
    };
    Body S0, S1;
    S0.d = load_desc(c);
    load_body(c, S0.d, S0.w, S0.c);
    S1.d = load_desc(c + nw);
    ChunkDesc d2 = load_desc(c + 2 * nw);
    // P: chunk c (loaded), Q: chunk c + nw (descriptor only); afterwards P holds
    // the descriptor of chunk c + 2nw
    auto step = [&](Body &P, Body &Q) {
        load_body(c + nw, Q.d, Q.w, Q.c);
        const ChunkDesc d3 = load_desc(c + 3 * nw);
        process(P.d, P.w, P.c);
        P.d = d2;
        d2 = d3;
        c += nw;
    };
    while (c < n_chunks) {
        step(S0, S1);
        if (c >= n_chunks) break;
        step(S1, S0);
    }
}

template <typename VT>
static int grad_val_grid(int32_t n_chunks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad_val_pipe<VT, kGradValWords>, 256, 0) !=
            cudaSuccess ||
        per_sm <= 0)
        per_sm = 1;
    const int64_t want = (static_cast<int64_t>(n_chunks) + 7) / 8;
    const int64_t lim = static_cast<int64_t>(per_sm) * sms;
    return static_cast<int>(want < lim ? want : lim);
}

cudaError_t launch_grad_val_chunks(const int32_t *rp, const int32_t *col, const void *chunks,
                                   const uint32_t *masks, int mwp, int32_t n_chunks, int vk,
                                   const void *g, const void *x, double alpha, void *grad_val,
                                   cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    if (mwp != kGradValWords) return cudaErrorInvalidValue;
    const ChunkDesc *c = static_cast<const ChunkDesc *>(chunks);
    if (vk == kF64)
        k_grad_val_pipe<double, kGradValWords><<<grad_val_grid<double>(n_chunks), 256, 0, s>>>(
            rp, col, c, masks, n_chunks, static_cast<const double *>(g), static_cast<const double *>(x), alpha,
            static_cast<double *>(grad_val));
    else
        k_grad_val_pipe<float, kGradValWords><<<grad_val_grid<float>(n_chunks), 256, 0, s>>>(
            rp, col, c, masks, n_chunks, static_cast<const float *>(g), static_cast<const float *>(x), alpha,
            static_cast<float *>(grad_val));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Transposed CRS on the device: count entries per column, exclusive scan,
// scatter each entry to its column (atomic cursor), then order every row of A^T
// by original position.  The result is independent of the atomic order.
// ---------------------------------------------------------------------------
__global__ void k_count_cols(const int32_t *__restrict__ col, int64_t nnz, int32_t *cnt) {
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < nnz;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(cnt + __ldg(col + k), 1);
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int32_t block_exclusive_scan(int32_t v, int32_t *out_excl, int32_t *s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t wv = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
        int32_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = wi - wv;  // exclusive warp offsets
        if (lane == 31) s_warp[32] = wi;                            // block total
    }
    __syncthreads();
    *out_excl = s_warp[w] + inc - v;
    const int32_t total = s_warp[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(const int32_t *__restrict__ in,
                                                               int64_t n, int32_t *sums) {
    __shared__ int32_t s_warp[33];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk;
    int32_t v = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + static_cast<int64_t>(i) * kScanThreads + threadIdx.x;
        if (j < n) v += in[j];
    }
    int32_t ex;
    const int32_t tot = block_exclusive_scan(v, &ex, s_warp);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in place (one block, sequential per thread).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t *sums, int32_t nb) {
    __shared__ int32_t s_warp[33];
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per;
    int32_t v = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) v += sums[b0 + i];
    int32_t ex;
    block_exclusive_scan(v, &ex, s_warp);
    int32_t run = ex;
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) {
            const int32_t t = sums[b0 + i];
            sums[b0 + i] = run;
            run += t;
        }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int32_t *__restrict__ in,
                                                             int64_t n,
                                                             const int32_t *__restrict__ offs,
                                                             int32_t *__restrict__ out) {
    __shared__ int32_t s_warp[33];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk +
                         static_cast<int64_t>(threadIdx.x) * kScanItems;
    int32_t loc[kScanItems];
    int32_t v = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        loc[i] = (j < n) ? in[j] : 0;
        v += loc[i];
    }
    int32_t ex;
    const int32_t tot = block_exclusive_scan(v, &ex, s_warp);
    int32_t run = offs[blockIdx.x] + ex;
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + i;
        if (j < n) out[j] = run;
        run += loc[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = offs[blockIdx.x] + tot;
}

// Counts of the columns inside [0, n_cols) only (inputs that were not validated).
__global__ void k_count_cols_checked(const int32_t *__restrict__ col, int64_t nnz, int32_t n_cols,
                                     int32_t *cnt) {
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < nnz;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t c = __ldg(col + k);
        if (c >= 0 && c < n_cols) atomicAdd(cnt + c, 1);
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of the entry indices k = 0..nnz-1 by column (8-bit
// digits, as many passes as the column range needs).  The entries of each
// column of A end up in increasing k, so every row of A^T lists its entries by
// increasing row of A: the unique order the oracle defines.  A pass is a digit
// histogram per CTA range, one exclusive scan of the histograms (digit-major,
// so the ranges of a digit follow each other in CTA order), and a stable
// scatter in which each CTA walks its range in order, 256 entries per round;
// inside a round a warp's entries find their equal-digit peers with a match
// instruction, and the warps' counts are combined in warp order.  The work is
// O(passes * nnz) whatever the column lengths (one dense column costs what a
// stencil costs), and the result does not depend on any atomic order.  The
// key of entry k is read as col[k] in every pass, so only the entry indices
// move (ping-pong between the two output arrays).  A column outside
// [0, n_cols) gets key n_cols (it sorts last; only the allocation-free entry
// point can meet one).
// ---------------------------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kRadixThreads = 256;  // one digit per thread
constexpr int kRadixMaxGrid = 1024;
constexpr int64_t kRadixHistLen = static_cast<int64_t>(kRadixBins) * kRadixMaxGrid;
static_assert(kRadixThreads == kRadixBins, "the scatter gives each thread one digit");

__device__ __forceinline__ int32_t radix_key(const int32_t *__restrict__ col, int32_t k, int32_t n_cols) {
    const int32_t c = __ldg(col + k);
    return (c >= 0 && c < n_cols) ? c : n_cols;
}

// hist[d * grid + g] = entries of CTA range g whose key has digit d.  vin: entry
// indices of the previous pass (nullptr: k itself).
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const int32_t *__restrict__ col,
                                                              const int32_t *__restrict__ vin, int64_t nnz,
                                                              int32_t n_cols, int shift, int64_t per,
                                                              int32_t *__restrict__ hist) {
    __shared__ int32_t s_cnt[kRadixBins];
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t e = min(nnz, b + per);
    for (int64_t i = b + threadIdx.x; i < e; i += kRadixThreads) {
        const int32_t k = vin ? vin[i] : static_cast<int32_t>(i);
        atomicAdd(&s_cnt[(radix_key(col, k, n_cols) >> shift) & (kRadixBins - 1)], 1);
    }
    __syncthreads();
    hist[static_cast<int64_t>(threadIdx.x) * gridDim.x + blockIdx.x] = s_cnt[threadIdx.x];
}

// Stable scatter of CTA range g: offs holds the exclusive scan of hist.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const int32_t *__restrict__ col,
                                                                 const int32_t *__restrict__ vin, int64_t nnz,
                                                                 int32_t n_cols, int shift, int64_t per,
                                                                 const int32_t *__restrict__ offs,
                                                                 int32_t *__restrict__ vout) {
    constexpr int NW = kRadixThreads / 32;
    __shared__ int32_t s_base[kRadixBins];   // next output position of each digit for this CTA
    __shared__ int32_t s_wc[NW][kRadixBins]; // a round's per-warp digit counts, then offsets
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    s_base[t] = offs[static_cast<int64_t>(t) * gridDim.x + blockIdx.x];
#pragma unroll
    for (int q = 0; q < NW; ++q) s_wc[q][t] = 0;
    __syncthreads();
    const int64_t b = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t e = min(nnz, b + per);
    for (int64_t r0 = b; r0 < e; r0 += kRadixThreads) {
        const int64_t i = r0 + t;
        const bool ok = i < e;
        int32_t k = 0;
        int d = kRadixBins;  // past the range: its own peer group, never written
        if (ok) {
            k = vin ? vin[i] : static_cast<int32_t>(i);
            d = (radix_key(col, k, n_cols) >> shift) & (kRadixBins - 1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) s_wc[w][d] = __popc(peers);
        __syncthreads();
        int32_t run = s_base[t];  // digit t: warps in order
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int32_t c = s_wc[q][t];
            s_wc[q][t] = run;
            run += c;
        }
        s_base[t] = run;
        __syncthreads();
        if (ok) {
            const int64_t pos = static_cast<int64_t>(s_wc[w][d]) + rank;
            if (pos >= 0 && pos < nnz) vout[pos] = k;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NW; ++q) s_wc[q][t] = 0;
        __syncthreads();
    }
}

__global__ void k_iota(int32_t *__restrict__ out, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = static_cast<int32_t>(i);
}

// colT[p] = the row of A holding entry perm[p]: the last row i with
// rp[i] <= perm[p] (binary search over rp[0..n_rows - 1], every read inside it).
__global__ void k_rows_of_entries(const int32_t *__restrict__ rp, int32_t n_rows, const int32_t *__restrict__ perm,
                                  int64_t nnz, int32_t *__restrict__ colT) {
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < nnz;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t k = perm[p];
        int32_t lo = 0, hi = n_rows - 1;
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo + 1) / 2;
            if (__ldg(rp + mid) <= k) lo = mid;
            else hi = mid - 1;
        }
        colT[p] = lo;
    }
}

static int radix_passes(int32_t n_cols) {
    // keys lie in [0, n_cols] (n_cols: an invalid column)
    int bits = 0;
    while (bits < 31 && (static_cast<int64_t>(n_cols) >> bits) != 0) ++bits;
    return (bits + kRadixBits - 1) / kRadixBits;
}

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total); sums holds
// (n + kScanChunk - 1) / kScanChunk + 1 entries.
static cudaError_t scan_counts(const int32_t *in, int64_t n, int32_t *sums, int32_t *out, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    k_scan_partial<<<static_cast<int>(nb), kScanThreads, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, static_cast<int32_t>(nb));
    k_scan_final<<<static_cast<int>(nb), kScanThreads, 0, s>>>(in, n, sums, out);
    return cudaGetLastError();
}

// Work layout of the transposed build (int32 entries): column counts
// (n_cols + 1), the column scan's block sums, the radix histograms, their scan
// (kRadixHistLen + 1) and its block sums.
static int64_t col_sums_len(int32_t n_cols) { return (static_cast<int64_t>(n_cols) + kScanChunk - 1) / kScanChunk + 1; }
constexpr int64_t kHistSumsLen = (kRadixHistLen + kScanChunk - 1) / kScanChunk + 1;

int64_t transpose_work_len(int32_t n_cols) {
    return static_cast<int64_t>(n_cols) + 1 + col_sums_len(n_cols) + 2 * kRadixHistLen + 1 + kHistSumsLen;
}

// The transposed structure into rowT (n_cols + 1), colT and perm (nnz each),
// with `work` of transpose_work_len(n_cols) entries.  checked: the arrays were
// not validated, so columns outside [0, n_cols) are left out of the counts (and
// sort last) and every read and write stays inside the stated sizes.
static cudaError_t transpose_into(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                                  int32_t *rowT, int32_t *colT, int32_t *perm, int32_t *work, bool checked,
                                  cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int32_t *cnt = work;
    int32_t *cnt_sums = cnt + n_cols + 1;
    int32_t *hist = cnt_sums + col_sums_len(n_cols);
    int32_t *offs = hist + kRadixHistLen;
    int32_t *hist_sums = offs + kRadixHistLen + 1;
    // row pointer of A^T: counts per column, exclusive scan
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (static_cast<size_t>(n_cols) + 1), s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        if (checked) k_count_cols_checked<<<8 * sms, 256, 0, s>>>(col, nnz, n_cols, cnt);
        else k_count_cols<<<8 * sms, 256, 0, s>>>(col, nnz, cnt);
    }
    if ((e = scan_counts(cnt, n_cols, cnt_sums, rowT, s)) != cudaSuccess) return e;
    if (nnz <= 0) return cudaGetLastError();
    // entry order: stable sort of k by column; the last pass writes perm
    const int passes = radix_passes(n_cols);
    if (passes == 0) {
        k_iota<<<4 * sms, 256, 0, s>>>(perm, nnz);
    } else {
        int64_t grid = (nnz + 4095) / 4096;
        if (grid > kRadixMaxGrid) grid = kRadixMaxGrid;
        const int64_t per = (nnz + grid - 1) / grid;
        const int32_t *src = nullptr;
        for (int j = 0; j < passes; ++j) {
            int32_t *dst = ((passes - 1 - j) % 2 == 0) ? perm : colT;
            const int shift = j * kRadixBits;
            k_radix_hist<<<static_cast<int>(grid), kRadixThreads, 0, s>>>(col, src, nnz, n_cols, shift, per, hist);
            if ((e = scan_counts(hist, kRadixBins * grid, hist_sums, offs, s)) != cudaSuccess) return e;
            k_radix_scatter<<<static_cast<int>(grid), kRadixThreads, 0, s>>>(col, src, nnz, n_cols, shift, per, offs,
                                                                            dst);
            src = dst;
        }
    }
    if (n_rows > 0) k_rows_of_entries<<<8 * sms, 256, 0, s>>>(rp, n_rows, perm, nnz, colT);
    return cudaGetLastError();
}

cudaError_t launch_transpose(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                             int32_t *rowT, int32_t *colT, int32_t *perm, int32_t *work, cudaStream_t s) {
    return transpose_into(n_rows, n_cols, nnz, rp, col, rowT, colT, perm, work, false, s);
}

// ---------------------------------------------------------------------------
// Transposed build without allocation.  Its work array (column counts, the
// column scan's block sums, the radix histograms and their scan) lives in one
// fixed device array that every GPU loading the library holds until the
// process exits.  The inputs are not validated: columns outside [0, n_cols) are
// left out and every read and write stays inside the stated sizes.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxCols = 1 << 20;
constexpr int64_t kNoAllocWorkLen = kNoAllocMaxCols + 1 + (kNoAllocMaxCols + kScanChunk - 1) / kScanChunk + 1 +
                                   2 * kRadixHistLen + 1 + kHistSumsLen;
static __device__ __align__(256) int32_t g_transpose_scratch[kNoAllocWorkLen];

int64_t transpose_noalloc_max_cols() { return kNoAllocMaxCols; }

// Device address of the fixed work array on the current device, looked up once
// per device with that device current (host code cannot use the array's name as
// a device address).  The lookup is serialised, so host threads making their
// first calls at the same time get the same address.  A cudaDeviceReset unloads
// the module and the cached address with it: the library does not support
// calls after one.
static int32_t *noalloc_scratch_ptr(cudaError_t *err) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static int32_t *ptrs[kMaxDevices] = {nullptr};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (ptrs[dev] == nullptr) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_transpose_scratch);
        if (*err != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<int32_t *>(p);
    }
    *err = cudaSuccess;
    return ptrs[dev];
}

cudaError_t launch_transpose_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                     const int32_t *col, int32_t *rowT, int32_t *colT, int32_t *perm,
                                     cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    int32_t *work = noalloc_scratch_ptr(&e);
    if (!work) return e;
    // the array keeps the previous call's contents; transpose_into clears what
    // must start at zero (the column counts) and overwrites the rest
    return transpose_into(n_rows, n_cols, nnz, rp, col, rowT, colT, perm, work, true, s);
}

// ---------------------------------------------------------------------------
// Conversions and fills.
// ---------------------------------------------------------------------------
__global__ void k_f64_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[i] = __double2float_rn(a[i]);
}
__global__ void k_f32_to_f64(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[i] = widen(a[i]);
}

cudaError_t launch_convert(const void *src, int sk, void *dst, int dk, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 16LL * sms));
    if (sk == kF64 && dk == kF32)
        k_f64_to_f32<<<grid, 256, 0, s>>>(static_cast<const double *>(src), static_cast<float *>(dst), n);
    else if (sk == kF32 && dk == kF64)
        k_f32_to_f64<<<grid, 256, 0, s>>>(static_cast<const float *>(src), static_cast<double *>(dst), n);
    else if (sk == dk)
        return cudaMemcpyAsync(dst, src, n * (sk == kF64 ? 8 : 4), cudaMemcpyDeviceToDevice, s);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Failure detection
// ---------------------------------------------------------------------------

static int elementwise_grid(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    return static_cast<int>(want < 16LL * sms ? want : 16LL * sms);
}

// Device-side CRS check: row_ptr[0] == 0, nondecreasing, row_ptr[n_rows] == nnz,
// 0 <= col < n_cols.  Every read stays inside [0, n_rows] of row_ptr and [0, nnz)
// of col_idx whatever their contents; a violation sets *bad (no trap).
__global__ void __launch_bounds__(256) k_validate(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                                  const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ col, int32_t *bad) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t == 0 && (__ldg(rp) != 0 || static_cast<int64_t>(__ldg(rp + n_rows)) != nnz)) atomicExch(bad, 1);
    for (int64_t i = t; i < n_rows; i += stride)
        if (__ldg(rp + i + 1) < __ldg(rp + i)) atomicExch(bad, 1);
    for (int64_t k = t; k < nnz; k += stride) {
        const int32_t c = __ldg(col + k);
        if (c < 0 || c >= n_cols) atomicExch(bad, 1);
    }
}

cudaError_t launch_validate(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                            int32_t *bad, cudaStream_t s) {
    const int64_t work = (static_cast<int64_t>(n_rows) > nnz) ? n_rows : nnz;
    k_validate<<<elementwise_grid(work > 0 ? work : 1), 256, 0, s>>>(n_rows, n_cols, nnz, rp, col, bad);
    return cudaGetLastError();
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// arrives on, with a wall-time limit of limit_ns; the wait gives up, the kernel
// records the timeout in *err and returns.  No copy is in flight on the barrier.
__global__ void k_wait_timeout(uint64_t limit_ns, int32_t *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) set_error(err, kDevErrTimeout);
}

cudaError_t launch_wait_timeout(uint64_t limit_ns, int32_t *err, cudaStream_t s) {
    k_wait_timeout<<<1, 32, 0, s>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace spmv
