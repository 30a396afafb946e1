// C ABI of the library (include/spmv.h): handle management, validation, the
// row-length-histogram autotuner and tile planning, the split plan, the reverse
// pass, the batched graph launch and the CG solvers.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "spmv.h"
#include "internal.h"
#include "cg.h"
#include "warp_kernel.cuh"
#include "slot_kernel.cuh"
#include "sell_kernel.cuh"

namespace spmv {
int64_t transpose_work_len(int32_t n_cols);

bool tile_ops(int vk, int xk, int yk, int acc, int R, int E, bool indirect, bool batched,
              TileOps *ops) {
    if (vk == kF64) {
        if (xk != kF64 || yk != kF64) return false;
        return tile_ops_f64(R, E, indirect, batched, ops);
    }
    return tile_ops_f32(xk, yk, acc, R, E, indirect, batched, ops);
}

bool warp_ops(int vk, int xk, int yk, int acc, int E, bool indirect, bool batched, WarpOps *ops) {
    if (vk == kF64) {
        if (xk != kF64 || yk != kF64) return false;
        return warp_ops_f64(E, indirect, batched, ops);
    }
    if (xk != kF32) return false;
    return warp_ops_f32(yk, acc, E, indirect, batched, ops);
}
}  // namespace spmv

using namespace spmv;

namespace {

struct TileTable {
    TileDesc *d = nullptr;
    int32_t n = 0;
    int32_t n_long = 0;
    std::vector<TileDesc> host;
};

std::vector<TileDesc> make_tiles(const int32_t *rp, int32_t n_rows, int cap, int rowcap, int mat,
                                 int32_t *n_long) {
    std::vector<TileDesc> t;
    int32_t nl = 0;
    int32_t r = 0;
    while (r < n_rows) {
        const int32_t k0 = rp[r];
        if (static_cast<int64_t>(rp[r + 1]) - k0 > cap) {
            TileDesc d{r, r + 1, k0, rp[r + 1], mat, 0, 0, 0};
            t.push_back(d);
            ++nl;
            ++r;
            continue;
        }
        const int32_t lim = static_cast<int32_t>(std::min<int64_t>(n_rows, static_cast<int64_t>(r) + rowcap));
        const int64_t target = static_cast<int64_t>(k0) + cap;
        const int32_t *it = std::upper_bound(rp + r + 1, rp + lim + 1, target,
                                             [](int64_t v, int32_t e) { return v < e; });
        const int32_t r1 = static_cast<int32_t>(it - rp) - 1;
        TileDesc d{r, r1, k0, rp[r1], mat, 0, 0, 0};
        t.push_back(d);
        r = r1;
    }
    if (n_long) *n_long = nl;
    return t;
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return SPMV_ERR_CUDA;        \
    } while (0)

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

// Slot-major copy of a matrix for plan family 4 (per entries-per-lane E).
struct SlotTable {
    ChunkDesc *d = nullptr;
    uint32_t *lmask = nullptr;  // 32 words per chunk
    void *vals = nullptr;       // n * 32E values, slot-major
    int32_t *cols = nullptr;    // n * 32E column indices, slot-major
    int32_t n = 0;
    int32_t n_long = 0, n_empty = 0;
    bool vals_valid = false;
};

// Sorted row-slice copy of a matrix for plan family 5 (per window sigma).
struct SellTable {
    int2 *d = nullptr;          // per slice: first slot row and width (width < 0: long row)
    int32_t *srows = nullptr;   // kSellC rows per slice (-1: none)
    int32_t *cstart = nullptr;  // n_ctas + 1: first slice of each CTA of a launch
    int32_t n_ctas = 0;
    void *vals = nullptr;       // slot_rows * 32 values
    int32_t *cols = nullptr;    // slot_rows * 32 column indices
    int32_t n = 0;
    int32_t n_long = 0;
    int64_t slot_rows = 0;
    bool vals_valid = false;
};

struct ChunkTable {
    ChunkDesc *d = nullptr;
    uint32_t *masks = nullptr;
    int32_t *cmat = nullptr;
    int32_t n = 0;
    int32_t n_long = 0;
    int32_t n_empty = 0;
};

// Cut rows into warp chunks: whole rows whose entries fit in 32*E slots from the
// 16-byte aligned start below the first entry, at most kWarpRowCap rows; one bit
// per slot marks the row starts.  Rows that do not fit alone become long chunks.
void make_chunks(const int32_t *rp, int32_t n_rows, int E, int32_t mat, std::vector<ChunkDesc> &out,
                 std::vector<uint32_t> &masks, std::vector<int32_t> *cmat, int32_t *n_long,
                 int32_t *n_empty) {
    const int64_t SL = 32LL * E;
    const int MW = ((E + 3) / 4) * 4;  // mask words per chunk, rows of 16 bytes
    int32_t r = 0;
    while (r < n_rows) {
        const int32_t k0 = rp[r];
        const int32_t base = k0 & ~3;
        const size_t mo = masks.size();
        masks.resize(mo + MW, 0u);
        if (cmat) cmat->push_back(mat);
        if (static_cast<int64_t>(rp[r + 1]) - base > SL) {
            out.push_back(ChunkDesc{k0, rp[r + 1], r, (r + 1) | kChunkLong});
            ++*n_long;
            ++r;
            continue;
        }
        bool empty = (rp[r + 1] == rp[r]);
        int32_t r1 = r + 1;
        while (r1 < n_rows && r1 - r < kWarpRowCap && static_cast<int64_t>(rp[r1 + 1]) - base <= SL) {
            empty = empty || (rp[r1 + 1] == rp[r1]);
            ++r1;
        }
        out.push_back(ChunkDesc{k0, rp[r1], r, r1 | (empty ? kChunkEmpty : 0)});
        if (empty) ++*n_empty;
        for (int32_t q = r; q < r1; ++q)
            if (rp[q + 1] > rp[q]) {
                const int32_t sl = rp[q] - base;
                masks[mo + (sl >> 5)] |= 1u << (sl & 31);
            }
        r = r1;
    }
}

spmv_status upload_chunks(ChunkTable *ct, const std::vector<ChunkDesc> &d, const std::vector<uint32_t> &m,
                          const std::vector<int32_t> *cmat) {
    ct->n = static_cast<int32_t>(d.size());
    if (dmalloc(&ct->d, d.size()) != cudaSuccess || dmalloc(&ct->masks, m.size()) != cudaSuccess)
        return SPMV_ERR_ALLOC;
    if (cmat && dmalloc(&ct->cmat, cmat->size()) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (!d.empty() && cudaMemcpy(ct->d, d.data(), sizeof(ChunkDesc) * d.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SPMV_ERR_CUDA;
    if (!m.empty() && cudaMemcpy(ct->masks, m.data(), 4 * m.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SPMV_ERR_CUDA;
    if (cmat && !cmat->empty() &&
        cudaMemcpy(ct->cmat, cmat->data(), 4 * cmat->size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SPMV_ERR_CUDA;
    return SPMV_OK;
}

void free_chunks(ChunkTable &ct) {
    cudaFree(ct.d);
    cudaFree(ct.masks);
    cudaFree(ct.cmat);
    ct = ChunkTable();
}

// Chunks for the slot-major layout: the same row packing as make_chunks, from
// the chunk's first entry itself (no alignment), with one word per lane: the row
// starts in its E slots (bits 0..E-1), the rows starting before them (bits
// kSlotPreShift..) and whether its last slot ends a row or the chunk (kSlotEnds).
void make_slot_chunks(const int32_t *rp, int32_t n_rows, int E, std::vector<ChunkDesc> &out,
                      std::vector<uint32_t> &lmask, int32_t *n_long, int32_t *n_empty) {
    const int64_t SL = 32LL * E;
    int32_t r = 0;
    while (r < n_rows) {
        const int32_t k0 = rp[r];
        const size_t mo = lmask.size();
        lmask.resize(mo + 32, 0u);
        if (static_cast<int64_t>(rp[r + 1]) - k0 > SL) {
            out.push_back(ChunkDesc{k0, rp[r + 1], r, (r + 1) | kChunkLong});
            ++*n_long;
            ++r;
            continue;
        }
        bool empty = (rp[r + 1] == rp[r]);
        int32_t r1 = r + 1;
        while (r1 < n_rows && r1 - r < kWarpRowCap && static_cast<int64_t>(rp[r1 + 1]) - k0 <= SL) {
            empty = empty || (rp[r1 + 1] == rp[r1]);
            ++r1;
        }
        out.push_back(ChunkDesc{k0, rp[r1], r, r1 | (empty ? kChunkEmpty : 0)});
        if (empty) ++*n_empty;
        for (int32_t q = r; q < r1; ++q)
            if (rp[q + 1] > rp[q]) {
                const int32_t sl = rp[q] - k0;
                lmask[mo + sl / E] |= 1u << (sl % E);
            }
        if (!empty) {
            const int64_t n_used = static_cast<int64_t>(rp[r1]) - k0;
            uint32_t pre = 0;
            int through_run = 0;  // lanes just before this one that lie inside one row
            for (int lane = 0; lane < 32; ++lane) {
                const uint32_t bits = lmask[mo + lane];
                const bool active = static_cast<int64_t>(lane) * E < n_used;
                const bool ends = static_cast<int64_t>(lane + 1) * E >= n_used ||
                                  (lane < 31 && (lmask[mo + lane + 1] & 1u));
                const bool started = bits != 0u;
                // a piece of a row begun in an earlier lane ends in this lane
                const bool pending = active && !(bits & 1u) && (started || ends);
                const uint32_t chain = pending ? static_cast<uint32_t>(1 + through_run) : 0u;
                through_run = (active && !ends && !started) ? through_run + 1 : 0;
                lmask[mo + lane] = bits | (pre << kSlotPreShift) | (ends ? kSlotEnds : 0u) |
                                   (chain << kSlotChainShift);
                pre += static_cast<uint32_t>(__builtin_popcount(bits));
            }
        }
        r = r1;
    }
}

// Rows longer than this are summed by a whole warp from the CRS arrays instead
// of by one lane of a slice.
constexpr int32_t kSellLongRow = 128;

// Slices of the sorted row-slice layout: in each window of sigma rows, the rows
// of at most kSellLongRow entries ordered by length (longest first, ties in row
// order) and cut into slices of kSellC; each longer row is a slice of its own
// (width -1, x = the row).  Slot rows are numbered consecutively over the slices
// after kSellU rows of padding (a short block loads the slot rows before it).
// Returns false when the slot rows do not fit in int32.
bool make_sell_slices(const int32_t *rp, int32_t n_rows, int32_t sigma, std::vector<int2> &out,
                      std::vector<int32_t> &srows, int32_t *n_long, int64_t *slot_rows) {
    int64_t off = kSellU;
    std::vector<int32_t> idx;
    for (int64_t w0 = 0; w0 < n_rows; w0 += sigma) {
        const int32_t w1 = static_cast<int32_t>(std::min<int64_t>(n_rows, w0 + sigma));
        idx.clear();
        for (int32_t r = static_cast<int32_t>(w0); r < w1; ++r) {
            if (rp[r + 1] - rp[r] > kSellLongRow) {
                out.push_back(make_int2(r, -1));
                srows.insert(srows.end(), kSellC, -1);
                ++*n_long;
            } else {
                idx.push_back(r);
            }
        }
        std::stable_sort(idx.begin(), idx.end(),
                         [rp](int32_t a, int32_t b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
        for (size_t i = 0; i < idx.size(); i += kSellC) {
            const int32_t w = rp[idx[i] + 1] - rp[idx[i]];
            if (off > INT32_MAX) return false;
            out.push_back(make_int2(static_cast<int32_t>(off), w));
            for (size_t l = 0; l < kSellC; ++l) srows.push_back(i + l < idx.size() ? idx[i + l] : -1);
            off += w;
        }
    }
    *slot_rows = off;
    return off <= INT32_MAX;
}

// Padding of the sorted row-slice layout (stored slots / entries - 1) from the
// row lengths alone: per window, a histogram of lengths gives every slice's width.
double sell_padding(const int32_t *rp, int32_t n_rows, int32_t sigma) {
    int64_t slots = 0, used = 0;
    std::vector<int32_t> hist(kSellLongRow + 1);
    for (int64_t w0 = 0; w0 < n_rows; w0 += sigma) {
        const int32_t w1 = static_cast<int32_t>(std::min<int64_t>(n_rows, w0 + sigma));
        std::fill(hist.begin(), hist.end(), 0);
        for (int32_t r = static_cast<int32_t>(w0); r < w1; ++r) {
            const int32_t len = rp[r + 1] - rp[r];
            if (len > kSellLongRow) continue;
            ++hist[len];
            used += len;
        }
        // walk the lengths from the longest: every kSellC-th row opens a slice of its width
        int64_t seen = 0;
        for (int32_t len = kSellLongRow; len >= 0; --len) {
            const int64_t c = hist[len];
            if (c == 0) continue;
            const int64_t opened = (seen + c + kSellC - 1) / kSellC - (seen + kSellC - 1) / kSellC;
            slots += opened * kSellC * len;
            seen += c;
        }
    }
    return used ? static_cast<double>(slots) / used - 1.0 : 0.0;
}

// Contiguous slice ranges of equal work for G CTAs: ws[g] is the first slice
// of CTA g.  A slice's work is its slots plus one slot row for its descriptor,
// rows and stores; a long row's is its entries plus the same.
void sell_ranges(const std::vector<int2> &d, const int32_t *rp, int G, std::vector<int32_t> &ws) {
    std::vector<int64_t> pre(d.size() + 1, 0);
    for (size_t i = 0; i < d.size(); ++i) {
        const int64_t wk = d[i].y >= 0 ? (static_cast<int64_t>(d[i].y) + 1) * kSellC
                                       : static_cast<int64_t>(rp[d[i].x + 1] - rp[d[i].x]) + kSellC;
        pre[i + 1] = pre[i] + wk;
    }
    const int64_t total = pre.back();
    ws.assign(static_cast<size_t>(G) + 1, 0);
    size_t i = 0;
    for (int g = 1; g < G; ++g) {
        const int64_t target = total * g / G;
        while (i < d.size() && pre[i] < target) ++i;
        ws[g] = static_cast<int32_t>(i);
    }
    ws[G] = static_cast<int32_t>(d.size());
}

void free_sell(SellTable &t) {
    cudaFree(t.d);
    cudaFree(t.srows);
    cudaFree(t.cstart);
    cudaFree(t.vals);
    cudaFree(t.cols);
    t = SellTable();
}

void free_slots(SlotTable &t) {
    cudaFree(t.d);
    cudaFree(t.lmask);
    cudaFree(t.vals);
    cudaFree(t.cols);
    t = SlotTable();
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

constexpr int32_t kCheckEvery = 8;  // CG iterations between residual read-backs

struct CgWork {
    int64_t n = 0;
    double *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *r32 = nullptr, *d32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    double *sc = nullptr, *partials = nullptr;
    double *host = nullptr;  // pinned scalars
    // kCheckEvery CG iterations captured once and replayed (host launch overhead
    // paid once per block); re-captured when the operands or the plan change
    cudaGraphExec_t inner32 = nullptr;  // FP32 inner CG of the IR solver
    int64_t inner32_key = -1;
    cudaGraphExec_t cg64 = nullptr;     // FP64 CG (x is the caller's pointer)
    const void *cg64_x = nullptr;
    int64_t cg64_key = -1;
};

struct spmv_matrix {
    int32_t n_rows = 0, n_cols = 0;
    int64_t nnz = 0;
    // symmetric CRS: the CRS arrays hold the upper triangle with the diagonal,
    // and the transposed slots (d_rowT, d_colT, d_perm, h_rowT) the transposed
    // structure of its strictly upper part (perm: positions in the values)
    bool sym = false;
    int vk = kF64;
    int device = 0;
    bool owns_structure = true;
    int32_t *d_rp = nullptr;
    int32_t *d_col = nullptr;
    void *d_val = nullptr;
    int32_t *d_err = nullptr;
    uint64_t values_version = 0;  // incremented by spmv_set_values (batches copy values)
    std::vector<int32_t> h_rp;
    // plan
    double col_random = 0.0;  // column_randomness() of the pattern
    int32_t max_row = 0x7fffffff;  // longest row (set by the tuner)
    int family = 0;  // 0 warp chunks, 1 row-vector, 2 staged tiles, 3 three-stage chunks
    int E = 16;      // entries per lane (family 0) or per thread segment (family 2)
    int T = 8;
    int acc32 = kAccFF;
    std::map<std::pair<int, int>, TileTable> tables;  // (cap, rowcap) -> tiles
    std::map<int, ChunkTable> chunks;                   // E -> warp chunks
    std::map<int, ChunkTable> chunksT;                  // E -> warp chunks of A^T
    std::map<int, SlotTable> slots;                     // E -> slot-major copy (family 4)
    std::map<int, SlotTable> slotsT;                    // E -> slot-major copy of A^T (reverse pass)
    std::map<int, SellTable> sells;                     // sigma -> sorted row-slice copy (family 5)
    std::map<int, SellTable> sellsT;                    // sigma -> sorted row-slice copy of A^T (reverse pass)
    double sell_padT = -1.0;                            // padding of A^T's slices (computed on first use)
    int32_t sigma = 4096;                               // family 5: rows per sorting window
    double sell_pad = 1.0;                              // padding of sorted slices of 4096-row windows
    int32_t *d_rmap = nullptr;                          // output row of each stored row
    // transposed structure (built on first use)
    bool has_T = false;
    int32_t *d_rowT = nullptr, *d_colT = nullptr, *d_perm = nullptr;
    // values of A^T in its row order (val[perm]): laid out by the second reverse
    // pass on the same values (valT_requested records the first one) and
    // invalidated by spmv_set_values
    void *d_valT = nullptr;
    bool valT_valid = false;
    bool valT_requested = false;
    std::vector<int32_t> h_rowT;
    std::map<std::pair<int, int>, TileTable> tablesT;
    // FP32 mirror for IR-CG
    spmv_matrix *mirror32 = nullptr;
    CgWork cg;
};

struct spmv_split {
    spmv_handle A = nullptr;
    int32_t nblocks = 0;
    std::vector<int32_t> block_start, halo_count;
    std::vector<int64_t> nnz_local, nnz_nonlocal;
    std::vector<int32_t> h_halo_map;
    int64_t total_halo = 0;
    int32_t *d_halo_map = nullptr;
    double *d_halo = nullptr;
    spmv_handle Aloc = nullptr, Anl = nullptr;
    cudaEvent_t ev_x = nullptr, ev_halo = nullptr;
    // vector mode: the whole matrix with each nonlocal column renumbered to
    // n + (its position in the concatenated halo), applied to xe = [x | halo]
    spmv_handle Avec = nullptr;
    double *d_xe = nullptr;
};

struct spmv_batch {
    int32_t count = 0;
    int vk = kF64;
    int device = 0;
    std::vector<spmv_handle> mats;
    TileTable tiles;
    ChunkTable chunks;
    int E = 16;
    int grid = 0;
    MatRef *d_mats = nullptr;
    std::vector<MatRef> h_mats;
    int32_t *d_err = nullptr;
    std::vector<const void *> cur_x;
    std::vector<void *> cur_y;
    double cur_alpha = 0.0, cur_beta = 0.0;
    bool graph_valid = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // slot-major path: one copy of all matrices (chunks of matrix m start at
    // slot_off[m]), the matrix of each chunk, and the member values versions the
    // copy was laid out from
    bool use_slots = false;
    SlotTable slots;
    int32_t *d_scmat = nullptr;
    std::vector<int32_t> slot_off;
    std::vector<uint64_t> vals_ver;
    // members tuned apart: member m runs with member_E[m] entries per lane; when
    // both 7 and 9 occur, `slots` holds the E = 7 members and `slots9` the E = 9
    // ones (slot_off[m]: the member's first chunk in its group's copy)
    bool mixed = false;
    std::vector<int32_t> member_E;
    std::vector<int32_t> slot_cnt;  // chunks of each member (mixed batches)
    SlotTable slots9;
    int32_t *d_scmat9 = nullptr;
};

namespace {

TileTable *get_table(spmv_matrix *h, int cap, int rowcap, bool transposed) {
    auto &tabs = transposed ? h->tablesT : h->tables;
    auto key = std::make_pair(cap, rowcap);
    auto it = tabs.find(key);
    if (it != tabs.end()) return &it->second;
    TileTable tt;
    const std::vector<int32_t> &rp = transposed ? h->h_rowT : h->h_rp;
    const int32_t nr = transposed ? h->n_cols : h->n_rows;
    tt.host = make_tiles(rp.data(), nr, cap, rowcap, 0, &tt.n_long);
    tt.n = static_cast<int32_t>(tt.host.size());
    if (dmalloc(&tt.d, tt.host.size()) != cudaSuccess) return nullptr;
    if (!tt.host.empty() &&
        cudaMemcpy(tt.d, tt.host.data(), sizeof(TileDesc) * tt.host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(tt.d);
        return nullptr;
    }
    auto res = tabs.emplace(key, std::move(tt));
    return &res.first->second;
}

void free_tables(std::map<std::pair<int, int>, TileTable> &tabs) {
    for (auto &kv : tabs) cudaFree(kv.second.d);
    tabs.clear();
}

// E values compiled for a (value, x, y, accumulator) combination, largest first.
int pick_E(int vk, int xk, int yk, int acc, int want) {
    const int cands[3] = {31, 15, 7};
    TileOps ops;
    int best = -1;
    for (int c : cands)
        if (tile_ops(vk, xk, yk, acc, 1, c, false, false, &ops)) {
            if (c == want) return c;
            if (best < 0 || std::abs(c - want) < std::abs(best - want)) best = c;
        }
    return best;
}

// Autotuner: from the row-length histogram and the column scatter choose the
// kernel and its work per lane.
//   Columns near the previous row's (stencils, banded matrices) and at least
//   12 entries per row: the sorted row-slice kernel (family 5, windows of 4096
//   rows), when its padding is at most 10 % (27-point 128^3: 113.0 against
//   139.1 us in FP64, 89.6 against 102.9 us with FP32 storage, against the best
//   chunk kernels).  With short rows it gains little alone and loses next to
//   other kernels: on the 7-point 160^3 matrix 69.3 against 71.5 us in a loop
//   of products, but 74-80 against 70-74 us right after a kernel that wrote
//   33 MB (the write-back of that kernel's dirty lines lands on a product
//   already at 90 % of the copy bandwidth), and FP64 CG 109 against 105 ms.
//   Scattered columns: one row per lane gathers x from as many places as the
//   slice has rows, so the slot-major chunk kernel (family 4) stays ahead
//   (Hamiltonian-like 150.4 against 167.3 us): FP64 with E = 7 entries per lane
//   for mean row lengths below 8 and E = 9 above (against the staged chunk
//   kernels 150.6 vs 196.6 us; E = 11, 13, 15 lose to 9; at 8.7 per row, the
//   split's local part, E = 9 takes the one-stream split from 245.9 to 237.1 us;
//   the 7-point matrix, 7 per row, keeps E = 7), FP32 storage with
//   E = 9 (130.2 us; E = 7 133.5, E = 11 135.9, E = 15 138.1, the staged
//   kernel 152 us).
//   Otherwise: family 4 as above for FP64, the two-stage staged chunk kernel
//   with E = 15 for FP32 storage.
// The row-vector kernel's lanes per row T (family 1) is the power of two
// nearest half the mean row length, used when chosen explicitly.
constexpr int32_t kSellSigma = 4096;
constexpr double kSellMaxPadding = 0.10;
constexpr double kSellMinRowLength = 12.0;
// Batched slot-major launch: each member's entries per lane from its own mean
// row length, E = 7 below this many entries per row, else 9.  The threshold is
// lower than a single matrix's (8): on the 256-matrix batch of 5-point
// Laplacians (4.9 per row) and Hamiltonian-like patterns (13 per row), giving
// the Laplacians their own E = 7 group took 0.836 ms against 0.803 ms with every
// member at E = 9 (FP32 storage: 0.660 against 0.631 ms); the whole batch at
// E = 7: 0.90 ms.  Members with shorter rows still get a group of their own.
constexpr double kBatchSlotMeanE9 = 4.0;

void autotune(spmv_matrix *h) {
    const double mean = h->n_rows ? static_cast<double>(h->nnz) / h->n_rows : 0.0;
    h->max_row = 0;
    for (int32_t i = 0; i < h->n_rows; ++i) h->max_row = std::max(h->max_row, h->h_rp[i + 1] - h->h_rp[i]);
    int T = 1;
    while (T < 32 && T < mean * 0.5) T <<= 1;
    h->T = T;
    const bool scattered = h->col_random > 0.25;
    h->sigma = kSellSigma;
    h->sell_pad = h->n_rows > 0 ? sell_padding(h->h_rp.data(), h->n_rows, kSellSigma) : 1.0;
    if (h->vk == kF32) {
        h->family = scattered ? 4 : 0;
        h->E = scattered ? 9 : 15;
    } else {
        h->family = 4;
        h->E = (mean < 8.0) ? 7 : 9;
    }
    if (!scattered && h->sell_pad <= kSellMaxPadding && (h->vk == kF32 || mean >= kSellMinRowLength))
        h->family = 5;
}

// Share of entries (sampled rows) whose column is more than 8 away from every
// column of the previous row: near 0 for stencils and banded matrices, large for
// scattered patterns whose x gathers find nothing in L1.
double column_randomness(const int32_t *rp, const int32_t *col, int32_t n_rows) {
    if (!col || n_rows < 2) return 0.0;
    const int32_t step = std::max<int32_t>(1, n_rows / 32768);
    int64_t far = 0, total = 0;
    std::vector<int32_t> prev;
    for (int32_t i = 1; i < n_rows; i += step) {
        prev.assign(col + rp[i - 1], col + rp[i]);
        std::sort(prev.begin(), prev.end());
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t c = col[k];
            auto it = std::lower_bound(prev.begin(), prev.end(), c);
            int64_t best = INT64_MAX;
            if (it != prev.end()) best = static_cast<int64_t>(*it) - c;
            if (it != prev.begin()) best = std::min<int64_t>(best, static_cast<int64_t>(c) - *(it - 1));
            far += (best > 8) ? 1 : 0;
            ++total;
        }
    }
    return total ? static_cast<double>(far) / total : 0.0;
}

ChunkTable *get_chunks(spmv_matrix *h, int E, bool transposed) {
    auto &tabs = transposed ? h->chunksT : h->chunks;
    auto it = tabs.find(E);
    if (it != tabs.end()) return &it->second;
    std::vector<ChunkDesc> d;
    std::vector<uint32_t> m;
    ChunkTable ct;
    const std::vector<int32_t> &rp = transposed ? h->h_rowT : h->h_rp;
    const int32_t nr = transposed ? h->n_cols : h->n_rows;
    make_chunks(rp.data(), nr, E, 0, d, m, nullptr, &ct.n_long, &ct.n_empty);
    if (upload_chunks(&ct, d, m, nullptr) != SPMV_OK) {
        free_chunks(ct);
        return nullptr;
    }
    return &tabs.emplace(E, ct).first->second;
}

// The slot-major copy for E (built on first use; its values are laid out again
// on the stream after spmv_set_values).  transposed: the copy of A^T, from the
// transposed structure and the values laid out in A^T order (d_valT).
SlotTable *get_slots(spmv_matrix *h, int E, cudaStream_t s, bool transposed = false) {
    auto &tabs = transposed ? h->slotsT : h->slots;
    const int32_t *d_col = transposed ? h->d_colT : h->d_col;
    const void *d_val = transposed ? h->d_valT : h->d_val;
    auto it = tabs.find(E);
    if (it == tabs.end()) {
        std::vector<ChunkDesc> d;
        std::vector<uint32_t> lm;
        SlotTable t;
        if (transposed)
            make_slot_chunks(h->h_rowT.data(), h->n_cols, E, d, lm, &t.n_long, &t.n_empty);
        else
            make_slot_chunks(h->h_rp.data(), h->n_rows, E, d, lm, &t.n_long, &t.n_empty);
        t.n = static_cast<int32_t>(d.size());
        const size_t nslots = static_cast<size_t>(t.n) * 32 * E;
        const size_t vb = (h->vk == kF64) ? 8 : 4;
        bool ok = dmalloc(&t.d, d.size()) == cudaSuccess && dmalloc(&t.lmask, lm.size()) == cudaSuccess &&
                  cudaMalloc(&t.vals, nslots * vb + 16) == cudaSuccess && dmalloc(&t.cols, nslots + 4) == cudaSuccess;
        ok = ok && (d.empty() || cudaMemcpy(t.d, d.data(), sizeof(ChunkDesc) * d.size(), cudaMemcpyHostToDevice) ==
                                     cudaSuccess);
        ok = ok && (lm.empty() || cudaMemcpy(t.lmask, lm.data(), 4 * lm.size(), cudaMemcpyHostToDevice) == cudaSuccess);
        ok = ok && launch_slot_relayout(t.d, E, static_cast<int64_t>(nslots), h->vk, d_val, d_col, t.vals, t.cols,
                                        s) == cudaSuccess;
        if (!ok) {
            free_slots(t);
            (void)cudaGetLastError();  // a failed allocation must not surface at a later launch check
            return nullptr;
        }
        t.vals_valid = true;
        it = tabs.emplace(E, t).first;
    }
    SlotTable &t = it->second;
    if (!t.vals_valid) {
        if (launch_slot_relayout(t.d, E, static_cast<int64_t>(t.n) * 32 * E, h->vk, d_val, nullptr, t.vals,
                                 nullptr, s) != cudaSuccess)
            return nullptr;
        t.vals_valid = true;
    }
    return &t;
}

// The sorted row-slice copy for window sigma (built on first use; its values are
// laid out again on the stream after spmv_set_values).  transposed: the copy of
// A^T, from the transposed structure and the values laid out in A^T order.
SellTable *get_sell(spmv_matrix *h, int32_t sigma, cudaStream_t s, bool transposed = false) {
    auto &tabs = transposed ? h->sellsT : h->sells;
    const int32_t *h_rp = transposed ? h->h_rowT.data() : h->h_rp.data();
    const int32_t nr = transposed ? h->n_cols : h->n_rows;
    const int32_t *d_rp = transposed ? h->d_rowT : h->d_rp;
    const int32_t *d_col = transposed ? h->d_colT : h->d_col;
    const void *d_val = transposed ? h->d_valT : h->d_val;
    auto it = tabs.find(sigma);
    if (it == tabs.end()) {
        std::vector<int2> d;
        std::vector<int32_t> sr;
        SellTable t;
        if (!make_sell_slices(h_rp, nr, sigma, d, sr, &t.n_long, &t.slot_rows)) return nullptr;
        t.n = static_cast<int32_t>(d.size());
        SellOps o;
        const int acc = (h->vk == kF32) ? kAccFF : kAccF64;
        t.n_ctas = sell_ops(h->vk, h->vk, h->vk, acc, &o, transposed ? 0x7fffffff : h->max_row) ? o.ctas_for(t.n) : 0;
        if (t.n_ctas <= 0) return nullptr;
        std::vector<int32_t> ws;
        sell_ranges(d, h_rp, t.n_ctas, ws);
        const size_t nslots = static_cast<size_t>(t.slot_rows) * kSellC;
        const size_t vb = (h->vk == kF64) ? 8 : 4;
        bool ok = dmalloc(&t.d, d.size()) == cudaSuccess && dmalloc(&t.srows, sr.size()) == cudaSuccess &&
                  dmalloc(&t.cstart, ws.size()) == cudaSuccess &&
                  cudaMalloc(&t.vals, nslots * vb + 16) == cudaSuccess && dmalloc(&t.cols, nslots + 4) == cudaSuccess;
        ok = ok && cudaMemcpy(t.cstart, ws.data(), 4 * ws.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        // the leading padding rows: value 0, column -1
        ok = ok && cudaMemsetAsync(t.vals, 0, static_cast<size_t>(kSellU) * kSellC * vb, s) == cudaSuccess &&
             cudaMemsetAsync(t.cols, 0xff, static_cast<size_t>(kSellU) * kSellC * 4, s) == cudaSuccess;
        ok = ok && (d.empty() || cudaMemcpy(t.d, d.data(), sizeof(int2) * d.size(), cudaMemcpyHostToDevice) ==
                                     cudaSuccess);
        ok = ok && (sr.empty() || cudaMemcpy(t.srows, sr.data(), 4 * sr.size(), cudaMemcpyHostToDevice) == cudaSuccess);
        ok = ok && launch_sell_relayout(t.d, t.srows, t.n, d_rp, h->vk, d_val, d_col, t.vals, t.cols, s) == cudaSuccess;
        if (!ok) {
            free_sell(t);
            (void)cudaGetLastError();  // a failed allocation must not surface at a later launch check
            return nullptr;
        }
        t.vals_valid = true;
        it = tabs.emplace(sigma, t).first;
    }
    SellTable &t = it->second;
    if (!t.vals_valid) {
        if (launch_sell_relayout(t.d, t.srows, t.n, d_rp, h->vk, d_val, nullptr, t.vals, nullptr, s) != cudaSuccess)
            return nullptr;
        t.vals_valid = true;
    }
    return &t;
}

void free_chunk_map(std::map<int, ChunkTable> &tabs) {
    for (auto &kv : tabs) free_chunks(kv.second);
    tabs.clear();
}

spmv_status upload_matrix(spmv_matrix *h, const int32_t *row_ptr, const int32_t *col_idx,
                          const void *val, int val_t, bool dev_ptrs, cudaStream_t s) {
    const size_t vsz = (h->vk == kF64) ? 8 : 4;
    const size_t nrp = static_cast<size_t>(h->n_rows) + 1 + kRowPad;
    const size_t nent = static_cast<size_t>(h->nnz) + kEntryPad;
    if (dmalloc(&h->d_rp, nrp) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (dmalloc(&h->d_col, nent) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (cudaMalloc(&h->d_val, nent * vsz) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (dmalloc(&h->d_err, 1) != cudaSuccess) return SPMV_ERR_ALLOC;
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), s));
    CK(cudaMemsetAsync(h->d_rp, 0, nrp * 4, s));
    CK(cudaMemsetAsync(h->d_col, 0, nent * 4, s));
    CK(cudaMemsetAsync(h->d_val, 0, nent * vsz, s));
    CK(cudaMemcpyAsync(h->d_rp, h->h_rp.data(), (static_cast<size_t>(h->n_rows) + 1) * 4,
                       cudaMemcpyHostToDevice, s));
    const cudaMemcpyKind kind = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (h->nnz > 0) {
        CK(cudaMemcpyAsync(h->d_col, col_idx, static_cast<size_t>(h->nnz) * 4, kind, s));
        if (val_t == h->vk) {
            CK(cudaMemcpyAsync(h->d_val, val, static_cast<size_t>(h->nnz) * vsz, kind, s));
        } else {
            // convert on the device through a staging buffer
            void *tmp = nullptr;
            const size_t tsz = static_cast<size_t>(h->nnz) * (val_t == kF64 ? 8 : 4);
            if (cudaMalloc(&tmp, tsz) != cudaSuccess) return SPMV_ERR_ALLOC;
            cudaError_t e = cudaMemcpyAsync(tmp, val, tsz, kind, s);
            if (e == cudaSuccess) e = launch_convert(tmp, val_t, h->d_val, h->vk, h->nnz, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(tmp);
            if (e != cudaSuccess) return SPMV_ERR_CUDA;
        }
    }
    (void)row_ptr;
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
}

void destroy_cg(CgWork &w) {
    if (w.inner32) cudaGraphExecDestroy(w.inner32);
    if (w.cg64) cudaGraphExecDestroy(w.cg64);
    cudaFree(w.r64); cudaFree(w.p64); cudaFree(w.q64);
    cudaFree(w.r32); cudaFree(w.d32); cudaFree(w.p32); cudaFree(w.q32);
    cudaFree(w.sc); cudaFree(w.partials);
    if (w.host) cudaFreeHost(w.host);
    w = CgWork();
}

void destroy_matrix(spmv_matrix *h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    if (h->owns_structure) {
        cudaFree(h->d_rp);
        cudaFree(h->d_col);
    }
    cudaFree(h->d_val);
    cudaFree(h->d_err);
    cudaFree(h->d_rowT);
    cudaFree(h->d_colT);
    cudaFree(h->d_perm);
    cudaFree(h->d_valT);
    free_tables(h->tables);
    free_tables(h->tablesT);
    free_chunk_map(h->chunks);
    free_chunk_map(h->chunksT);
    for (auto &kv : h->slots) free_slots(kv.second);
    for (auto &kv : h->slotsT) free_slots(kv.second);
    for (auto &kv : h->sells) free_sell(kv.second);
    for (auto &kv : h->sellsT) free_sell(kv.second);
    cudaFree(h->d_rmap);
    destroy_cg(h->cg);
    if (h->mirror32) destroy_matrix(h->mirror32);
    delete h;
}

spmv_status create_from_host(spmv_handle *out, int32_t n_rows, int32_t n_cols, int64_t nnz,
                             std::vector<int32_t> &&h_rp, const int32_t *col_idx, const void *val,
                             int val_t, int store_t, bool dev_ptrs, cudaStream_t s,
                             const int32_t *host_col) {
    spmv_matrix *h = new (std::nothrow) spmv_matrix();
    if (!h) return SPMV_ERR_ALLOC;
    cudaGetDevice(&h->device);
    h->n_rows = n_rows;
    h->n_cols = n_cols;
    h->nnz = nnz;
    h->vk = store_t;
    h->h_rp = std::move(h_rp);
    h->col_random = column_randomness(h->h_rp.data(), host_col, n_rows);
    spmv_status st = upload_matrix(h, nullptr, col_idx, val, val_t, dev_ptrs, s);
    if (st != SPMV_OK) {
        destroy_matrix(h);
        return st;
    }
    autotune(h);
    *out = h;
    return SPMV_OK;
}

spmv_status validate_host(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *rp,
                          const int32_t *col) {
    if (rp[0] != 0) return SPMV_ERR_INVALID_INDEX;
    for (int32_t i = 0; i < n_rows; ++i)
        if (rp[i + 1] < rp[i]) return SPMV_ERR_INVALID_INDEX;
    if (rp[n_rows] != nnz) return SPMV_ERR_INVALID_INDEX;
    for (int64_t k = 0; k < nnz; ++k)
        if (col[k] < 0 || col[k] >= n_cols) return SPMV_ERR_INVALID_INDEX;
    return SPMV_OK;
}

struct TileRun {
    TileOps ops;
    TileTable *tt;
    int grid;
};

// Select the compiled kernel and tile table for an apply of h with group width R.
spmv_status prepare_run(spmv_matrix *h, int xk, int yk, int R, int E, bool transposed, TileRun *run) {
    const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
    if (!tile_ops(h->vk, xk, yk, acc, R, E, transposed, false, &run->ops)) return SPMV_ERR_UNSUPPORTED;
    const TileCfg c = run->ops.cfg();
    run->tt = get_table(h, c.cap, c.rowcap, transposed);
    if (!run->tt) return SPMV_ERR_ALLOC;
    const int lim = run->ops.grid_limit();
    if (lim <= 0) return SPMV_ERR_CUDA;
    run->grid = std::min<int>(run->tt->n, lim);
    return SPMV_OK;
}

// The row-slice launch of h for these operands (plan family 5, no row map):
// its compiled configuration and parameters, with the slice copy built on first
// use; false when h does not run on the row slices here.
bool sell_launch_of(spmv_matrix *h, double alpha, const void *x, int xk, double beta, void *y, int yk,
                    cudaStream_t s, SellOps *ops, SellParams *lp) {
    if (h->family != 5 || h->d_rmap) return false;
    const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
    SellTable *lt = nullptr;
    if (!sell_ops(h->vk, xk, yk, acc, ops, h->max_row) || (lt = get_sell(h, h->sigma, s)) == nullptr) return false;
    *lp = SellParams{};
    lp->slices = lt->d;
    lp->srows = lt->srows;
    lp->cstart = lt->cstart;
    lp->n_ctas = lt->n_ctas;
    lp->vals = lt->vals;
    lp->cols = lt->cols;
    lp->m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, x, y, nullptr};
    lp->n_slices = lt->n;
    lp->alpha = alpha;
    lp->beta = beta;
    return true;
}

spmv_status apply_impl(spmv_matrix *h, double alpha, const void *x, int xk, double beta, void *y,
                       int yk, cudaStream_t s) {
    if (h->n_rows == 0) return SPMV_OK;
    const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
    {
        SellOps lops;
        SellParams lp;
        if (sell_launch_of(h, alpha, x, xk, beta, y, yk, s, &lops, &lp))
            return lops.launch(lp, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    }
    if (h->family == 6 && !h->d_rmap) {
        SlotOps tops;
        SlotTable *tt = nullptr;
        if (slot_ops_tv(h->vk, xk, yk, acc, h->E, &tops) && (tt = get_slots(h, h->E, s)) != nullptr) {
            SlotParams sp{};
            sp.chunks = tt->d;
            sp.lmask = tt->lmask;
            sp.vals = tt->vals;
            sp.cols = tt->cols;
            sp.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, x, y, nullptr};
            sp.n_chunks = tt->n;
            sp.alpha = alpha;
            sp.beta = beta;
            sp.err = h->d_err;
            return tops.launch(sp, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
        }
    }
    SlotOps sops;
    SlotTable *t = nullptr;
    if ((h->family == 4 || h->family == 5 || h->family == 6) &&
        ((h->d_rmap && slot_ops(h->vk, xk, yk, acc, h->E, true, &sops)) ||
         slot_ops(h->vk, xk, yk, acc, h->E, false, &sops)) &&
        (t = get_slots(h, h->E, s)) != nullptr) {
        SlotParams sp{};
        sp.chunks = t->d;
        sp.lmask = t->lmask;
        sp.vals = t->vals;
        sp.cols = t->cols;
        sp.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, x, y, h->d_rmap};
        sp.n_chunks = t->n;
        sp.alpha = alpha;
        sp.beta = beta;
        sp.err = h->d_err;
        return sops.launch(sp, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    }
    // the staged chunk kernels (also families 4 and 5 in the vector and
    // accumulator combinations their kernels are not compiled for, FP32 storage
    // with an FP64 result or FP64 accumulation, and when their copies could not
    // be allocated)
    if (h->family == 0 || h->family == 3 || h->family == 4 || h->family == 5 || h->family == 6 || h->d_rmap) {
        int E = h->E;
        if ((h->family == 4 || h->family == 5 || h->family == 6) && E != 7 && E != 15) E = 15;
        WarpOps ops;
        // family 3 selects the three-stage kernel of the same chunking
        const bool ok3 = h->family == 3 && warp_ops(h->vk, xk, yk, acc, E + 100, false, false, &ops);
        if (!ok3 && !warp_ops(h->vk, xk, yk, acc, E, false, false, &ops)) {
            E = 16;
            if (!warp_ops(h->vk, xk, yk, acc, E, false, false, &ops)) return SPMV_ERR_UNSUPPORTED;
        }
        ChunkTable *ct = get_chunks(h, E, false);
        if (!ct) return SPMV_ERR_ALLOC;
        WarpParams wp{};
        wp.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, x, y, h->d_rmap};
        wp.chunks = ct->d;
        wp.masks = ct->masks;
        wp.n_chunks = ct->n;
        wp.alpha = alpha;
        wp.beta = beta;
        wp.err = h->d_err;
        return ops.launch(wp, ct->n, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    }
    KParams p{};
    p.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, x, y, nullptr};
    p.rhs_count = 1;
    p.ldx = 1;
    p.ldy = 1;
    p.alpha = alpha;
    p.beta = beta;
    p.err = h->d_err;
    if (h->family == 1) {
        return launch_rowvec(p, h->n_rows, h->vk, xk, yk, acc, h->T, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    }
    int E = pick_E(h->vk, xk, yk, acc, h->E);
    if (E < 0) return SPMV_ERR_UNSUPPORTED;
    TileRun run;
    spmv_status st = prepare_run(h, xk, yk, 1, E, false, &run);
    if (st != SPMV_OK) return st;
    p.tiles = run.tt->d;
    p.n_tiles = run.tt->n;
    return run.ops.launch(p, run.grid, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
}

spmv_status ensure_transpose(spmv_matrix *h, cudaStream_t s) {
    if (h->has_T) return SPMV_OK;
    const size_t nT = static_cast<size_t>(h->n_cols) + 1 + kRowPad;
    const size_t nent = static_cast<size_t>(h->nnz) + kEntryPad;
    if (dmalloc(&h->d_rowT, nT) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (dmalloc(&h->d_colT, nent) != cudaSuccess) return SPMV_ERR_ALLOC;
    if (dmalloc(&h->d_perm, nent) != cudaSuccess) return SPMV_ERR_ALLOC;
    int32_t *work = nullptr;
    if (dmalloc(&work, static_cast<size_t>(transpose_work_len(h->n_cols))) != cudaSuccess) return SPMV_ERR_ALLOC;
    cudaError_t e = cudaMemsetAsync(h->d_rowT, 0, nT * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_colT, 0, nent * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_perm, 0, nent * 4, s);
    if (e == cudaSuccess)
        e = launch_transpose(h->n_rows, h->n_cols, h->nnz, h->d_rp, h->d_col, h->d_rowT, h->d_colT,
                             h->d_perm, work, s);
    h->h_rowT.assign(static_cast<size_t>(h->n_cols) + 1, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_rowT.data(), h->d_rowT, h->h_rowT.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(work);
    if (e != cudaSuccess) return SPMV_ERR_CUDA;
    h->has_T = true;
    return SPMV_OK;
}

spmv_status ensure_cg(spmv_matrix *h, bool mixed) {
    CgWork &w = h->cg;
    const int64_t n = h->n_rows;
    if (w.sc == nullptr) {
        w.n = n;
        if (dmalloc(&w.sc, kScCount) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.partials, static_cast<size_t>(cg_partials_len())) != cudaSuccess) return SPMV_ERR_ALLOC;
        // the reductions' ticket word (after the partials) starts at zero
        if (cudaMemset(w.partials, 0, static_cast<size_t>(cg_partials_len()) * 8) != cudaSuccess) return SPMV_ERR_CUDA;
        if (cudaMallocHost(reinterpret_cast<void **>(&w.host), 8 * sizeof(double)) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.r64, n) != cudaSuccess) return SPMV_ERR_ALLOC;
    }
    if (!mixed && w.p64 == nullptr) {
        if (dmalloc(&w.p64, n) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.q64, n) != cudaSuccess) return SPMV_ERR_ALLOC;
    }
    if (mixed && w.r32 == nullptr) {
        if (dmalloc(&w.r32, n) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.d32, n) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.p32, n) != cudaSuccess) return SPMV_ERR_ALLOC;
        if (dmalloc(&w.q32, n) != cudaSuccess) return SPMV_ERR_ALLOC;
    }
    return SPMV_OK;
}

spmv_status ensure_mirror32(spmv_matrix *h, cudaStream_t s) {
    if (h->vk == kF32) return SPMV_OK;
    if (h->mirror32) return SPMV_OK;
    spmv_matrix *m = new (std::nothrow) spmv_matrix();
    if (!m) return SPMV_ERR_ALLOC;
    m->device = h->device;
    m->n_rows = h->n_rows;
    m->n_cols = h->n_cols;
    m->nnz = h->nnz;
    m->vk = kF32;
    m->owns_structure = false;
    m->d_rp = h->d_rp;
    m->d_col = h->d_col;
    m->h_rp = h->h_rp;
    m->col_random = h->col_random;
    const size_t nent = static_cast<size_t>(h->nnz) + kEntryPad;
    if (cudaMalloc(&m->d_val, nent * 4) != cudaSuccess || dmalloc(&m->d_err, 1) != cudaSuccess) {
        destroy_matrix(m);
        return SPMV_ERR_ALLOC;
    }
    cudaError_t e = cudaMemsetAsync(m->d_val, 0, nent * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_err, 0, 4, s);
    if (e == cudaSuccess) e = launch_convert(h->d_val, kF64, m->d_val, kF32, h->nnz, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        destroy_matrix(m);
        return SPMV_ERR_CUDA;
    }
    autotune(m);
    h->mirror32 = m;
    return SPMV_OK;
}

}  // namespace

// Everything an apply needs (chunk tables) is built before a capture, so no
// allocation happens while a stream is being captured.
static spmv_status ready_for_capture(spmv_matrix *h, int xk, int yk) {
    const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
    SellOps lops;
    if (h->family == 5 && !h->d_rmap && sell_ops(h->vk, xk, yk, acc, &lops, h->max_row) &&
        get_sell(h, h->sigma, nullptr))
        return cudaDeviceSynchronize() == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    SlotOps sops;
    if ((h->family == 4 || h->family == 5 || h->family == 6) &&
        (slot_ops(h->vk, xk, yk, acc, h->E, h->d_rmap != nullptr, &sops) ||
         (h->family == 6 && !h->d_rmap && slot_ops_tv(h->vk, xk, yk, acc, h->E, &sops))) &&
        get_slots(h, h->E, nullptr))
        return cudaDeviceSynchronize() == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
    if (h->family == 0 || h->family == 3 || h->family == 4 || h->family == 5 || h->family == 6 || h->d_rmap) {
        int E = h->E;
        if ((h->family == 4 || h->family == 5 || h->family == 6) && E != 7 && E != 15) E = 15;
        WarpOps ops;
        const bool ok3 = h->family == 3 && warp_ops(h->vk, xk, yk, acc, E + 100, false, false, &ops);
        if (!ok3 && !warp_ops(h->vk, xk, yk, acc, E, false, false, &ops)) E = 16;
        return get_chunks(h, E, false) ? SPMV_OK : SPMV_ERR_ALLOC;
    }
    if (h->family == 2) {
        const int E = pick_E(h->vk, xk, yk, acc, h->E);
        TileRun run;
        return prepare_run(h, xk, yk, 1, E, false, &run);
    }
    return SPMV_OK;
}

// Capture `body` (which enqueues kernels on the given stream) into a graph.
template <typename F>
static spmv_status capture_graph(F body, cudaGraphExec_t *exec) {
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    spmv_status st = SPMV_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = body(cap);
        e = cudaStreamEndCapture(cap, &g);
    }
    if (e == cudaSuccess && st == SPMV_OK) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (st != SPMV_OK) return st;
    return e == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
}

// Symmetric CRS (Sect. 1.3.1): the handle stores U, the upper triangle with the
// diagonal, once.  The product y = alpha*(U + U_s^T)*x + beta*y runs in two
// passes with a fixed summation order: the row sums of U on the autotuned
// kernel (with beta), then the row sums of U_s^T (the strictly upper part,
// transposed) added onto y by the warp-chunk kernel that reads each value
// through its position in U.
static spmv_status create_symmetric_index(spmv_matrix *h, const int32_t *col_host, cudaStream_t s) {
    const int32_t n = h->n_rows;
    std::vector<int32_t> rowS(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = h->h_rp[i]; k < h->h_rp[i + 1]; ++k)
            if (col_host[k] != i) rowS[static_cast<size_t>(col_host[k]) + 1] += 1;
    for (int32_t j = 0; j < n; ++j) rowS[j + 1] += rowS[j];
    const int64_t ns = rowS[n];
    std::vector<int32_t> colS(static_cast<size_t>(ns)), permS(static_cast<size_t>(ns));
    std::vector<int32_t> next(rowS.begin(), rowS.end() - 1);
    for (int32_t i = 0; i < n; ++i)  // rows of U_s^T list their entries by increasing position in U
        for (int32_t k = h->h_rp[i]; k < h->h_rp[i + 1]; ++k)
            if (col_host[k] != i) {
                const int32_t p = next[col_host[k]]++;
                colS[p] = i;
                permS[p] = k;
            }
    const size_t nT = static_cast<size_t>(n) + 1 + kRowPad;
    const size_t nent = static_cast<size_t>(ns) + kEntryPad;
    if (dmalloc(&h->d_rowT, nT) != cudaSuccess || dmalloc(&h->d_colT, nent) != cudaSuccess ||
        dmalloc(&h->d_perm, nent) != cudaSuccess)
        return SPMV_ERR_ALLOC;
    CK(cudaMemsetAsync(h->d_rowT, 0, nT * 4, s));
    CK(cudaMemsetAsync(h->d_colT, 0, nent * 4, s));
    CK(cudaMemsetAsync(h->d_perm, 0, nent * 4, s));
    CK(cudaMemcpyAsync(h->d_rowT, rowS.data(), rowS.size() * 4, cudaMemcpyHostToDevice, s));
    if (ns) {
        CK(cudaMemcpyAsync(h->d_colT, colS.data(), static_cast<size_t>(ns) * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->d_perm, permS.data(), static_cast<size_t>(ns) * 4, cudaMemcpyHostToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    h->h_rowT = std::move(rowS);
    h->has_T = true;
    return SPMV_OK;
}

static spmv_status apply_sym(spmv_matrix *h, double alpha, const void *x, int xk, double beta, void *y, int yk,
                      cudaStream_t s) {
    const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
    const int32_t n = h->n_rows;
    const int64_t ns = h->h_rowT.empty() ? 0 : h->h_rowT[n];
    WarpOps ops;
    const double meanT = n ? static_cast<double>(ns) / n : 0.0;
    int ET = (meanT < 20.0) ? 7 : 15;
    if (!warp_ops(h->vk, xk, yk, acc, ET, true, false, &ops)) ET = (ET == 7) ? 15 : 7;
    if (ns > 0 && !warp_ops(h->vk, xk, yk, acc, ET, true, false, &ops)) return SPMV_ERR_UNSUPPORTED;
    spmv_status st = apply_impl(h, alpha, x, xk, beta, y, yk, s);
    if (st != SPMV_OK || ns == 0 || n == 0) return st;
    ChunkTable *ct = get_chunks(h, ET, true);
    if (!ct) return SPMV_ERR_ALLOC;
    WarpParams wp{};
    wp.m = MatRef{h->d_rowT, h->d_colT, h->d_perm, h->d_val, x, y, nullptr};
    wp.chunks = ct->d;
    wp.masks = ct->masks;
    wp.n_chunks = ct->n;
    wp.alpha = alpha;
    wp.beta = 1.0;
    wp.err = h->d_err;
    return ops.launch(wp, ct->n, s) == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
}

extern "C" {

const char *spmv_status_string(spmv_status s) {
    switch (s) {
    case SPMV_OK: return "SPMV_OK";
    case SPMV_ERR_INVALID_ARG: return "SPMV_ERR_INVALID_ARG: invalid argument";
    case SPMV_ERR_INVALID_INDEX: return "SPMV_ERR_INVALID_INDEX: invalid row_ptr or column index";
    case SPMV_ERR_CUDA: return "SPMV_ERR_CUDA: CUDA runtime or kernel error";
    case SPMV_ERR_ALLOC: return "SPMV_ERR_ALLOC: allocation failed";
    case SPMV_ERR_UNSUPPORTED: return "SPMV_ERR_UNSUPPORTED: combination not provided";
    case SPMV_ERR_TIMEOUT: return "SPMV_ERR_TIMEOUT: bounded device wait gave up";
    case SPMV_ERR_NOT_CONVERGED: return "SPMV_ERR_NOT_CONVERGED: iteration cap reached";
    }
    return "unknown status";
}

int32_t spmv_version(void) { return 100; }

spmv_status spmv_create(spmv_handle *out, int32_t n_rows, int32_t n_cols, int64_t nnz,
                        const int32_t *row_ptr, const int32_t *col_idx, const void *val,
                        spmv_dtype val_t, int is_device_ptr, void *stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return SPMV_ERR_INVALID_ARG;
    if (val_t != SPMV_F64 && val_t != SPMV_F32) return SPMV_ERR_INVALID_ARG;
    if (!row_ptr || (nnz > 0 && (!col_idx || !val))) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> h_rp(static_cast<size_t>(n_rows) + 1);
    std::vector<int32_t> h_col;
    const int32_t *col_host = col_idx;
    if (is_device_ptr) {
        CK(cudaMemcpyAsync(h_rp.data(), row_ptr, h_rp.size() * 4, cudaMemcpyDeviceToHost, s));
        h_col.resize(static_cast<size_t>(nnz));
        if (nnz) CK(cudaMemcpyAsync(h_col.data(), col_idx, static_cast<size_t>(nnz) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        col_host = h_col.data();
    } else {
        std::memcpy(h_rp.data(), row_ptr, h_rp.size() * 4);
    }
    spmv_status st = validate_host(n_rows, n_cols, nnz, h_rp.data(), col_host);
    if (st != SPMV_OK) return st;
    return create_from_host(out, n_rows, n_cols, nnz, std::move(h_rp), col_idx, val, val_t, val_t,
                            is_device_ptr != 0, s, col_host);
}

void spmv_destroy(spmv_handle h) { destroy_matrix(h); }

spmv_status spmv_set_values(spmv_handle h, const void *val, spmv_dtype t, void *stream) {
    if (!h || (h->nnz > 0 && !val)) return SPMV_ERR_INVALID_ARG;
    if (t != SPMV_F64 && t != SPMV_F32) return SPMV_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->nnz == 0) return SPMV_OK;
    CK(launch_convert(val, t, h->d_val, h->vk, h->nnz, s));
    if (h->mirror32) CK(launch_convert(val, t, h->mirror32->d_val, kF32, h->nnz, s));
    h->valT_valid = false;
    h->valT_requested = false;
    ++h->values_version;
    for (auto &kv : h->slots) kv.second.vals_valid = false;
    for (auto &kv : h->sells) kv.second.vals_valid = false;
    return SPMV_OK;
}

spmv_status spmv_get_info(spmv_handle h, int32_t *n_rows, int32_t *n_cols, int64_t *nnz, int32_t *plan) {
    if (!h) return SPMV_ERR_INVALID_ARG;
    if (n_rows) *n_rows = h->n_rows;
    if (n_cols) *n_cols = h->n_cols;
    if (nnz) *nnz = h->nnz;
    if (plan) {
        DeviceGuard g(h->device);
        const int acc = (h->vk == kF32) ? h->acc32 : kAccF64;
        int32_t E = h->E, nunits = 0, rowcap = 0, nlong = 0, threads = 256;
        if (h->family == 2) {
            E = pick_E(h->vk, h->vk, h->vk, acc, h->E);
            TileOps ops;
            if (E > 0 && tile_ops(h->vk, h->vk, h->vk, acc, 1, E, false, false, &ops)) {
                const TileCfg c = ops.cfg();
                TileTable *tt = get_table(h, c.cap, c.rowcap, false);
                if (tt) {
                    nunits = tt->n;
                    nlong = tt->n_long;
                }
                rowcap = c.rowcap;
                threads = c.threads;
            }
        } else if (h->family == 5) {
            SellTable *t = get_sell(h, h->sigma, nullptr);
            if (t) {
                nunits = t->n;
                nlong = t->n_long;
            }
            E = h->sigma;
            rowcap = kSellC;
            if (cudaDeviceSynchronize() != cudaSuccess) return SPMV_ERR_CUDA;
        } else if (h->family == 4 || h->family == 6) {
            SlotTable *t = get_slots(h, E, nullptr);
            if (t) {
                nunits = t->n;
                nlong = t->n_long;
            }
            rowcap = kWarpRowCap;
            if (cudaDeviceSynchronize() != cudaSuccess) return SPMV_ERR_CUDA;
        } else {
            WarpOps ops;
            const bool ok3 = h->family == 3 && warp_ops(h->vk, h->vk, h->vk, acc, E + 100, false, false, &ops);
            if (!ok3 && !warp_ops(h->vk, h->vk, h->vk, acc, E, false, false, &ops)) E = 16;
            ChunkTable *ct = get_chunks(h, E, false);
            if (ct) {
                nunits = ct->n;
                nlong = ct->n_long;
            }
            rowcap = kWarpRowCap;
        }
        plan[0] = h->family;
        plan[1] = E;
        plan[2] = threads;
        plan[3] = nunits;
        plan[4] = rowcap;
        plan[5] = h->T;
        plan[6] = nlong;
        plan[7] = h->vk;
    }
    return SPMV_OK;
}

spmv_status spmv_row_histogram(spmv_handle h, int32_t nbins, int64_t *counts) {
    if (!h || nbins < 1 || !counts) return SPMV_ERR_INVALID_ARG;
    for (int32_t b = 0; b < nbins; ++b) counts[b] = 0;
    for (int32_t i = 0; i < h->n_rows; ++i) {
        const int32_t len = h->h_rp[i + 1] - h->h_rp[i];
        counts[len < nbins - 1 ? len : nbins - 1] += 1;
    }
    return SPMV_OK;
}

spmv_status spmv_set_plan(spmv_handle h, int32_t family, int32_t param) {
    if (!h || family < 0 || family > 6) return SPMV_ERR_INVALID_ARG;
    if (family == 6) {
        const bool f64 = h->vk == kF64;
        if (param != 0 && !(f64 ? (param == 7 || param == 9) : (param == 9 || param == 15)))
            return SPMV_ERR_INVALID_ARG;
        h->family = 6;
        h->E = param ? param : 9;
        return SPMV_OK;
    }
    if (family == 5) {
        if (param != 0 && (param < 32 || param > (1 << 20) || (param & (param - 1)))) return SPMV_ERR_INVALID_ARG;
        h->family = 5;
        h->sigma = param ? param : 4096;
        return SPMV_OK;
    }
    if (family == 4) {
        if (param != 0 && param != 7 && param != 9 && param != 11 && param != 15) return SPMV_ERR_INVALID_ARG;
        h->family = 4;
        h->E = param ? param : (h->vk == kF32 ? 15 : 9);
        return SPMV_OK;
    }
    if (family == 3) {
        if (param != 0 && param != 7 && param != 11 && param != 15) return SPMV_ERR_INVALID_ARG;
        h->family = 3;
        h->E = param ? param : 7;
        return SPMV_OK;
    }
    if (family == 0) {
        if (param != 0 && param != 7 && param != 8 && param != 15 && param != 16) return SPMV_ERR_INVALID_ARG;
        h->family = 0;
        h->E = param ? param : 16;
    } else if (family == 2) {
        if (param != 0 && (param < 3 || param > 31 || param % 2 == 0)) return SPMV_ERR_INVALID_ARG;
        h->family = 2;
        h->E = param ? param : 15;
    } else {
        if (param != 0 && (param < 1 || param > 32 || (param & (param - 1)))) return SPMV_ERR_INVALID_ARG;
        h->family = 1;
        if (param) h->T = param;
    }
    return SPMV_OK;
}

spmv_status spmv_set_accumulator(spmv_handle h, int32_t acc) {
    if (!h || (acc != 0 && acc != 1)) return SPMV_ERR_INVALID_ARG;
    h->acc32 = (acc == 0) ? kAccF64 : kAccFF;
    return SPMV_OK;
}

spmv_status spmv_apply(spmv_handle h, double alpha, const void *x, spmv_dtype xt, double beta,
                       void *y, spmv_dtype yt, void *stream) {
    if (!h) return SPMV_ERR_INVALID_ARG;
    if ((h->n_rows > 0 && !y) || (h->n_cols > 0 && h->n_rows > 0 && !x)) return SPMV_ERR_INVALID_ARG;
    if (h->vk == kF64 && (xt != SPMV_F64 || yt != SPMV_F64)) return SPMV_ERR_UNSUPPORTED;
    if (h->vk == kF32 && xt != SPMV_F32) return SPMV_ERR_UNSUPPORTED;
    if (yt != SPMV_F64 && yt != SPMV_F32) return SPMV_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (h->sym) return apply_sym(h, alpha, x, xt, beta, y, yt, static_cast<cudaStream_t>(stream));
    return apply_impl(h, alpha, x, xt, beta, y, yt, static_cast<cudaStream_t>(stream));
}

spmv_status spmv_create_symmetric(spmv_handle *out, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                  const int32_t *col_idx, const void *val, spmv_dtype val_t, int is_device_ptr,
                                  void *stream) {
    if (!out) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return SPMV_ERR_INVALID_ARG;
    if (val_t != SPMV_F64 && val_t != SPMV_F32) return SPMV_ERR_INVALID_ARG;
    if (!row_ptr || (nnz > 0 && (!col_idx || !val))) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> h_rp(static_cast<size_t>(n) + 1);
    std::vector<int32_t> h_col(static_cast<size_t>(nnz));
    if (is_device_ptr) {
        CK(cudaMemcpyAsync(h_rp.data(), row_ptr, h_rp.size() * 4, cudaMemcpyDeviceToHost, s));
        if (nnz) CK(cudaMemcpyAsync(h_col.data(), col_idx, static_cast<size_t>(nnz) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::memcpy(h_rp.data(), row_ptr, h_rp.size() * 4);
        if (nnz) std::memcpy(h_col.data(), col_idx, static_cast<size_t>(nnz) * 4);
    }
    spmv_status st = validate_host(n, n, nnz, h_rp.data(), h_col.data());
    if (st != SPMV_OK) return st;
    for (int32_t i = 0; i < n; ++i)  // the upper triangle: no entry left of the diagonal
        for (int32_t k = h_rp[i]; k < h_rp[i + 1]; ++k)
            if (h_col[k] < i) return SPMV_ERR_INVALID_INDEX;
    spmv_handle h = nullptr;
    st = create_from_host(&h, n, n, nnz, std::move(h_rp), col_idx, val, val_t, val_t, is_device_ptr != 0, s,
                          h_col.data());
    if (st != SPMV_OK) return st;
    DeviceGuard g(h->device);
    h->sym = true;
    st = create_symmetric_index(h, h_col.data(), s);
    if (st != SPMV_OK) {
        destroy_matrix(h);
        return st;
    }
    *out = h;
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// Split form
// ---------------------------------------------------------------------------

spmv_status spmv_split_create(spmv_split_handle *out, spmv_handle h, int32_t nblocks,
                              const int32_t *block_row_start, int32_t *halo_count_out) {
    if (!out || !h || nblocks < 1) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    if (h->n_rows != h->n_cols) return SPMV_ERR_INVALID_ARG;
    if (h->vk != kF64 || h->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    const int32_t n = h->n_rows;
    const int64_t nnz = h->nnz;
    std::vector<int32_t> bs(static_cast<size_t>(nblocks) + 1);
    if (block_row_start) {
        for (int b = 0; b <= nblocks; ++b) bs[b] = block_row_start[b];
        if (bs[0] != 0 || bs[nblocks] != n) return SPMV_ERR_INVALID_ARG;
        for (int b = 0; b < nblocks; ++b)
            if (bs[b + 1] < bs[b]) return SPMV_ERR_INVALID_ARG;
    } else {
        // Sect. 3.2: balanced nonzeros; block b starts at the first row whose
        // offset is at least ceil(b*nnz/nblocks)
        bs[0] = 0;
        for (int b = 1; b < nblocks; ++b) {
            const int64_t target = (static_cast<int64_t>(b) * nnz + nblocks - 1) / nblocks;
            const int32_t *it = std::lower_bound(h->h_rp.data(), h->h_rp.data() + n, target,
                                                 [](int32_t e, int64_t v) { return e < v; });
            bs[b] = static_cast<int32_t>(it - h->h_rp.data());
        }
        bs[nblocks] = n;
    }
    // bring the column indices to the host for the one-time bookkeeping
    std::vector<int32_t> col(static_cast<size_t>(nnz));
    if (nnz) CK(cudaMemcpy(col.data(), h->d_col, static_cast<size_t>(nnz) * 4, cudaMemcpyDeviceToHost));
    std::vector<double> val(static_cast<size_t>(nnz));
    if (nnz) CK(cudaMemcpy(val.data(), h->d_val, static_cast<size_t>(nnz) * 8, cudaMemcpyDeviceToHost));

    spmv_split *sp = new (std::nothrow) spmv_split();
    if (!sp) return SPMV_ERR_ALLOC;
    sp->A = h;
    sp->nblocks = nblocks;
    sp->block_start = bs;
    sp->halo_count.assign(nblocks, 0);
    sp->nnz_local.assign(nblocks, 0);
    sp->nnz_nonlocal.assign(nblocks, 0);

    std::vector<int32_t> pos(static_cast<size_t>(n) + 1, -1);
    std::vector<int32_t> rp_loc(static_cast<size_t>(n) + 1, 0), rp_nl(static_cast<size_t>(n) + 1, 0);
    std::vector<int32_t> col_loc, col_nl;
    std::vector<double> val_loc, val_nl;
    std::vector<int32_t> col_vec(static_cast<size_t>(nnz));
    col_loc.reserve(static_cast<size_t>(nnz));
    val_loc.reserve(static_cast<size_t>(nnz));
    for (int b = 0; b < nblocks; ++b) {
        const int32_t lo = bs[b], hi = bs[b + 1];
        // mark the nonlocal columns of this block, then number them in order
        std::vector<char> used;
        used.assign(static_cast<size_t>(n), 0);
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = h->h_rp[i]; k < h->h_rp[i + 1]; ++k) {
                const int32_t c = col[k];
                if (c < lo || c >= hi) used[c] = 1;
            }
        const int64_t off = sp->total_halo;
        int32_t cnt = 0;
        for (int32_t c = 0; c < n; ++c)
            if (used[c]) {
                pos[c] = static_cast<int32_t>(off + cnt);
                sp->h_halo_map.push_back(c);
                ++cnt;
            }
        sp->halo_count[b] = cnt;
        sp->total_halo += cnt;
        for (int32_t i = lo; i < hi; ++i) {
            for (int32_t k = h->h_rp[i]; k < h->h_rp[i + 1]; ++k) {
                const int32_t c = col[k];
                if (c >= lo && c < hi) {
                    col_loc.push_back(c);
                    val_loc.push_back(val[k]);
                    col_vec[k] = c;
                } else {
                    col_nl.push_back(pos[c]);
                    val_nl.push_back(val[k]);
                    col_vec[k] = n + pos[c];
                }
            }
            rp_loc[i + 1] = static_cast<int32_t>(col_loc.size());
            rp_nl[i + 1] = static_cast<int32_t>(col_nl.size());
        }
        sp->nnz_local[b] = rp_loc[hi] - rp_loc[lo];
        sp->nnz_nonlocal[b] = rp_nl[hi] - rp_nl[lo];
    }
    if (sp->total_halo + n >= (int64_t(1) << 31)) {
        delete sp;
        return SPMV_ERR_UNSUPPORTED;
    }
    cudaStream_t s = nullptr;
    spmv_status st = create_from_host(&sp->Aloc, n, n, static_cast<int64_t>(col_loc.size()),
                                      std::vector<int32_t>(rp_loc), col_loc.data(), val_loc.data(),
                                      kF64, kF64, false, s, col_loc.data());
    // the nonlocal part keeps only rows with nonlocal entries; each stored row
    // carries the output row it updates
    std::vector<int32_t> nl_rows, rp_c(1, 0);
    for (int32_t i = 0; i < n; ++i)
        if (rp_nl[i + 1] > rp_nl[i]) {
            nl_rows.push_back(i);
            rp_c.push_back(rp_nl[i + 1]);
        }
    if (st == SPMV_OK)
        st = create_from_host(&sp->Anl, static_cast<int32_t>(nl_rows.size()), static_cast<int32_t>(sp->total_halo),
                              static_cast<int64_t>(col_nl.size()), std::move(rp_c),
                              col_nl.data(), val_nl.data(), kF64, kF64, false, s, nullptr);
    if (st == SPMV_OK) {
        if (dmalloc(&sp->Anl->d_rmap, nl_rows.size()) != cudaSuccess) st = SPMV_ERR_ALLOC;
        else if (!nl_rows.empty() && cudaMemcpy(sp->Anl->d_rmap, nl_rows.data(), 4 * nl_rows.size(),
                                                cudaMemcpyHostToDevice) != cudaSuccess)
            st = SPMV_ERR_CUDA;
    }
    if (st == SPMV_OK) {
        if (dmalloc(&sp->d_halo_map, static_cast<size_t>(sp->total_halo)) != cudaSuccess ||
            dmalloc(&sp->d_halo, static_cast<size_t>(sp->total_halo)) != cudaSuccess)
            st = SPMV_ERR_ALLOC;
    }
    if (st == SPMV_OK && sp->total_halo > 0 &&
        cudaMemcpy(sp->d_halo_map, sp->h_halo_map.data(), static_cast<size_t>(sp->total_halo) * 4,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        st = SPMV_ERR_CUDA;
    if (st == SPMV_OK)
        st = create_from_host(&sp->Avec, n, static_cast<int32_t>(n + sp->total_halo), nnz,
                              std::vector<int32_t>(h->h_rp), col_vec.data(), val.data(), kF64, kF64, false, s,
                              col_vec.data());
    if (st == SPMV_OK && dmalloc(&sp->d_xe, static_cast<size_t>(n + sp->total_halo)) != cudaSuccess)
        st = SPMV_ERR_ALLOC;
    if (st == SPMV_OK && (cudaEventCreateWithFlags(&sp->ev_x, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&sp->ev_halo, cudaEventDisableTiming) != cudaSuccess))
        st = SPMV_ERR_CUDA;
    if (st != SPMV_OK) {
        spmv_split_destroy(sp);
        return st;
    }
    // Plans of the parts (measured on the Hamiltonian-like matrix, 8 blocks): the
    // local part takes the autotuned plan (slot-major); the nonlocal part runs
    // the slot-major kernel with 7 entries per lane and its row epilogue (row
    // map, old y) loaded ahead of the FMA chains (split 283 -> 267 us against the
    // staged three-stage kernel).
    if (sp->Aloc->family == 3) {
        const double mean = n ? static_cast<double>(sp->Aloc->nnz) / n : 0.0;
        sp->Aloc->family = 0;
        sp->Aloc->E = (mean < 20.0) ? 7 : 15;
    }
    sp->Anl->family = 4;
    sp->Anl->E = 7;
    if (halo_count_out)
        for (int b = 0; b < nblocks; ++b) halo_count_out[b] = sp->halo_count[b];
    *out = sp;
    return SPMV_OK;
}

void spmv_split_destroy(spmv_split_handle hs) {
    if (!hs) return;
    DeviceGuard g(hs->A ? hs->A->device : 0);
    cudaDeviceSynchronize();
    destroy_matrix(hs->Aloc);
    destroy_matrix(hs->Anl);
    destroy_matrix(hs->Avec);
    cudaFree(hs->d_xe);
    cudaFree(hs->d_halo_map);
    cudaFree(hs->d_halo);
    if (hs->ev_x) cudaEventDestroy(hs->ev_x);
    if (hs->ev_halo) cudaEventDestroy(hs->ev_halo);
    delete hs;
}

spmv_status spmv_split_get_plan(spmv_split_handle hs, int32_t *nblocks, int32_t *block_start,
                                int32_t *halo_count, int64_t *total_halo, int32_t *halo_map,
                                int64_t *nnz_local, int64_t *nnz_nonlocal) {
    if (!hs) return SPMV_ERR_INVALID_ARG;
    if (nblocks) *nblocks = hs->nblocks;
    if (block_start) std::copy(hs->block_start.begin(), hs->block_start.end(), block_start);
    if (halo_count) std::copy(hs->halo_count.begin(), hs->halo_count.end(), halo_count);
    if (total_halo) *total_halo = hs->total_halo;
    if (halo_map) std::copy(hs->h_halo_map.begin(), hs->h_halo_map.end(), halo_map);
    if (nnz_local) std::copy(hs->nnz_local.begin(), hs->nnz_local.end(), nnz_local);
    if (nnz_nonlocal) std::copy(hs->nnz_nonlocal.begin(), hs->nnz_nonlocal.end(), nnz_nonlocal);
    return SPMV_OK;
}

spmv_status spmv_apply_split(spmv_split_handle hs, double alpha, const double *x, double beta,
                             double *y, void *s_compute, void *s_comm) {
    if (!hs) return SPMV_ERR_INVALID_ARG;
    spmv_matrix *A = hs->A;
    if (A->n_rows > 0 && (!x || !y)) return SPMV_ERR_INVALID_ARG;
    DeviceGuard g(A->device);
    cudaStream_t sc = static_cast<cudaStream_t>(s_compute);
    cudaStream_t sm = static_cast<cudaStream_t>(s_comm);
    // stream 2 ("communication"): wait until x is ready, gather the halo
    if (sm != sc) {
        CK(cudaEventRecord(hs->ev_x, sc));
        CK(cudaStreamWaitEvent(sm, hs->ev_x, 0));
    }
    CK(launch_gather(x, hs->d_halo_map, hs->d_halo, hs->total_halo, sm));
    if (sm != sc) CK(cudaEventRecord(hs->ev_halo, sm));
    // stream 1: local part (overlaps the gather), then the nonlocal part
    spmv_status st = apply_impl(hs->Aloc, alpha, x, kF64, beta, y, kF64, sc);
    if (st != SPMV_OK) return st;
    if (sm != sc) CK(cudaStreamWaitEvent(sc, hs->ev_halo, 0));
    if (hs->Anl->nnz > 0) st = apply_impl(hs->Anl, alpha, hs->d_halo, kF64, 1.0, y, kF64, sc);
    return st;
}

// Vector mode (Sect. 3.4, Fig. kernel_schemes (a)): the whole halo is gathered
// first, then one pass over the full matrix reads local columns from x and
// nonlocal ones from the halo (both in xe), writing y once.
spmv_status spmv_apply_split_vector(spmv_split_handle hs, double alpha, const double *x, double beta,
                                    double *y, void *stream) {
    if (!hs) return SPMV_ERR_INVALID_ARG;
    spmv_matrix *A = hs->A;
    if (A->n_rows > 0 && (!x || !y)) return SPMV_ERR_INVALID_ARG;
    if (!hs->Avec) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = A->n_rows;
    if (n > 0) CK(cudaMemcpyAsync(hs->d_xe, x, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s));
    CK(launch_gather(x, hs->d_halo_map, hs->d_xe + n, hs->total_halo, s));
    return apply_impl(hs->Avec, alpha, hs->d_xe, kF64, beta, y, kF64, s);
}

spmv_status spmv_split_get_halo(spmv_split_handle hs, double *halo_out, void *stream) {
    if (!hs || (!halo_out && hs->total_halo > 0)) return SPMV_ERR_INVALID_ARG;
    DeviceGuard g(hs->A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (hs->total_halo > 0)
        CK(cudaMemcpyAsync(halo_out, hs->d_halo, static_cast<size_t>(hs->total_halo) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// Block vectors
// ---------------------------------------------------------------------------

spmv_status spmm_apply(spmv_handle h, int32_t nrhs, double alpha, const void *X, double beta,
                       void *Y, spmv_dtype vt, void *stream) {
    if (!h || nrhs < 1 || nrhs > 64) return SPMV_ERR_INVALID_ARG;
    if (h->n_rows > 0 && (!X || !Y)) return SPMV_ERR_INVALID_ARG;
    if (vt != SPMV_F64 || h->vk != kF64 || h->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->n_rows == 0) return SPMV_OK;
    if (nrhs == 1) return apply_impl(h, alpha, X, kF64, beta, Y, kF64, s);
    int32_t c0 = 0;
    // Groups of 4 right-hand sides on the sorted row slices (one FMA chain per
    // row and right-hand side, no carries), when the slices pad little and, for
    // scattered columns, X fits in L2: each group gathers 32 bytes of a row of X
    // per entry, which costs a DRAM burst apiece once X is out of L2, where the
    // tile kernel reads whole rows of X once.  Measured (ms, slices against the
    // tile kernel): 27-point 128^3 nrhs 4 / 8 / 16 / 32: 0.384 / 0.767 / 1.774 /
    // 3.566 against 0.589 / 1.155 / 2.242 / 4.261; Hamiltonian-like (X of 134 MB
    // per 4 right-hand sides) nrhs 4: 0.465 against 0.591, nrhs 8 / 16 / 32:
    // 1.461 / 3.999 / 8.156 against 1.105 / 2.125 / 4.104.
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device);
    const bool x_fits = static_cast<double>(h->n_cols) * nrhs * 8.0 <= 1.25 * l2;
    SellTable *t = nullptr;
    if (nrhs >= kSellR && h->sell_pad <= kSellMaxPadding && (h->col_random <= 0.25 || x_fits) &&
        (t = get_sell(h, kSellSigma, s)) != nullptr) {
        const bool vec = (nrhs % 2 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(Y) % 16 == 0);
        SellParams b{};
        b.slices = t->d;
        b.srows = t->srows;
        b.cstart = t->cstart;
        b.vals = t->vals;
        b.cols = t->cols;
        b.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, nullptr, nullptr, nullptr};
        b.n_slices = t->n;
        b.n_ctas = t->n_ctas;
        b.alpha = alpha;
        b.beta = beta;
        for (; c0 + kSellR <= nrhs; c0 += kSellR)
            if (launch_sell_mr(b, static_cast<const double *>(X) + c0, static_cast<double *>(Y) + c0, nrhs, nrhs,
                               vec, s) != cudaSuccess)
                return SPMV_ERR_CUDA;
    }
    // the remaining right-hand sides (all of them without the slices): the tile
    // kernel, up to 32 per launch
    for (; c0 < nrhs; c0 += 32) {
        const int cnt = std::min(32, nrhs - c0);
        int R = 2;
        while (R < cnt) R <<= 1;
        TileRun run;
        spmv_status st = prepare_run(h, kF64, kF64, R, 15, false, &run);
        if (st != SPMV_OK) return st;
        KParams p{};
        p.m = MatRef{h->d_rp, h->d_col, h->d_val, nullptr, static_cast<const double *>(X) + c0,
                     static_cast<double *>(Y) + c0};
        p.tiles = run.tt->d;
        p.n_tiles = run.tt->n;
        p.rhs_count = cnt;
        p.ldx = nrhs;
        p.ldy = nrhs;
        p.alpha = alpha;
        p.beta = beta;
        p.err = h->d_err;
        if (run.ops.launch(p, run.grid, s) != cudaSuccess) return SPMV_ERR_CUDA;
    }
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// Reverse pass
// ---------------------------------------------------------------------------

spmv_status spmv_backward(spmv_handle h, double alpha, const void *g, const void *x, void *grad_x,
                          void *grad_val, void *stream) {
    if (!h) return SPMV_ERR_INVALID_ARG;
    if (h->sym) return SPMV_ERR_UNSUPPORTED;
    if (grad_x && h->n_rows > 0 && !g) return SPMV_ERR_INVALID_ARG;
    if (grad_val && h->nnz > 0 && (!g || !x)) return SPMV_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grad_x && h->n_cols > 0) {
        spmv_status st = ensure_transpose(h, s);
        if (st != SPMV_OK) return st;
        // grad_x = alpha * A^T g: warp chunks over the rows of A^T.  The first
        // reverse pass on a set of values reads them through the permutation
        // (val[perm], inside the staged chunk kernel); a second one on the same
        // values lays them out in the order of A^T once (a streaming permutation
        // pass), and from then on the product runs like a forward product on a
        // slot-major copy of A^T.
        const size_t vb = (h->vk == kF64) ? 8 : 4;
        if (!h->valT_valid && h->valT_requested && h->nnz > 0) {
            if (!h->d_valT && cudaMalloc(&h->d_valT, static_cast<size_t>(h->nnz) * vb) != cudaSuccess) {
                h->d_valT = nullptr;
                return SPMV_ERR_ALLOC;
            }
            CK(launch_permute(h->d_val, h->d_perm, h->d_valT, h->nnz, h->vk, s));
            h->valT_valid = true;
            for (auto &kv : h->slotsT) kv.second.vals_valid = false;
            for (auto &kv : h->sellsT) kv.second.vals_valid = false;
        }
        const bool ind = !h->valT_valid;
        h->valT_requested = true;
        bool done = false;
        const double meanT = h->n_cols ? static_cast<double>(h->nnz) / h->n_cols : 0.0;
        if (!ind && h->col_random <= 0.25 && meanT >= kSellMinRowLength) {
            // A^T of a stencil-like matrix with long rows: the sorted row-slice
            // kernel on a row-slice copy of A^T (as the tuner picks for a forward
            // product of such a matrix)
            if (h->sell_padT < 0.0) h->sell_padT = sell_padding(h->h_rowT.data(), h->n_cols, kSellSigma);
            SellOps lops;
            const int acc = (h->vk == kF32) ? kAccFF : kAccF64;
            SellTable *t = nullptr;
            // without its copy (allocation failed) the slot-major path below runs
            if (h->sell_padT <= kSellMaxPadding && sell_ops(h->vk, h->vk, h->vk, acc, &lops) &&
                (t = get_sell(h, kSellSigma, s, true)) != nullptr) {
                SellParams lp{};
                lp.slices = t->d;
                lp.srows = t->srows;
                lp.cstart = t->cstart;
                lp.vals = t->vals;
                lp.cols = t->cols;
                lp.m = MatRef{h->d_rowT, h->d_colT, h->d_valT, nullptr, g, grad_x, nullptr};
                lp.n_slices = t->n;
                lp.n_ctas = t->n_ctas;
                lp.alpha = alpha;
                lp.beta = 0.0;
                if (lops.launch(lp, s) != cudaSuccess) return SPMV_ERR_CUDA;
                done = true;
            }
        }
        if (!ind && !done) {
            // A^T's values in its own order: the slot-major kernel on a slot-major
            // copy of A^T (E by A^T's mean row length, as for a forward product)
            const int ES = (h->vk == kF32) ? 15 : ((meanT < 8.0) ? 7 : 9);
            SlotOps sops;
            const int acc = (h->vk == kF32) ? kAccFF : kAccF64;
            if (slot_ops(h->vk, h->vk, h->vk, acc, ES, false, &sops)) {
                SlotTable *t = get_slots(h, ES, s, true);
                if (!t) return SPMV_ERR_ALLOC;
                SlotParams sp{};
                sp.chunks = t->d;
                sp.lmask = t->lmask;
                sp.vals = t->vals;
                sp.cols = t->cols;
                sp.m = MatRef{h->d_rowT, h->d_colT, h->d_valT, nullptr, g, grad_x, nullptr};
                sp.n_chunks = t->n;
                sp.alpha = alpha;
                sp.beta = 0.0;
                sp.err = h->d_err;
                if (sops.launch(sp, s) != cudaSuccess) return SPMV_ERR_CUDA;
                done = true;
            }
        }
        if (!done) {
            WarpOps ops;
            const int acc = (h->vk == kF32) ? kAccFF : kAccF64;
            int ET = (meanT < 20.0) ? 7 : 15;
            if (!warp_ops(h->vk, h->vk, h->vk, acc, ET, ind, false, &ops)) ET = 15;
            if (!warp_ops(h->vk, h->vk, h->vk, acc, ET, ind, false, &ops)) return SPMV_ERR_UNSUPPORTED;
            ChunkTable *ct = get_chunks(h, ET, true);
            if (!ct) return SPMV_ERR_ALLOC;
            WarpParams wp{};
            wp.m = ind ? MatRef{h->d_rowT, h->d_colT, h->d_perm, h->d_val, g, grad_x, nullptr}
                       : MatRef{h->d_rowT, h->d_colT, h->d_valT, nullptr, g, grad_x, nullptr};
            wp.chunks = ct->d;
            wp.masks = ct->masks;
            wp.n_chunks = ct->n;
            wp.alpha = alpha;
            wp.beta = 0.0;
            wp.err = h->d_err;
            if (ops.launch(wp, ct->n, s) != cudaSuccess) return SPMV_ERR_CUDA;
        }
    }
    if (grad_val && h->nnz > 0) {
        // warp chunks of kGradValE entries per lane: rows from the row-start bitmasks
        ChunkTable *ct = get_chunks(h, kGradValE, false);
        if (!ct) return SPMV_ERR_ALLOC;
        const int mwp = ((kGradValE + 3) / 4) * 4;
        if (launch_grad_val_chunks(h->d_rp, h->d_col, ct->d, ct->masks, mwp, ct->n, h->vk, g, x, alpha,
                                   grad_val, s) != cudaSuccess)
            return SPMV_ERR_CUDA;
    }
    return SPMV_OK;
}

spmv_status spmv_get_transpose(spmv_handle h, int32_t *rowT_ptr, int32_t *colT_idx, int32_t *perm,
                               void *stream) {
    if (!h) return SPMV_ERR_INVALID_ARG;
    if (h->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    spmv_status st = ensure_transpose(h, s);
    if (st != SPMV_OK) return st;
    if (rowT_ptr) std::copy(h->h_rowT.begin(), h->h_rowT.end(), rowT_ptr);
    if (colT_idx && h->nnz) CK(cudaMemcpyAsync(colT_idx, h->d_colT, static_cast<size_t>(h->nnz) * 4, cudaMemcpyDeviceToHost, s));
    if (perm && h->nnz) CK(cudaMemcpyAsync(perm, h->d_perm, static_cast<size_t>(h->nnz) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
}

spmv_status spmv_transpose_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                   const int32_t *row_ptr, const int32_t *col_idx,
                                   int32_t *rowT_ptr, int32_t *colT_idx, int32_t *perm,
                                   void *stream) {
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return SPMV_ERR_INVALID_ARG;
    if (n_cols > transpose_noalloc_max_cols()) return SPMV_ERR_UNSUPPORTED;
    if (!row_ptr || !rowT_ptr || (nnz > 0 && (!col_idx || !colT_idx || !perm))) return SPMV_ERR_INVALID_ARG;
    cudaError_t e = launch_transpose_noalloc(n_rows, n_cols, nnz, row_ptr, col_idx, rowT_ptr, colT_idx,
                                             perm, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPMV_OK : SPMV_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Batched persistent launch
// ---------------------------------------------------------------------------

spmv_status spmv_batched_create(spmv_batch_handle *out, int32_t count, const spmv_handle *mats) {
    if (!out || count < 1 || !mats) return SPMV_ERR_INVALID_ARG;
    *out = nullptr;
    const int vk = mats[0] ? mats[0]->vk : -1;
    for (int32_t m = 0; m < count; ++m)
        if (!mats[m] || mats[m]->vk != vk) return SPMV_ERR_INVALID_ARG;
    for (int32_t m = 0; m < count; ++m)
        if (mats[m]->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard dg(mats[0]->device);
    spmv_batch *b = new (std::nothrow) spmv_batch();
    if (!b) return SPMV_ERR_ALLOC;
    b->count = count;
    b->vk = vk;
    b->device = mats[0]->device;
    b->mats.assign(mats, mats + count);
    const int acc = (vk == kF32) ? kAccFF : kAccF64;
    WarpOps ops;
    // entries per lane from the batch's combined row-length histogram (mean row
    // length); 16 is compiled for both storage types
    int64_t nnz = 0, rows = 0;
    for (int32_t m = 0; m < count; ++m) {
        nnz += mats[m]->nnz;
        rows += mats[m]->n_rows;
    }
    b->E = (rows && static_cast<double>(nnz) / rows < 20.0) ? 7 : 15;
    // slot-major entries per lane from each member's own row-length histogram
    // (its mean row length): 7 below kBatchSlotMeanE9 entries per row, else 9
    b->member_E.resize(static_cast<size_t>(count));
    bool any7 = false, any9 = false;
    for (int32_t m = 0; m < count; ++m) {
        const double mean = mats[m]->n_rows ? static_cast<double>(mats[m]->nnz) / mats[m]->n_rows : 0.0;
        b->member_E[m] = (mean < kBatchSlotMeanE9) ? 7 : 9;
        (b->member_E[m] == 7 ? any7 : any9) = true;
    }
    SlotOps sops;
    if (any7 && any9 && slot_ops_batched(vk, acc, 7, &sops) && slot_ops_batched(vk, acc, 9, &sops)) {
        // two groups, one copy each, one launch over both
        b->mixed = true;
        b->use_slots = true;
        b->E = 7;
        b->slot_off.assign(static_cast<size_t>(count) + 1, 0);
        b->slot_cnt.assign(static_cast<size_t>(count), 0);
        b->vals_ver.assign(static_cast<size_t>(count), 0);
        const size_t vb = (vk == kF64) ? 8 : 4;
        bool ok = true;
        for (int g = 0; g < 2 && ok; ++g) {
            const int EG = g == 0 ? 7 : 9;
            SlotTable &t = g == 0 ? b->slots : b->slots9;
            int32_t *&dcm = g == 0 ? b->d_scmat : b->d_scmat9;
            std::vector<ChunkDesc> d;
            std::vector<uint32_t> lm;
            std::vector<int32_t> cm;
            for (int32_t m = 0; m < count; ++m) {
                if (b->member_E[m] != EG) continue;
                b->slot_off[m] = static_cast<int32_t>(d.size());
                make_slot_chunks(mats[m]->h_rp.data(), mats[m]->n_rows, EG, d, lm, &t.n_long, &t.n_empty);
                b->slot_cnt[m] = static_cast<int32_t>(d.size()) - b->slot_off[m];
                cm.resize(d.size(), m);
            }
            t.n = static_cast<int32_t>(d.size());
            const size_t nslots = d.size() * 32 * EG;
            ok = dmalloc(&t.d, d.size()) == cudaSuccess && dmalloc(&t.lmask, lm.size()) == cudaSuccess &&
                 dmalloc(&dcm, cm.size()) == cudaSuccess && cudaMalloc(&t.vals, nslots * vb + 16) == cudaSuccess &&
                 dmalloc(&t.cols, nslots + 4) == cudaSuccess;
            ok = ok && (d.empty() || cudaMemcpy(t.d, d.data(), sizeof(ChunkDesc) * d.size(), cudaMemcpyHostToDevice) ==
                                         cudaSuccess);
            ok = ok && (lm.empty() || cudaMemcpy(t.lmask, lm.data(), 4 * lm.size(), cudaMemcpyHostToDevice) == cudaSuccess);
            ok = ok && (cm.empty() || cudaMemcpy(dcm, cm.data(), 4 * cm.size(), cudaMemcpyHostToDevice) == cudaSuccess);
            for (int32_t m = 0; ok && m < count; ++m) {
                if (b->member_E[m] != EG) continue;
                const int64_t off = b->slot_off[m];
                const int64_t nch = b->slot_cnt[m];
                ok = launch_slot_relayout(t.d + off, EG, nch * 32 * EG, vk, mats[m]->d_val, mats[m]->d_col,
                                          static_cast<char *>(t.vals) + off * 32 * EG * vb, t.cols + off * 32 * EG,
                                          nullptr) == cudaSuccess;
                b->vals_ver[m] = mats[m]->values_version;
            }
            t.vals_valid = true;
        }
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
        b->h_mats.resize(static_cast<size_t>(count));
        for (int32_t m = 0; m < count; ++m)
            b->h_mats[m] = MatRef{mats[m]->d_rp, mats[m]->d_col, mats[m]->d_val, nullptr, nullptr, nullptr, nullptr};
        b->cur_x.assign(static_cast<size_t>(count), nullptr);
        b->cur_y.assign(static_cast<size_t>(count), nullptr);
        if (ok && (dmalloc(&b->d_mats, b->h_mats.size()) != cudaSuccess || dmalloc(&b->d_err, 1) != cudaSuccess))
            ok = false;
        if (ok && cudaMemset(b->d_err, 0, 4) != cudaSuccess) ok = false;
        if (!ok) {
            spmv_batched_destroy(b);
            return SPMV_ERR_ALLOC;
        }
        *out = b;
        return SPMV_OK;
    }
    const int ES = any7 ? 7 : 9;
    if (slot_ops_batched(vk, acc, ES, &sops)) {
        // the slot-major chunk kernel over one concatenated copy of all matrices
        b->E = ES;
        b->use_slots = true;
        b->slot_off.assign(static_cast<size_t>(count) + 1, 0);
        b->vals_ver.assign(static_cast<size_t>(count), 0);
        std::vector<ChunkDesc> d;
        std::vector<uint32_t> lm;
        std::vector<int32_t> cm;
        for (int32_t m = 0; m < count; ++m) {
            b->slot_off[m] = static_cast<int32_t>(d.size());
            make_slot_chunks(mats[m]->h_rp.data(), mats[m]->n_rows, ES, d, lm, &b->slots.n_long, &b->slots.n_empty);
            cm.resize(d.size(), m);
        }
        b->slot_off[count] = static_cast<int32_t>(d.size());
        b->slots.n = static_cast<int32_t>(d.size());
        const size_t nslots = d.size() * 32 * ES;
        const size_t vb = (vk == kF64) ? 8 : 4;
        bool ok = dmalloc(&b->slots.d, d.size()) == cudaSuccess && dmalloc(&b->slots.lmask, lm.size()) == cudaSuccess &&
                  dmalloc(&b->d_scmat, cm.size()) == cudaSuccess &&
                  cudaMalloc(&b->slots.vals, nslots * vb + 16) == cudaSuccess &&
                  dmalloc(&b->slots.cols, nslots + 4) == cudaSuccess;
        ok = ok && (d.empty() || cudaMemcpy(b->slots.d, d.data(), sizeof(ChunkDesc) * d.size(),
                                            cudaMemcpyHostToDevice) == cudaSuccess);
        ok = ok && (lm.empty() || cudaMemcpy(b->slots.lmask, lm.data(), 4 * lm.size(), cudaMemcpyHostToDevice) ==
                                      cudaSuccess);
        ok = ok && (cm.empty() || cudaMemcpy(b->d_scmat, cm.data(), 4 * cm.size(), cudaMemcpyHostToDevice) ==
                                      cudaSuccess);
        for (int32_t m = 0; ok && m < count; ++m) {
            const int64_t off = b->slot_off[m], nch = b->slot_off[m + 1] - off;
            ok = launch_slot_relayout(b->slots.d + off, ES, nch * 32 * ES, vk, mats[m]->d_val, mats[m]->d_col,
                                      static_cast<char *>(b->slots.vals) + off * 32 * ES * vb,
                                      b->slots.cols + off * 32 * ES, nullptr) == cudaSuccess;
            b->vals_ver[m] = mats[m]->values_version;
        }
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
        b->slots.vals_valid = true;
        b->h_mats.resize(static_cast<size_t>(count));
        for (int32_t m = 0; m < count; ++m)
            b->h_mats[m] = MatRef{mats[m]->d_rp, mats[m]->d_col, mats[m]->d_val, nullptr, nullptr, nullptr, nullptr};
        b->cur_x.assign(static_cast<size_t>(count), nullptr);
        b->cur_y.assign(static_cast<size_t>(count), nullptr);
        if (ok && (dmalloc(&b->d_mats, b->h_mats.size()) != cudaSuccess || dmalloc(&b->d_err, 1) != cudaSuccess))
            ok = false;
        if (ok && cudaMemset(b->d_err, 0, 4) != cudaSuccess) ok = false;
        b->grid = 0;
        if (!ok) {
            spmv_batched_destroy(b);
            return SPMV_ERR_ALLOC;
        }
        *out = b;
        return SPMV_OK;
    }
    if (!warp_ops(vk, vk, vk, acc, b->E, false, true, &ops)) b->E = 15;
    if (!warp_ops(vk, vk, vk, acc, b->E, false, true, &ops)) {
        delete b;
        return SPMV_ERR_UNSUPPORTED;
    }
    std::vector<ChunkDesc> d;
    std::vector<uint32_t> mk;
    std::vector<int32_t> cm;
    for (int32_t m = 0; m < count; ++m)
        make_chunks(mats[m]->h_rp.data(), mats[m]->n_rows, b->E, m, d, mk, &cm, &b->chunks.n_long,
                    &b->chunks.n_empty);
    b->h_mats.resize(static_cast<size_t>(count));
    for (int32_t m = 0; m < count; ++m)
        b->h_mats[m] = MatRef{mats[m]->d_rp, mats[m]->d_col, mats[m]->d_val, nullptr, nullptr, nullptr, nullptr};
    b->cur_x.assign(static_cast<size_t>(count), nullptr);
    b->cur_y.assign(static_cast<size_t>(count), nullptr);
    spmv_status st = upload_chunks(&b->chunks, d, mk, &cm);
    if (st == SPMV_OK && (dmalloc(&b->d_mats, b->h_mats.size()) != cudaSuccess || dmalloc(&b->d_err, 1) != cudaSuccess))
        st = SPMV_ERR_ALLOC;
    if (st == SPMV_OK && cudaMemset(b->d_err, 0, 4) != cudaSuccess) st = SPMV_ERR_CUDA;
    b->grid = (b->chunks.n + 7) / 8;
    if (st != SPMV_OK) {
        spmv_batched_destroy(b);
        return st;
    }
    *out = b;
    return SPMV_OK;
}

void spmv_batched_destroy(spmv_batch_handle b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    free_chunks(b->chunks);
    free_slots(b->slots);
    free_slots(b->slots9);
    cudaFree(b->d_scmat);
    cudaFree(b->d_scmat9);
    cudaFree(b->d_mats);
    cudaFree(b->d_err);
    delete b;
}

spmv_status spmv_batched_apply(spmv_batch_handle b, double alpha, const void *const *x, double beta,
                               void *const *y, void *stream) {
    if (!b || !x || !y) return SPMV_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool recapture = (alpha != b->cur_alpha || beta != b->cur_beta || !b->graph_valid);
    bool ptrs_changed = false;
    for (int32_t m = 0; m < b->count; ++m) {
        if (b->mats[m]->n_rows > 0 && (!x[m] || !y[m])) return SPMV_ERR_INVALID_ARG;
        if (x[m] != b->cur_x[m] || y[m] != b->cur_y[m]) ptrs_changed = true;
    }
    if (ptrs_changed) {
        for (int32_t m = 0; m < b->count; ++m) {
            b->cur_x[m] = x[m];
            b->cur_y[m] = y[m];
            b->h_mats[m].x = x[m];
            b->h_mats[m].y = y[m];
        }
        // the table is read by the kernel when the graph runs; copy it in stream order
        CK(cudaMemcpyAsync(b->d_mats, b->h_mats.data(), sizeof(MatRef) * b->h_mats.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    const int acc = (b->vk == kF32) ? kAccFF : kAccF64;
    if (b->use_slots) {
        if (b->slots.n == 0 && b->slots9.n == 0) return SPMV_OK;
        // members given new values since the copy: lay their values out again
        const size_t vb = (b->vk == kF64) ? 8 : 4;
        for (int32_t m = 0; m < b->count; ++m)
            if (b->mats[m]->values_version != b->vals_ver[m]) {
                const int EG = b->mixed ? b->member_E[m] : b->E;
                const SlotTable &t = (b->mixed && EG == 9) ? b->slots9 : b->slots;
                const int64_t off = b->slot_off[m];
                const int64_t nch = b->mixed ? b->slot_cnt[m] : b->slot_off[m + 1] - off;
                CK(launch_slot_relayout(t.d + off, EG, nch * 32 * EG, b->vk, b->mats[m]->d_val, nullptr,
                                        static_cast<char *>(t.vals) + off * 32 * EG * vb, nullptr, s));
                b->vals_ver[m] = b->mats[m]->values_version;
            }
        SlotOps sops;
        if (!b->mixed && !slot_ops_batched(b->vk, acc, b->E, &sops)) return SPMV_ERR_UNSUPPORTED;
        if (recapture) {
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
            b->graph_valid = false;
            SlotParams p{};
            p.chunks = b->slots.d;
            p.lmask = b->slots.lmask;
            p.vals = b->slots.vals;
            p.cols = b->slots.cols;
            p.mats = b->d_mats;
            p.cmat = b->d_scmat;
            p.n_chunks = b->slots.n;
            p.alpha = alpha;
            p.beta = beta;
            SlotParams p9 = p;
            if (b->mixed) {
                p9.chunks = b->slots9.d;
                p9.lmask = b->slots9.lmask;
                p9.vals = b->slots9.vals;
                p9.cols = b->slots9.cols;
                p9.cmat = b->d_scmat9;
                p9.n_chunks = b->slots9.n;
            }
            cudaStream_t cap;
            CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = cudaSuccess;
                if (b->mixed) {
                    // the two groups as two kernel nodes of the one graph
                    SlotOps s7, s9;
                    if (!slot_ops_batched(b->vk, acc, 7, &s7) || !slot_ops_batched(b->vk, acc, 9, &s9)) {
                        le = cudaErrorInvalidValue;
                    } else {
                        le = s7.launch(p, cap);
                        if (le == cudaSuccess) le = s9.launch(p9, cap);
                    }
                } else {
                    le = sops.launch(p, cap);
                }
                e = cudaStreamEndCapture(cap, &b->graph);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) return SPMV_ERR_CUDA;
            b->graph_valid = true;
            b->cur_alpha = alpha;
            b->cur_beta = beta;
        }
        CK(cudaGraphLaunch(b->exec, s));
        return SPMV_OK;
    }
    if (b->chunks.n == 0) return SPMV_OK;
    WarpOps ops;
    if (!warp_ops(b->vk, b->vk, b->vk, acc, b->E, false, true, &ops)) return SPMV_ERR_UNSUPPORTED;
    if (recapture) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        b->graph_valid = false;
        WarpParams p{};
        p.mats = b->d_mats;
        p.chunks = b->chunks.d;
        p.masks = b->chunks.masks;
        p.cmat = b->chunks.cmat;
        p.n_chunks = b->chunks.n;
        p.alpha = alpha;
        p.beta = beta;
        p.err = b->d_err;
        cudaStream_t cap;
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = ops.launch(p, b->chunks.n, cap);
            e = cudaStreamEndCapture(cap, &b->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return SPMV_ERR_CUDA;
        b->graph_valid = true;
        b->cur_alpha = alpha;
        b->cur_beta = beta;
    }
    CK(cudaGraphLaunch(b->exec, s));
    return SPMV_OK;
}

spmv_status spmv_batched_get_info(spmv_batch_handle b, int32_t *plan) {
    if (!b || !plan) return SPMV_ERR_INVALID_ARG;
    plan[0] = b->mixed ? 0 : b->E;
    plan[1] = 256;
    plan[2] = b->use_slots ? b->slots.n + b->slots9.n : b->chunks.n;
    plan[3] = b->grid;
    return SPMV_OK;
}

spmv_status spmv_batched_get_member_plan(spmv_batch_handle b, int32_t *entries_per_lane) {
    if (!b || !entries_per_lane) return SPMV_ERR_INVALID_ARG;
    for (int32_t m = 0; m < b->count; ++m)
        entries_per_lane[m] = b->use_slots ? (b->mixed ? b->member_E[m] : b->E) : b->E;
    return SPMV_OK;
}

// ---------------------------------------------------------------------------
// CG solvers
// ---------------------------------------------------------------------------

spmv_status spmv_cg(spmv_handle h, const double *b, double *x, double tol, int32_t max_iter,
                    double *stats, void *stream) {
    if (!h || !b || !x || h->n_rows != h->n_cols || h->vk != kF64 || max_iter < 0) return SPMV_ERR_INVALID_ARG;
    if (h->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    spmv_status st = ensure_cg(h, false);
    if (st != SPMV_OK) return st;
    CgWork &w = h->cg;
    const int64_t n = h->n_rows;
    // x = 0, r = b, p = b, rho = b.b
    CK(cudaMemsetAsync(x, 0, static_cast<size_t>(n) * 8, s));
    CK(cudaMemcpyAsync(w.r64, b, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.p64, b, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cg_dot(b, kF64, b, kF64, n, w.partials, w.sc, kOpStore, kScRho, s));
    CK(cudaMemcpyAsync(w.host, w.sc + kScRho, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bb = w.host[0];
    double rho = bb;
    int32_t it = 0;
    // the residual is read back every kCheckEvery iterations (one host round trip
    // per check, not per iteration); CG may run up to kCheckEvery-1 extra steps
    auto iter = [&](cudaStream_t cs) -> spmv_status {
        spmv_status s2 = apply_impl(h, 1.0, w.p64, kF64, 0.0, w.q64, kF64, cs);
        if (s2 != SPMV_OK) return s2;
        if (cg_dot(w.p64, kF64, w.q64, kF64, n, w.partials, w.sc, kOpAlpha, 0, cs) != cudaSuccess ||
            cg_update64(x, w.r64, w.p64, w.q64, n, w.partials, w.sc, cs) != cudaSuccess ||
            cg_direction(w.p64, w.r64, kF64, w.sc, n, cs) != cudaSuccess)
            return SPMV_ERR_CUDA;
        return SPMV_OK;
    };
    const int64_t key = static_cast<int64_t>(h->family) * 1000 + h->E;
    while (it < max_iter && std::sqrt(rho) > tol * std::sqrt(bb)) {
        if (max_iter - it >= kCheckEvery && w.cg64 && w.cg64_key == key && w.cg64_x == x) {
            CK(cudaGraphLaunch(w.cg64, s));
            it += kCheckEvery;
        } else {
            const int blk = std::min<int32_t>(kCheckEvery, max_iter - it);
            for (int j = 0; j < blk; ++j) {
                st = iter(s);
                if (st != SPMV_OK) return st;
            }
            it += blk;
            if (blk == kCheckEvery && (!w.cg64 || w.cg64_key != key || w.cg64_x != x)) {
                if (w.cg64) { cudaGraphExecDestroy(w.cg64); w.cg64 = nullptr; }
                st = ready_for_capture(h, kF64, kF64);
                if (st == SPMV_OK)
                    st = capture_graph([&](cudaStream_t cs) -> spmv_status {
                        for (int j = 0; j < kCheckEvery; ++j) {
                            const spmv_status s3 = iter(cs);
                            if (s3 != SPMV_OK) return s3;
                        }
                        return SPMV_OK;
                    }, &w.cg64);
                if (st != SPMV_OK) return st;
                w.cg64_key = key;
                w.cg64_x = x;
            }
        }
        CK(cudaMemcpyAsync(w.host, w.sc + kScRho, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        rho = w.host[0];
    }
    // true residual in FP64
    CK(cudaMemcpyAsync(w.r64, b, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s));
    st = apply_impl(h, -1.0, x, kF64, 1.0, w.r64, kF64, s);
    if (st != SPMV_OK) return st;
    CK(cg_dot(w.r64, kF64, w.r64, kF64, n, w.partials, w.sc, kOpStore, kScNorm, s));
    CK(cudaMemcpyAsync(w.host, w.sc + kScNorm, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double relres = bb > 0 ? std::sqrt(w.host[0] / bb) : 0.0;
    if (stats) {
        stats[0] = 1;
        stats[1] = it;
        stats[2] = relres;
        stats[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return (std::sqrt(rho) > tol * std::sqrt(bb)) ? SPMV_ERR_NOT_CONVERGED : SPMV_OK;
}

spmv_status spmv_ir_cg(spmv_handle h, const double *b, double *x, double outer_tol,
                       int32_t max_outer, double inner_tol, int32_t max_inner, double *stats,
                       void *stream) {
    if (!h || !b || !x || h->n_rows != h->n_cols || h->vk != kF64 || max_outer < 0 || max_inner < 1)
        return SPMV_ERR_INVALID_ARG;
    if (h->sym) return SPMV_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    spmv_status st = ensure_cg(h, true);
    if (st != SPMV_OK) return st;
    st = ensure_mirror32(h, s);
    if (st != SPMV_OK) return st;
    spmv_matrix *A32 = h->mirror32;
    CgWork &w = h->cg;
    const int64_t n = h->n_rows;
    CK(cudaMemsetAsync(x, 0, static_cast<size_t>(n) * 8, s));
    CK(cg_dot(b, kF64, b, kF64, n, w.partials, w.sc, kOpStore, kScNorm, s));
    CK(cudaMemcpyAsync(w.host, w.sc + kScNorm, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(w.host[0]);
    int32_t outer = 0;
    int64_t inner_total = 0;
    double relres = 0.0;
    bool converged = false;
    for (;;) {
        // outer (FP64): r = b - A x, ||r||
        CK(cudaMemcpyAsync(w.r64, b, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToDevice, s));
        st = apply_impl(h, -1.0, x, kF64, 1.0, w.r64, kF64, s);
        if (st != SPMV_OK) return st;
        CK(cg_dot(w.r64, kF64, w.r64, kF64, n, w.partials, w.sc, kOpStore, kScNorm, s));
        CK(cudaMemcpyAsync(w.host, w.sc + kScNorm, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double rnorm = std::sqrt(w.host[0]);
        relres = bnorm > 0 ? rnorm / bnorm : 0.0;
        if (relres <= outer_tol) { converged = true; break; }
        if (outer >= max_outer) break;
        // inner (FP32 storage): CG on A d = r / ||r||
        CK(cg_scale_to32(w.r64, w.r32, 1.0 / rnorm, n, s));
        CK(cudaMemsetAsync(w.d32, 0, static_cast<size_t>(n) * 4, s));
        CK(cudaMemcpyAsync(w.p32, w.r32, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToDevice, s));
        CK(cg_dot(w.r32, kF32, w.r32, kF32, n, w.partials, w.sc, kOpStore, kScRho, s));
        CK(cudaMemcpyAsync(w.host, w.sc + kScRho, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double rho0 = w.host[0];
        double rho = rho0;
        int32_t it = 0;
        auto inner_iter = [&](cudaStream_t cs) -> spmv_status {
            // q = A p with p.q (and the step alpha) reduced by the product itself
            // on the row slices; elsewhere the product, then the dot
            SellOps lo;
            SellParams lp;
            if (sell_launch_of(A32, 1.0, w.p32, kF32, 0.0, w.q32, kF32, cs, &lo, &lp) && lo.launch_dot &&
                lp.n_slices > 0 && lp.n_ctas <= cg_partials_cap()) {
                if (lo.launch_dot(lp, cg_red_out(w.partials, w.sc, kOpAlpha, 0), cs) != cudaSuccess)
                    return SPMV_ERR_CUDA;
            } else {
                spmv_status s2 = apply_impl(A32, 1.0, w.p32, kF32, 0.0, w.q32, kF32, cs);
                if (s2 != SPMV_OK) return s2;
                if (cg_dot(w.p32, kF32, w.q32, kF32, n, w.partials, w.sc, kOpAlpha, 0, cs) != cudaSuccess)
                    return SPMV_ERR_CUDA;
            }
            if (cg_update32(w.d32, w.r32, w.p32, w.q32, n, w.partials, w.sc, cs) != cudaSuccess ||
                cg_direction(w.p32, w.r32, kF32, w.sc, n, cs) != cudaSuccess)
                return SPMV_ERR_CUDA;
            return SPMV_OK;
        };
        const int64_t key = static_cast<int64_t>(A32->family) * 1000 + A32->E;
        while (it < max_inner && std::sqrt(rho) > inner_tol * std::sqrt(rho0)) {
            if (max_inner - it >= kCheckEvery && w.inner32 && w.inner32_key == key) {
                CK(cudaGraphLaunch(w.inner32, s));
                it += kCheckEvery;
            } else {
                // plain launches (also the first block, which prepares every
                // kernel before the block is captured)
                const int blk = std::min<int32_t>(kCheckEvery, max_inner - it);
                for (int j = 0; j < blk; ++j) {
                    st = inner_iter(s);
                    if (st != SPMV_OK) return st;
                }
                it += blk;
                if (blk == kCheckEvery && (!w.inner32 || w.inner32_key != key)) {
                    if (w.inner32) { cudaGraphExecDestroy(w.inner32); w.inner32 = nullptr; }
                    st = ready_for_capture(A32, kF32, kF32);
                    if (st == SPMV_OK)
                        st = capture_graph([&](cudaStream_t cs) -> spmv_status {
                            for (int j = 0; j < kCheckEvery; ++j) {
                                const spmv_status s3 = inner_iter(cs);
                                if (s3 != SPMV_OK) return s3;
                            }
                            return SPMV_OK;
                        }, &w.inner32);
                    if (st != SPMV_OK) return st;
                    w.inner32_key = key;
                }
            }
            CK(cudaMemcpyAsync(w.host, w.sc + kScRho, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            rho = w.host[0];
        }
        inner_total += it;
        // update (FP64): x += ||r|| d
        CK(cg_axpy_64_32(x, w.d32, rnorm, n, s));
        ++outer;
    }
    if (stats) {
        stats[0] = outer;
        stats[1] = static_cast<double>(inner_total);
        stats[2] = relres;
        stats[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return converged ? SPMV_OK : SPMV_ERR_NOT_CONVERGED;
}

spmv_status spmv_validate_device(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, void *stream) {
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return SPMV_ERR_INVALID_ARG;
    if (!row_ptr || (nnz > 0 && !col_idx)) return SPMV_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *bad = nullptr;
    if (dmalloc(&bad, 1) != cudaSuccess) return SPMV_ERR_ALLOC;
    int32_t v = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, s);
    if (e == cudaSuccess) e = launch_validate(n_rows, n_cols, nnz, row_ptr, col_idx, bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bad);
    if (e != cudaSuccess) return SPMV_ERR_CUDA;
    return v ? SPMV_ERR_INVALID_INDEX : SPMV_OK;
}

spmv_status spmv_selftest_wait_timeout(spmv_handle h, int64_t limit_ns, void *stream) {
    if (!h || limit_ns < 1000 || limit_ns > static_cast<int64_t>(kWaitLimitNs)) return SPMV_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_wait_timeout(static_cast<uint64_t>(limit_ns), h->d_err, s));
    return spmv_check_device_error(h, stream);
}

spmv_status spmv_check_device_error(spmv_handle h, void *stream) {
    if (!h) return SPMV_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    CK(cudaMemcpyAsync(&v, h->d_err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (v != 0) {
        CK(cudaMemsetAsync(h->d_err, 0, 4, s));
        CK(cudaStreamSynchronize(s));
        return SPMV_ERR_TIMEOUT;
    }
    return SPMV_OK;
}

}  // extern "C"
