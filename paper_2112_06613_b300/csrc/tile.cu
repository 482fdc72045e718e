// All-pairs tile kernel over length buckets (Methods "GPU-based network generation":
// every pair tested, the matrix in tiles; a count pass, then a write pass).
//
// The paper fills the adjacency matrix block by block on the GPU, one
// Levenshtein dynamic programme per entry with an early abort (Methods
// "GPU-based network generation", Listing 1). For l_max <= 1 the distance test
// has a closed form that needs no DP:
//   equal lengths:   lev <= 1  <=>  at most one mismatching position (Hamming);
//   lengths L, L+1:  lev <= 1  <=>  the shorter string a equals the longer b
//                    with one character deleted  <=>  LCP(a, b) + LCS(a, b) >= L,
//                    i.e. the first mismatch f1 of a vs b lies after the last
//                    mismatch l2 of a vs b shifted down by one position.
//   lengths differing by 2 or more: never (lev >= |len a - len b|).
// l_max = 0 is equality.
//
// Word layout inside the kernel ("interleaved", W 32-bit words per string,
// 6 five-bit fields per word, bits 30-31 unused): position k lives in word
// k % W, field k / W. XOR of two words marks mismatching fields; a carry trick
// sets bit 4 of each non-zero field: t = (((x | HI) - LOW) | x) & HI. Shifting
// word w's result right by (4 - w) puts position W*f + w at bit 5*f + w, so the
// OR over the W words is a 32-bit mask with one bit per position, in position
// order (W <= 5, strings up to 30; for W <= 3 the shift is a left shift done
// as a multiply-add, see posmask_fma). Then
//   equal length: adjacent <=> (m & (m - 1)) == 0;
//   L vs L+1:     m1 = mask(a, b), m2 = mask(a, b >> one position);
//                 adjacent <=> (m2 & (m1 | -m1)) == 0  (no m2 bit at or above
//                 the lowest m1 bit). m1 != 0 always: position L holds pad in a
//                 and a letter in b.
// Longer strings (W = 6..8, up to 48) build a 64-bit position mask field by
// field: the same tests, slower, and absent from the synthetic workloads.
//
// Work decomposition: a persistent grid walks a list of items. An item is a
// block of up to 256*R row strings (held in registers, R per thread) against a
// block of column strings staged through shared memory in chunks of 512 (each
// thread reads the same column word: a broadcast). Items of the (L, L) bucket
// are restricted to the upper triangle; items that touch the diagonal test
// column position > row position per pair.
//
// Count pass: per-row hits accumulate in registers; hits on the column string
// are added with one atomic per hitting lane (hits are rare: ~3e-4 of pairs).
// Write pass: each hit takes a slot in its row with an atomic cursor and writes
// the neighbour's input index; rows are sorted afterwards (rowsort.cu).
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace tcr {
namespace {

constexpr uint32_t kHI = 0x21084210u;   // bit 4 of fields 0..5
constexpr uint32_t kLOW = 0x02108421u;  // bit 0 of fields 0..5
constexpr uint32_t kRowPad = 0x3fffffffu;  // every field 31: matches no letter, no pad
constexpr uint32_t kColPad = 0x3def7bdeu;  // every field 30: matches neither letters nor 31

constexpr int kThreads = 256;
constexpr int kChunk = 512;      // column strings per shared-memory stage
constexpr int kColBlock = 2048;  // column strings per item

enum Kind : int32_t { kRect = 0, kDiag = 1, kShortRows = 2, kLongRows = 3 };

struct Item {
    int32_t a0, a1;  // row positions (row-side bucket order)
    int32_t b0, b1;  // column positions (column-side bucket order)
    int32_t W, kind;
};

template <int W>
struct Rows {
    static constexpr int R = W <= 5 ? 8 : 4;
};

template <int W>
using Mask = typename std::conditional<(W <= 5), uint32_t, uint64_t>::type;

// Interleave a canonical string into W words, starting at position OFF
// (OFF = 1 yields the string shifted down by one position).
template <int W, int OFF>
__device__ __forceinline__ void interleave(const Canon& c, uint32_t (&out)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) out[w] = 0;
#pragma unroll
    for (int k = 0; k < 6 * W; ++k) {
        const int src = k + OFF;
        if (src < kMaxLen) {
            const uint32_t code = (uint32_t)(c.w[src / kCodesPerWord] >> (5 * (src % kCodesPerWord))) & 31u;
            out[k % W] |= code << (5 * (k / W));
        }
    }
}

__device__ __forceinline__ uint32_t field_mismatch(uint32_t x) {
    return (((x | kHI) - kLOW) | x) & kHI;
}

// x * m + c on the integer multiply-add unit (the FMA pipe), leaving the
// ALU pipe to the logic operations.
__device__ __forceinline__ uint32_t imad(uint32_t x, uint32_t m, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(m), "r"(c));
    return r;
}

// Up to three words (strings of at most 18): the same mask with position
// W*f + w at bit 5*f + 4 + w (still increasing with the position), built with
// three logic operations and two multiply-adds per word. The multipliers carry
// an extra 2^31 term so they are not powers of two; it only reaches bit 31,
// which is masked off (y) or never set (t has no bit 0).
template <int W>
__device__ __forceinline__ uint32_t posmask_fma(const uint32_t (&a)[W], const uint32_t (&b)[W]) {
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t x = a[w] ^ b[w];
        const uint32_t z = x | kHI;
        const uint32_t y = imad(z, 0x80000001u, 0u - kLOW);  // z - LOW
        const uint32_t t = (y | x) & kHI;
        m = imad(t, (1u << w) | 0x80000000u, m);  // m + (t << w)
    }
    return m;
}

template <int W>
__device__ __forceinline__ Mask<W> posmask(const uint32_t (&a)[W], const uint32_t (&b)[W]) {
    if constexpr (W <= 3) {
        return posmask_fma<W>(a, b);
    } else if constexpr (W <= 5) {
        uint32_t m = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) m |= field_mismatch(a[w] ^ b[w]) >> (4 - w);
        return m;
    } else {
        uint64_t m = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t t = field_mismatch(a[w] ^ b[w]);
#pragma unroll
            for (int f = 0; f < 6; ++f) m |= (uint64_t)((t >> (5 * f + 4)) & 1u) << (W * f + w);
        }
        return m;
    }
}

template <int W>
__device__ __forceinline__ bool same_len_adjacent(const uint32_t (&a)[W], const uint32_t (&b)[W], int T) {
    const Mask<W> m = posmask<W>(a, b);
    if constexpr (W <= 3) {
        // m - 1 as a multiply-add (bit 0 of m is never set, so the 2^31 term cancels out of the test)
        return T == 0 ? (m == 0) : ((m & imad(m, 0x80000001u, 0xffffffffu)) == 0);
    } else {
        return T == 0 ? (m == 0) : ((m & (m - 1)) == 0);
    }
}

// a shorter (length L), b longer (L + 1), bs = b shifted down by one position.
template <int W>
__device__ __forceinline__ bool indel_adjacent(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                               const uint32_t (&bs)[W]) {
    const Mask<W> m1 = posmask<W>(a, b);
    const Mask<W> m2 = posmask<W>(a, bs);
    if constexpr (W <= 3) {
        return (m2 & (m1 | imad(m1, 0xffffffffu, 0u))) == 0;  // -m1 on the multiply-add unit
    } else {
        return (m2 & (m1 | (Mask<W>)(Mask<W>(0) - m1))) == 0;
    }
}

template <int W>
__device__ __forceinline__ void load_words(const uint32_t* p, uint32_t (&o)[W]) {
    if constexpr (W <= 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint32_t t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] = t[w];
    } else {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint4 u = *reinterpret_cast<const uint4*>(p + 4);
        const uint32_t t[8] = {v.x, v.y, v.z, v.w, u.x, u.y, u.z, u.w};
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] = t[w];
    }
}

constexpr int kHitBuf = 128;  // kept hits staged per warp and column chunk

struct Smem {
    uint32_t b[kChunk][8];   // column strings (W words, padded to 4 or 8)
    uint32_t bs[kChunk][8];  // column strings shifted by one position (kShortRows)
    int32_t id[kChunk];
    int item;
    int2 hits[kThreads / 32][kHitBuf];  // count pass: hits of the current chunk, per warp
    int nhits[kThreads / 32];
};

struct Args {
    const Item* items;
    int nitems;
    int* counter;
    const Canon* rowc;
    const int32_t* row_id;
    const Canon* colc;
    const int32_t* col_id;
    int32_t* count;
    const int64_t* off;
    int32_t* cursor;
    int32_t* out;
    int* err;
    int sym;
    int T;
    int2* pairs;                // count pass: hits kept for the scatter (null: none)
    unsigned long long* pcur;
    int64_t pcap;
};

template <int W, int KIND, bool WRITE>
__device__ __forceinline__ void process_item(const Args& g, const Item& it, Smem& sm) {
    constexpr int R = Rows<W>::R;
    constexpr int WP = W <= 4 ? 4 : 8;
    const int tid = threadIdx.x;
    uint32_t a[R][W];
    uint32_t as[R][W];  // rows shifted (kLongRows only)
    int32_t rid[R];
    int32_t rpos[R];
    int32_t rc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int pos = it.a0 + tid + kThreads * r;
        rpos[r] = pos;
        rc[r] = 0;
        if (pos < it.a1) {
            const Canon c = load_canon(g.rowc + pos);
            interleave<W, 0>(c, a[r]);
            if constexpr (KIND == kLongRows) interleave<W, 1>(c, as[r]);
            rid[r] = g.row_id[pos];
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                a[r][w] = kRowPad;
                as[r][w] = kRowPad;
            }
            rid[r] = -1;
        }
    }
    for (int c0 = it.b0; c0 < it.b1; c0 += kChunk) {
        __syncthreads();
        for (int t = tid; t < kChunk; t += kThreads) {
            const int pos = c0 + t;
            uint32_t bw[W], bsw[W];
            if (pos < it.b1) {
                const Canon c = load_canon(g.colc + pos);
                interleave<W, 0>(c, bw);
                if constexpr (KIND == kShortRows) interleave<W, 1>(c, bsw);
                sm.id[t] = g.col_id[pos];
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w) bw[w] = bsw[w] = kColPad;
                sm.id[t] = -1;
            }
#pragma unroll
            for (int w = 0; w < WP; ++w) {
                sm.b[t][w] = w < W ? bw[w] : 0u;
                if constexpr (KIND == kShortRows) sm.bs[t][w] = w < W ? bsw[w] : 0u;
            }
        }
        __syncthreads();
        const int nb = min(kChunk, it.b1 - c0);
        int lim[R];
        if constexpr (KIND == kDiag) {
#pragma unroll
            for (int r = 0; r < R; ++r) lim[r] = rpos[r] - c0;  // need jj > lim
        }
        for (int jj = 0; jj < nb; ++jj) {
            uint32_t b[W];
            load_words<W>(&sm.b[jj][0], b);
            uint32_t bs[W];
            if constexpr (KIND == kShortRows) load_words<W>(&sm.bs[jj][0], bs);
            unsigned hit = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                bool h;
                if constexpr (KIND == kShortRows) {
                    h = indel_adjacent<W>(a[r], b, bs);
                } else if constexpr (KIND == kLongRows) {
                    h = indel_adjacent<W>(b, a[r], as[r]);
                } else {
                    h = same_len_adjacent<W>(a[r], b, g.T);
                    if constexpr (KIND == kDiag) h = h && (jj > lim[r]);
                }
                hit |= (unsigned)h << r;
            }
            if (hit) {
                const int32_t bid = sm.id[jj];
                if constexpr (!WRITE) {
                    if (g.pcur) {  // keep the hits: staged per warp, moved out at the chunk's end
                        const int wq = tid >> 5;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if ((hit >> r) & 1u) {
                                const int slot = atomicAdd(&sm.nhits[wq], 1);
                                if (slot < kHitBuf) {
                                    sm.hits[wq][slot] = make_int2(rid[r], bid);
                                } else {
                                    const unsigned long long pos = atomicAdd(g.pcur, 1ull);
                                    if ((long long)pos < g.pcap) g.pairs[pos] = make_int2(rid[r], bid);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) rc[r] += (hit >> r) & 1u;
                    if (g.sym) atomicAdd(&g.count[bid], __popc(hit));
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if ((hit >> r) & 1u) {
                            const int32_t aid = rid[r];
                            const int32_t sa = atomicAdd(&g.cursor[aid], 1);
                            // slots beyond the counted row length would mean the
                            // passes disagree: flag instead of writing
                            if (g.off[aid] + sa < g.off[aid + 1]) g.out[g.off[aid] + sa] = bid;
                            else atomicExch(g.err, 1);
                            if (g.sym) {
                                const int32_t sb = atomicAdd(&g.cursor[bid], 1);
                                if (g.off[bid] + sb < g.off[bid + 1]) g.out[g.off[bid] + sb] = aid;
                                else atomicExch(g.err, 1);
                            }
                        }
                    }
                }
            }
        }
        if constexpr (!WRITE) {
            if (g.pcur) {  // move this warp's staged hits out: one cursor update
                __syncwarp();
                const int wq = tid >> 5, lane = tid & 31;
                const int k = min(sm.nhits[wq], kHitBuf);
                if (k > 0) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(g.pcur, (unsigned long long)k);
                    base = __shfl_sync(kFull, base, 0);
                    for (int t = lane; t < k; t += 32)
                        if ((long long)(base + t) < g.pcap) g.pairs[base + t] = sm.hits[wq][t];
                }
                __syncwarp();
                if (lane == 0) sm.nhits[wq] = 0;
                __syncwarp();
            }
        }
    }
    if constexpr (!WRITE) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (rc[r]) atomicAdd(&g.count[rid[r]], rc[r]);
    }
}

template <bool WRITE, int KIND>
__device__ __forceinline__ void dispatch_w(const Args& g, const Item& it, Smem& sm) {
    switch (it.W) {
        case 1: process_item<1, KIND, WRITE>(g, it, sm); break;
        case 2: process_item<2, KIND, WRITE>(g, it, sm); break;
        case 3: process_item<3, KIND, WRITE>(g, it, sm); break;
        case 4: process_item<4, KIND, WRITE>(g, it, sm); break;
        case 5: process_item<5, KIND, WRITE>(g, it, sm); break;
        case 6: process_item<6, KIND, WRITE>(g, it, sm); break;
        case 7: process_item<7, KIND, WRITE>(g, it, sm); break;
        default: process_item<8, KIND, WRITE>(g, it, sm); break;
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(kThreads, 2) k_tile(Args g) {
    __shared__ Smem sm;
    if (threadIdx.x < kThreads / 32) sm.nhits[threadIdx.x] = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm.item = atomicAdd(g.counter, 1);
        __syncthreads();
        const int i = sm.item;
        if (i >= g.nitems) break;
        const Item it = g.items[i];
        switch (it.kind) {
            case kRect: dispatch_w<WRITE, kRect>(g, it, sm); break;
            case kDiag: dispatch_w<WRITE, kDiag>(g, it, sm); break;
            case kShortRows: dispatch_w<WRITE, kShortRows>(g, it, sm); break;
            default: dispatch_w<WRITE, kLongRows>(g, it, sm); break;
        }
    }
}

int words_for(int len) { return (len + 5) / 6; }
int rows_per_item(int W) { return kThreads * (W <= 5 ? 8 : 4); }

// Row blocks x column blocks of one bucket pair.
void add_rect(std::vector<Item>& v, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int W, int kind, int64_t& pairs) {
    if (r1 <= r0 || c1 <= c0) return;
    const int rb = rows_per_item(W);
    for (int64_t a = r0; a < r1; a += rb)
        for (int64_t b = c0; b < c1; b += kColBlock)
            v.push_back(Item{(int32_t)a, (int32_t)std::min<int64_t>(a + rb, r1), (int32_t)b,
                             (int32_t)std::min<int64_t>(b + kColBlock, c1), W, kind});
    pairs += (r1 - r0) * (c1 - c0);
}

// Upper triangle (column position > row position) of one bucket.
void add_triangle(std::vector<Item>& v, int64_t s, int64_t e, int W, int64_t& pairs) {
    if (e - s < 2) return;
    const int rb = rows_per_item(W);
    for (int64_t a = s; a < e; a += rb) {
        const int64_t a1 = std::min<int64_t>(a + rb, e);
        for (int64_t b = s; b < e; b += kColBlock) {
            const int64_t b1 = std::min<int64_t>(b + kColBlock, e);
            if (b1 - 1 <= a) continue;          // every column <= every row
            const int kind = (b > a1 - 1) ? kRect : kDiag;  // all columns > all rows: no check
            v.push_back(Item{(int32_t)a, (int32_t)a1, (int32_t)b, (int32_t)b1, W, kind});
        }
    }
    pairs += (e - s) * (e - s - 1) / 2;
}

}  // namespace

namespace {
__global__ void k_scatter_pairs(const int2* __restrict__ pairs, int64_t npairs, int sym,
                                const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                                int32_t* __restrict__ out, int* __restrict__ err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npairs;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = pairs[k];
        const int32_t sa = atomicAdd(&cursor[p.x], 1);
        if (off[p.x] + sa < off[p.x + 1]) out[off[p.x] + sa] = p.y;
        else atomicExch(err, 1);
        if (sym) {
            const int32_t sb = atomicAdd(&cursor[p.y], 1);
            if (off[p.y] + sb < off[p.y + 1]) out[off[p.y] + sb] = p.x;
            else atomicExch(err, 1);
        }
    }
}
}  // namespace

tcrnet_status scatter_pairs(const int2* pairs, int64_t npairs, bool sym, const int64_t* off, int32_t* cursor,
                            int32_t* cols_out, int* err, cudaStream_t s) {
    if (npairs <= 0) return TCRNET_OK;
    const int64_t blocks = std::min<int64_t>(ceil_div(npairs, 256), 148LL * 64);
    k_scatter_pairs<<<(unsigned)blocks, 256, 0, s>>>(pairs, npairs, sym ? 1 : 0, off, cursor, cols_out, err);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

tcrnet_status tile_pass(const TileSide& rows, const TileSide& cols, bool sym, int threshold, bool write,
                        int32_t* count, const int64_t* off, int32_t* cursor, int32_t* cols_out,
                        int64_t* pairs, cudaStream_t s, int num_sms, const PairSink* sink) {
    if (threshold >= 2)
        return dp_pass(rows, cols, sym, std::min(threshold, kMaxLen), write, count, off, cursor, cols_out, pairs, s,
                       num_sms, sink);
    std::vector<Item> items;
    int64_t np = 0;
    for (int L = 1; L <= kMaxLen; ++L) {
        const int64_t rs = rows.bucket_off[L], re = rows.bucket_off[L + 1];
        if (re <= rs) continue;
        if (sym) {
            add_triangle(items, rs, re, words_for(L), np);
            if (threshold >= 1 && L + 1 <= kMaxLen)
                add_rect(items, rs, re, cols.bucket_off[L + 1], cols.bucket_off[L + 2], words_for(L + 1),
                         kShortRows, np);
        } else {
            add_rect(items, rs, re, cols.bucket_off[L], cols.bucket_off[L + 1], words_for(L), kRect, np);
            if (threshold >= 1) {
                if (L + 1 <= kMaxLen)
                    add_rect(items, rs, re, cols.bucket_off[L + 1], cols.bucket_off[L + 2], words_for(L + 1),
                             kShortRows, np);
                if (L - 1 >= 1)
                    add_rect(items, rs, re, cols.bucket_off[L - 1], cols.bucket_off[L], words_for(L), kLongRows,
                             np);
            }
        }
    }
    if (pairs) *pairs = np;
    if (items.empty()) return TCRNET_OK;
    // Heaviest items first (more words, larger blocks) so the persistent grid ends evenly.
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        const int64_t cx = (int64_t)(x.a1 - x.a0) * (x.b1 - x.b0) * x.W * (x.kind >= kShortRows ? 2 : 1);
        const int64_t cy = (int64_t)(y.a1 - y.a0) * (y.b1 - y.b0) * y.W * (y.kind >= kShortRows ? 2 : 1);
        return cx > cy;
    });
    DevBuf d_items, d_counter;
    TCR_CHECK(d_items.alloc(sizeof(Item) * items.size(), s));
    TCR_CHECK(d_counter.alloc(sizeof(int) * 2, s));  // [0] item counter, [1] error flag
    TCR_CUDA(cudaMemcpyAsync(d_items.as<void>(), items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, s));
    TCR_CUDA(cudaMemsetAsync(d_counter.as<void>(), 0, sizeof(int) * 2, s));
    Args g;
    g.items = d_items.as<Item>();
    g.nitems = (int)items.size();
    g.counter = d_counter.as<int>();
    g.rowc = rows.canon;
    g.row_id = rows.id;
    g.colc = cols.canon;
    g.col_id = cols.id;
    g.count = count;
    g.off = off;
    g.cursor = cursor;
    g.out = cols_out;
    g.err = d_counter.as<int>() + 1;
    g.sym = sym ? 1 : 0;
    g.T = threshold;
    const bool keep = !write && sink && sink->pairs;
    g.pairs = keep ? sink->pairs : nullptr;
    g.pcur = keep ? sink->cursor : nullptr;
    g.pcap = keep ? sink->cap : 0;
    int per_sm = 0;
    if (write) {
        TCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<true>, kThreads, 0));
    } else {
        TCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<false>, kThreads, 0));
    }
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<int64_t>((int64_t)items.size(), (int64_t)num_sms * per_sm);
    if (write)
        k_tile<true><<<grid, kThreads, 0, s>>>(g);
    else
        k_tile<false><<<grid, kThreads, 0, s>>>(g);
    TCR_LAUNCH_CHECK();
    if (write) {
        int h_err = 0;
        TCR_CUDA(cudaMemcpyAsync(&h_err, g.err, sizeof(int), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        if (h_err) return TCRNET_EDEVICE;
    }
    return TCRNET_OK;
}

}  // namespace tcr
