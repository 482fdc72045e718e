// All-pairs test for l_max >= 2: bit-parallel Levenshtein distance.
//
// For l_max >= 2 the closed forms of tile.cu do not apply; the distance is
// computed (Methods "Levenshtein distance", Eq. levenshtein) with the
// bit-vector formulation of the dynamic programme by Myers (1999), in the
// global-distance form described by Hyyrö (2001): the column of the DP table is
// held as vertical difference bits VP/VN (+1 / -1 between consecutive rows);
// one text character updates the whole column with a dozen word operations.
// Pattern = the column string b (its per-letter position masks Peq[c] are built
// once per stage in shared memory), text = the row string a. Initial column
// D[i][0] = i (all +1), score = D[m][0] = m; each step shifts the horizontal
// differences up by one row with a +1 entering at row 0 (D[0][j] = j), and the
// score follows the last row. lev <= l_max is then score <= l_max. Only bucket
// pairs with |len a - len b| <= l_max are visited (lev >= |len a - len b|).
//
// Strings are at most 48 long, so one 64-bit word holds a column; bucket pairs
// whose column strings have at most 32 letters (most CDR3s) run the same
// recurrence on 32-bit words, half the integer work per step. One row string
// per thread (256 rows per item), columns staged 256 at a time.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace tcr {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;
constexpr int kColBlock = 2048;
constexpr int kLetters = 20;

struct DpItem {
    int32_t a0, a1, b0, b1;
    int32_t La, Lb;
    int32_t diag;  // same bucket: only column position > row position
    int32_t pad;
};

struct DpArgs {
    const DpItem* items;
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
    int2* pairs;  // count pass: hits kept for the scatter (null: none)
    unsigned long long* pcur;
    int64_t pcap;
};

template <typename Word>
struct DpSmem {
    Word peq[kChunk][kLetters];
    int32_t id[kChunk];
    int item;
};

// lev(a, b) by the bit-vector recurrence; peq = position masks of b (length
// 1 <= Lb <= bits of Word). Bits above Lb - 1 never reach the ones below
// (carries and shifts move up only), so they need no masking.
template <typename Word>
__device__ __forceinline__ int myers_distance(const Word* __restrict__ peq, int Lb, const Canon& a, int La) {
    Word vp = ~Word(0), vn = Word(0);
    const Word top = Word(1) << (Lb - 1);
    int score = Lb;
#pragma unroll
    for (int j = 0; j < kMaxLen; ++j) {
        if (j < La) {
            const uint32_t c = (uint32_t)(a.w[j / kCodesPerWord] >> (5 * (j % kCodesPerWord))) & 31u;
            const Word eq = peq[c - 1];
            const Word xv = eq | vn;
            const Word xh = (((eq & vp) + vp) ^ vp) | eq;
            Word hp = vn | ~(xh | vp);
            Word hn = vp & xh;
            score += (hp & top) ? 1 : 0;
            score -= (hn & top) ? 1 : 0;
            hp = (hp << 1) | Word(1);
            hn = hn << 1;
            vp = hn | ~(xv | hp);
            vn = hp & xv;
        }
    }
    return score;
}

// Two columns against one row at once: two independent recurrences in one loop
// over the row's letters, so each step has two dependency chains to overlap.
template <typename Word>
__device__ __forceinline__ void myers_distance2(const Word* __restrict__ peq0, const Word* __restrict__ peq1, int Lb,
                                                const Canon& a, int La, int& d0, int& d1) {
    Word vp0 = ~Word(0), vn0 = Word(0), vp1 = ~Word(0), vn1 = Word(0);
    const Word top = Word(1) << (Lb - 1);
    int s0 = Lb, s1 = Lb;
#pragma unroll
    for (int j = 0; j < kMaxLen; ++j) {
        if (j < La) {
            const uint32_t c = (uint32_t)(a.w[j / kCodesPerWord] >> (5 * (j % kCodesPerWord))) & 31u;
            const Word e0 = peq0[c - 1], e1 = peq1[c - 1];
            const Word xv0 = e0 | vn0, xv1 = e1 | vn1;
            const Word xh0 = (((e0 & vp0) + vp0) ^ vp0) | e0;
            const Word xh1 = (((e1 & vp1) + vp1) ^ vp1) | e1;
            Word hp0 = vn0 | ~(xh0 | vp0), hp1 = vn1 | ~(xh1 | vp1);
            Word hn0 = vp0 & xh0, hn1 = vp1 & xh1;
            s0 += ((hp0 & top) ? 1 : 0) - ((hn0 & top) ? 1 : 0);
            s1 += ((hp1 & top) ? 1 : 0) - ((hn1 & top) ? 1 : 0);
            hp0 = (hp0 << 1) | Word(1);
            hp1 = (hp1 << 1) | Word(1);
            hn0 <<= 1;
            hn1 <<= 1;
            vp0 = hn0 | ~(xv0 | hp0);
            vp1 = hn1 | ~(xv1 | hp1);
            vn0 = hp0 & xv0;
            vn1 = hp1 & xv1;
        }
    }
    d0 = s0;
    d1 = s1;
}

template <bool WRITE, typename Word>
__global__ void __launch_bounds__(kThreads) k_dp(DpArgs g) {
    __shared__ DpSmem<Word> sm;
    const int tid = threadIdx.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.item = atomicAdd(g.counter, 1);
        __syncthreads();
        const int i = sm.item;
        if (i >= g.nitems) break;
        const DpItem it = g.items[i];
        const int row = it.a0 + tid;
        const bool valid = row < it.a1;
        Canon a;
        a.w[0] = a.w[1] = a.w[2] = a.w[3] = 0;
        int32_t aid = -1;
        if (valid) {
            a = load_canon(g.rowc + row);
            aid = g.row_id[row];
        }
        int32_t cnt = 0;
        for (int c0 = it.b0; c0 < it.b1; c0 += kChunk) {
            __syncthreads();
            for (int t = tid; t < kChunk; t += kThreads) {
                const int pos = c0 + t;
                Word* pq = sm.peq[t];
#pragma unroll
                for (int c = 0; c < kLetters; ++c) pq[c] = Word(0);
                if (pos < it.b1) {
                    const Canon b = load_canon(g.colc + pos);
#pragma unroll
                    for (int k = 0; k < kMaxLen; ++k) {
                        if (k < it.Lb) {
                            const uint32_t c = (uint32_t)(b.w[k / kCodesPerWord] >> (5 * (k % kCodesPerWord))) & 31u;
                            pq[c - 1] |= Word(1) << k;
                        }
                    }
                    sm.id[t] = g.col_id[pos];
                } else {
                    sm.id[t] = -1;
                }
            }
            __syncthreads();
            const int nb = min(kChunk, it.b1 - c0);
            {
                // every lane runs the loop (rows past the item's end compute and
                // discard), so the count pass can keep its hits warp by warp
                for (int j2 = 0; j2 < nb; j2 += 2) {
                    const bool has1 = j2 + 1 < nb;
                    const bool use0 = valid && !(it.diag && c0 + j2 <= row);
                    const bool use1 = valid && has1 && !(it.diag && c0 + j2 + 1 <= row);
                    int dd[2] = {g.T + 1, g.T + 1};
                    if (use0 || use1)
                        myers_distance2<Word>(sm.peq[j2], sm.peq[has1 ? j2 + 1 : j2], it.Lb, a, it.La, dd[0], dd[1]);
                    if constexpr (!WRITE) {
                        if (g.pcur) {
                            const bool k0 = use0 && dd[0] <= g.T, k1 = use1 && dd[1] <= g.T;
                            warp_append_pairs(g.pcur, (int)k0 + (int)k1, [&](long long base) {
                                if (k0) {
                                    if (base < g.pcap) g.pairs[base] = make_int2(aid, sm.id[j2]);
                                    ++base;
                                }
                                if (k1 && base < g.pcap) g.pairs[base] = make_int2(aid, sm.id[j2 + 1]);
                            });
                        }
                    }
                    if (!use0 && !use1) continue;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                    const int jj = j2 + h;
                    if (!(h == 0 ? use0 : use1) || dd[h] > g.T) continue;
                    const int32_t bid = sm.id[jj];
                    if constexpr (!WRITE) {
                        ++cnt;
                        if (g.sym) atomicAdd(&g.count[bid], 1);
                    } else {
                        const int32_t sa = atomicAdd(&g.cursor[aid], 1);
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
            if (valid && cnt) atomicAdd(&g.count[aid], cnt);
        }
    }
}

void add_block(std::vector<DpItem>& v, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int La, int Lb, bool diag,
               int64_t& pairs) {
    if (r1 <= r0 || c1 <= c0) return;
    for (int64_t a = r0; a < r1; a += kThreads) {
        const int64_t a1 = std::min<int64_t>(a + kThreads, r1);
        for (int64_t b = c0; b < c1; b += kColBlock) {
            const int64_t b1 = std::min<int64_t>(b + kColBlock, c1);
            if (diag && b1 - 1 <= a) continue;  // every column <= every row
            v.push_back(DpItem{(int32_t)a, (int32_t)a1, (int32_t)b, (int32_t)b1, La, Lb,
                               (diag && b <= a1 - 1) ? 1 : 0, 0});
        }
    }
    pairs += diag ? (r1 - r0) * (r1 - r0 - 1) / 2 : (r1 - r0) * (c1 - c0);
}

}  // namespace

tcrnet_status dp_pass(const TileSide& rows, const TileSide& cols, bool sym, int threshold, bool write,
                      int32_t* count, const int64_t* off, int32_t* cursor, int32_t* cols_out, int64_t* pairs,
                      cudaStream_t s, int num_sms, const PairSink* sink) {
    std::vector<DpItem> items;
    int64_t np = 0;
    for (int La = 1; La <= kMaxLen; ++La) {
        const int64_t rs = rows.bucket_off[La], re = rows.bucket_off[La + 1];
        if (re <= rs) continue;
        if (sym) {
            add_block(items, rs, re, rs, re, La, La, true, np);
            for (int d = 1; d <= threshold && La + d <= kMaxLen; ++d)
                add_block(items, rs, re, cols.bucket_off[La + d], cols.bucket_off[La + d + 1], La, La + d, false, np);
        } else {
            for (int Lb = std::max(1, La - threshold); Lb <= std::min(kMaxLen, La + threshold); ++Lb)
                add_block(items, rs, re, cols.bucket_off[Lb], cols.bucket_off[Lb + 1], La, Lb, false, np);
        }
    }
    if (pairs) *pairs = np;
    if (items.empty()) return TCRNET_OK;
    // column strings of <= 32 letters first (32-bit words), then the rest;
    // heaviest items first within each group
    std::stable_sort(items.begin(), items.end(), [](const DpItem& x, const DpItem& y) {
        const bool nx = x.Lb <= 32, ny = y.Lb <= 32;
        if (nx != ny) return nx;
        return (int64_t)(x.a1 - x.a0) * (x.b1 - x.b0) * x.La > (int64_t)(y.a1 - y.a0) * (y.b1 - y.b0) * y.La;
    });
    const int n_narrow = (int)(std::partition_point(items.begin(), items.end(),
                                                    [](const DpItem& x) { return x.Lb <= 32; }) -
                               items.begin());
    const int n_wide = (int)items.size() - n_narrow;
    DevBuf d_items, d_counter;
    TCR_CHECK(d_items.alloc(sizeof(DpItem) * items.size(), s));
    TCR_CHECK(d_counter.alloc(sizeof(int) * 3, s));  // [0] narrow items taken, [1] error, [2] wide items taken
    TCR_CUDA(cudaMemcpyAsync(d_items.as<void>(), items.data(), sizeof(DpItem) * items.size(),
                             cudaMemcpyHostToDevice, s));
    TCR_CUDA(cudaMemsetAsync(d_counter.as<void>(), 0, sizeof(int) * 3, s));
    auto launch = [&](auto kernel, const DpItem* list, int nitems, int* counter) -> tcrnet_status {
        if (nitems == 0) return TCRNET_OK;
        const bool keep = !write && sink && sink->pairs;
        DpArgs g{list, nitems, counter, rows.canon, rows.id, cols.canon, cols.id,
                 count, off, cursor, cols_out, d_counter.as<int>() + 1, sym ? 1 : 0, threshold,
                 keep ? sink->pairs : nullptr, keep ? sink->cursor : nullptr, keep ? sink->cap : 0};
        int per_sm = 0;
        TCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
        const int grid = (int)std::min<int64_t>((int64_t)nitems, (int64_t)num_sms * std::max(per_sm, 1));
        kernel<<<grid, kThreads, 0, s>>>(g);
        TCR_LAUNCH_CHECK();
        return TCRNET_OK;
    };
    const DpItem* d0 = d_items.as<DpItem>();
    if (write) {
        TCR_CHECK(launch(k_dp<true, uint32_t>, d0, n_narrow, d_counter.as<int>()));
        TCR_CHECK(launch(k_dp<true, uint64_t>, d0 + n_narrow, n_wide, d_counter.as<int>() + 2));
    } else {
        TCR_CHECK(launch(k_dp<false, uint32_t>, d0, n_narrow, d_counter.as<int>()));
        TCR_CHECK(launch(k_dp<false, uint64_t>, d0 + n_narrow, n_wide, d_counter.as<int>() + 2));
    }
    if (write) {
        int h_err = 0;
        TCR_CUDA(cudaMemcpyAsync(&h_err, d_counter.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        if (h_err) return TCRNET_EDEVICE;
    }
    return TCRNET_OK;
}

}  // namespace tcr
