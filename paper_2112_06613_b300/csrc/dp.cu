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
// Strings are at most 48 long, so one 64-bit word holds a column. One row string
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
};

struct DpSmem {
    uint64_t peq[kChunk][kLetters];
    int32_t id[kChunk];
    int item;
};

// lev(a, b) by the bit-vector recurrence; peq = position masks of b (length Lb >= 1).
__device__ __forceinline__ int myers_distance(const uint64_t* __restrict__ peq, int Lb, const Canon& a, int La) {
    uint64_t vp = ~0ull, vn = 0ull;
    const uint64_t top = 1ull << (Lb - 1);
    int score = Lb;
#pragma unroll
    for (int j = 0; j < kMaxLen; ++j) {
        if (j < La) {
            const uint32_t c = (uint32_t)(a.w[j / kCodesPerWord] >> (5 * (j % kCodesPerWord))) & 31u;
            const uint64_t eq = peq[c - 1];
            const uint64_t xv = eq | vn;
            const uint64_t xh = (((eq & vp) + vp) ^ vp) | eq;
            uint64_t hp = vn | ~(xh | vp);
            uint64_t hn = vp & xh;
            score += (hp & top) ? 1 : 0;
            score -= (hn & top) ? 1 : 0;
            hp = (hp << 1) | 1ull;
            hn = hn << 1;
            vp = hn | ~(xv | hp);
            vn = hp & xv;
        }
    }
    return score;
}

template <bool WRITE>
__global__ void __launch_bounds__(kThreads) k_dp(DpArgs g) {
    __shared__ DpSmem sm;
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
                uint64_t* pq = sm.peq[t];
#pragma unroll
                for (int c = 0; c < kLetters; ++c) pq[c] = 0ull;
                if (pos < it.b1) {
                    const Canon b = load_canon(g.colc + pos);
#pragma unroll
                    for (int k = 0; k < kMaxLen; ++k) {
                        if (k < it.Lb) {
                            const uint32_t c = (uint32_t)(b.w[k / kCodesPerWord] >> (5 * (k % kCodesPerWord))) & 31u;
                            pq[c - 1] |= 1ull << k;
                        }
                    }
                    sm.id[t] = g.col_id[pos];
                } else {
                    sm.id[t] = -1;
                }
            }
            __syncthreads();
            const int nb = min(kChunk, it.b1 - c0);
            if (valid) {
                for (int jj = 0; jj < nb; ++jj) {
                    if (it.diag && c0 + jj <= row) continue;
                    const int d = myers_distance(sm.peq[jj], it.Lb, a, it.La);
                    if (d > g.T) continue;
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
                      cudaStream_t s, int num_sms) {
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
    std::stable_sort(items.begin(), items.end(), [](const DpItem& x, const DpItem& y) {
        return (int64_t)(x.a1 - x.a0) * (x.b1 - x.b0) * x.La > (int64_t)(y.a1 - y.a0) * (y.b1 - y.b0) * y.La;
    });
    DevBuf d_items, d_counter;
    TCR_CHECK(d_items.alloc(sizeof(DpItem) * items.size(), s));
    TCR_CHECK(d_counter.alloc(sizeof(int) * 2, s));
    TCR_CUDA(cudaMemcpyAsync(d_items.as<void>(), items.data(), sizeof(DpItem) * items.size(),
                             cudaMemcpyHostToDevice, s));
    TCR_CUDA(cudaMemsetAsync(d_counter.as<void>(), 0, sizeof(int) * 2, s));
    DpArgs g{d_items.as<DpItem>(), (int)items.size(), d_counter.as<int>(), rows.canon, rows.id, cols.canon, cols.id,
             count, off, cursor, cols_out, d_counter.as<int>() + 1, sym ? 1 : 0, threshold};
    int per_sm = 0;
    if (write) {
        TCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dp<true>, kThreads, 0));
    } else {
        TCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dp<false>, kThreads, 0));
    }
    const int grid = (int)std::min<int64_t>((int64_t)items.size(), (int64_t)num_sms * std::max(per_sm, 1));
    if (write)
        k_dp<true><<<grid, kThreads, 0, s>>>(g);
    else
        k_dp<false><<<grid, kThreads, 0, s>>>(g);
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
