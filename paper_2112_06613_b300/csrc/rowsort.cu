// Per-row ordering of the CSR columns: each row's neighbours ascending (the rows of the
// adjacency matrix of Methods "Adjacency matrix", stored sparse).
//
// The write passes place a row's neighbours in arrival order (atomic cursors),
// so each row segment is sorted afterwards; the result is then independent of
// scheduling, i.e. bit-exact and deterministic. Values inside a CSR row are
// distinct node ids; candidate rows (l_max = 2) hold repeats, which every
// class below sorts too (the networks compare-exchange, the merges are stable).
//
//   len <= 8:           one lane, values in registers, Batcher's odd-even
//                       merge network for 8 (19 comparators); a warp takes 32
//                       consecutive rows at once.
//   9 .. 512:           one warp, values in registers (K = 1..16 per lane,
//                       network position lane * K + r), bitonic network:
//                       stages with partner distance < K exchange registers,
//                       longer ones exchange lanes by shuffle. K = 1 stops at
//                       the next power of two above the row length. Rows of
//                       65..256 and 257..512 are listed and sorted by their own
//                       kernels, so wide register arrays do not lower the
//                       occupancy of the kernel that sorts the many short rows.
//   513 .. 16384:       shared-memory bitonic network with the stages of
//                       partner distance < 256 in registers (warp chunks of 8
//                       values per lane): rows up to 4096 by a 256-thread group
//                       (four per block, named barriers), longer ones by the
//                       1024-thread block.
//   > 16384:            one block; 16384-value chunks sorted in shared memory,
//                       then pairwise merges through a scratch buffer where each
//                       value finds its output slot by binary search in the
//                       partner run.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace tcr {
namespace {

constexpr int kLaneMax = 8;
constexpr int kShortMax = 64;
constexpr int kWideMax = 256;
static_assert(kSortWideMin == kShortMax + 1 && kSortMidMin == kWideMax + 1 && kSortBigMin == 2 * kWideMax + 1,
              "the classes a caller lists are the classes of the kernels below");
constexpr int kBlockThreads = 1024;
constexpr int kBlockCap = 16384;
constexpr int kSortWarps = 8;
constexpr int32_t kInf = 0x7fffffff;

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__device__ __forceinline__ void cmp_swap(int32_t& a, int32_t& b) {
    const int32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Sort len <= 8 values held by one thread (Batcher's odd-even merge sort, n = 8).
__device__ __forceinline__ void lane_sort8(int32_t* __restrict__ row, int len) {
    int32_t v[kLaneMax];
#pragma unroll
    for (int t = 0; t < kLaneMax; ++t) v[t] = t < len ? row[t] : kInf;
    cmp_swap(v[0], v[1]); cmp_swap(v[2], v[3]); cmp_swap(v[4], v[5]); cmp_swap(v[6], v[7]);
    cmp_swap(v[0], v[2]); cmp_swap(v[1], v[3]); cmp_swap(v[4], v[6]); cmp_swap(v[5], v[7]);
    cmp_swap(v[1], v[2]); cmp_swap(v[5], v[6]);
    cmp_swap(v[0], v[4]); cmp_swap(v[1], v[5]); cmp_swap(v[2], v[6]); cmp_swap(v[3], v[7]);
    cmp_swap(v[2], v[4]); cmp_swap(v[3], v[5]);
    cmp_swap(v[1], v[2]); cmp_swap(v[3], v[4]); cmp_swap(v[5], v[6]);
#pragma unroll
    for (int t = 0; t < kLaneMax; ++t)
        if (t < len) row[t] = v[t];
}

// Sort one row of len <= 32 * K values held K per lane (see the file comment).
template <int K>
__device__ __forceinline__ void warp_sort_regs(int32_t* __restrict__ row, int len, int lane) {
    constexpr int P = 32 * K;
    int32_t v[K];
    // coalesced load; which value sits at which network position is irrelevant
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = r * 32 + lane;
        v[r] = e < len ? row[e] : kInf;
    }
    // K = 1: value e sits at position e, so positions >= len hold kInf and a
    // network over the next power of two above len sorts the row
    const int pmax = K == 1 ? next_pow2(len) : P;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
        if (k > pmax) break;
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    if ((r & j) == 0) {
                        const int r2 = r | j;
                        const bool up = ((lane * K + r) & k) == 0;
                        const int32_t a = v[r], b = v[r2];
                        const int32_t mn = min(a, b), mx = max(a, b);
                        v[r] = up ? mn : mx;
                        v[r2] = up ? mx : mn;
                    }
                }
            } else {
                const int jl = j / K;
                const bool lower = (lane & jl) == 0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int32_t p = __shfl_xor_sync(kFull, v[r], jl);
                    const bool up = ((lane * K + r) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = lane * K + r;
        if (e < len) row[e] = v[r];
    }
}

// Bitonic stages on one warp's chunk of kChunkVals values of a shared-memory
// network (positions c0 .. c0 + kChunkVals - 1, held K per lane at lane * K +
// r): for each merge size k from k_first to k_last, the stages with partner
// distance below the chunk size. Directions come from the global position, so
// chunks of one network cooperate without block barriers for those stages.
constexpr int kChunkK = 8;
constexpr int kChunkVals = 32 * kChunkK;

template <int J>
__device__ __forceinline__ void chunk_reg_stage(int32_t (&v)[kChunkK], int pos0, int k) {
#pragma unroll
    for (int r = 0; r < kChunkK; ++r) {
        if ((r & J) == 0) {
            const int r2 = r | J;
            const bool up = ((pos0 + r) & k) == 0;
            const int32_t a = v[r], b = v[r2];
            const int32_t mn = min(a, b), mx = max(a, b);
            v[r] = up ? mn : mx;
            v[r2] = up ? mx : mn;
        }
    }
}

__device__ __forceinline__ void chunk_stages(int32_t* s, int c0, int k_first, int k_last, int lane) {
    constexpr int K = kChunkK;
    static_assert(K == 8, "register stages are written out for 8 values per lane");
    int32_t v[K];
#pragma unroll
    for (int r = 0; r < K; ++r) v[r] = s[c0 + lane * K + r];
    for (int k = k_first; k <= k_last; k <<= 1) {
        for (int j = (k >> 1) < (kChunkVals >> 1) ? (k >> 1) : (kChunkVals >> 1); j > 0; j >>= 1) {
            if (j == 4) chunk_reg_stage<4>(v, c0 + lane * K, k);
            else if (j == 2) chunk_reg_stage<2>(v, c0 + lane * K, k);
            else if (j == 1) chunk_reg_stage<1>(v, c0 + lane * K, k);
            else {
                const int jl = j / K;
                const bool lower = (lane & jl) == 0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int32_t p = __shfl_xor_sync(kFull, v[r], jl);
                    const bool up = ((c0 + lane * K + r) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) s[c0 + lane * K + r] = v[r];
}

// Bitonic sort of s[0, P) (P a power of two, P >= kChunkVals) by nt threads
// (t = index among them, a whole number of warps) that meet at bar(): stages
// whose partners are a chunk or more apart go through shared memory with a
// barrier each; all shorter ones run inside the warps' chunks in registers.
template <typename Bar>
__device__ __forceinline__ void group_bitonic(int32_t* s, int P, int t, int nt, Bar bar) {
    const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
    const int nchunks = P / kChunkVals;
    for (int c = warp; c < nchunks; c += nwarps) chunk_stages(s, c * kChunkVals, 2, kChunkVals, lane);
    bar();
    for (int k = 2 * kChunkVals; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= kChunkVals; j >>= 1) {
            const int lj = __ffs(j) - 1;
            for (int i = t; i < (P >> 1); i += nt) {
                const int lo = ((i >> lj) << (lj + 1)) | (i & (j - 1));
                const int hi = lo + j;
                const bool up = (lo & k) == 0;
                const int32_t x = s[lo], y = s[hi];
                if ((x > y) == up) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            bar();
        }
        for (int c = warp; c < nchunks; c += nwarps) chunk_stages(s, c * kChunkVals, k, k, lane);
        bar();
    }
}

__device__ __forceinline__ void block_bitonic(int32_t* s, int P) {
    group_bitonic(s, P, threadIdx.x, kBlockThreads, [] __device__() { __syncthreads(); });
}

// Rows of at most 64 values; longer rows are listed for the kernels below
// (unless wide is null: the caller listed them). A warp takes 32 consecutive
// rows: each lane sorts its own row when it has at most 8 values, then the
// warp sorts the rows of 9..64 values one by one.
__global__ void __launch_bounds__(kSortWarps * 32)
k_sort_warp(const int64_t* __restrict__ off, int32_t* __restrict__ cols, int64_t n, int32_t* __restrict__ wide,
            int* __restrict__ nwide, int32_t* __restrict__ mid, int* __restrict__ nmid, int32_t* __restrict__ big,
            int* __restrict__ nbig) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kSortWarps + warp;
    const int64_t stride = (int64_t)gridDim.x * kSortWarps;
    for (int64_t r0 = gw * 32; r0 < n; r0 += stride * 32) {
        const int64_t r = r0 + lane;
        int64_t base = 0;
        int len = 0;
        if (r < n) {
            base = off[r];
            const int64_t len64 = off[r + 1] - base;
            len = len64 > (int64_t)kInf ? kInf : (int)len64;
        }
        if (len >= 2 && len <= kLaneMax) lane_sort8(cols + base, len);
        else if (!wide) {}  // the long rows were listed by the caller
        else if (len > 2 * kWideMax) big[atomicAdd(nbig, 1)] = (int32_t)r;  // few, long: a block each
        else if (len > kWideMax) mid[atomicAdd(nmid, 1)] = (int32_t)r;
        else if (len > kShortMax) wide[atomicAdd(nwide, 1)] = (int32_t)r;
        uint32_t todo = __ballot_sync(kFull, len > kLaneMax && len <= kShortMax);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t b = __shfl_sync(kFull, base, j);
            const int l = __shfl_sync(kFull, len, j);
            if (l <= 32) warp_sort_regs<1>(cols + b, l, lane);
            else warp_sort_regs<2>(cols + b, l, lane);
        }
    }
}

// Rows of 65..256 values (listed by k_sort_warp). Register budget for four
// blocks per SM (64 registers, no spill; 80 left three).
__global__ void __launch_bounds__(kSortWarps * 32, 4)
k_sort_warp_wide(const int64_t* __restrict__ off, int32_t* __restrict__ cols, const int32_t* __restrict__ rows,
                 const int* __restrict__ nrows) {
    dep_entry();  // launched dependent on the kernel before it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int count = *nrows;
    for (int64_t k = (int64_t)blockIdx.x * kSortWarps + warp; k < count; k += (int64_t)gridDim.x * kSortWarps) {
        const int64_t r = rows[k];
        const int64_t base = off[r];
        const int len = (int)(off[r + 1] - base);
        if (len <= 128) warp_sort_regs<4>(cols + base, len, lane);
        else warp_sort_regs<8>(cols + base, len, lane);
    }
}

// Rows of 257..512 values (K = 16), listed by k_sort_warp; a kernel of its own
// so that it gets the registers it needs (three blocks per SM: 80 registers
// with a 4-byte spill, against 128 and two blocks unbounded; measured faster).
template <int K>
__global__ void __launch_bounds__(kSortWarps * 32, 3)
k_sort_warp_mid(const int64_t* __restrict__ off, int32_t* __restrict__ cols, const int32_t* __restrict__ mid,
                const int* __restrict__ nmid) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int count = *nmid;
    for (int64_t k = (int64_t)blockIdx.x * kSortWarps + warp; k < count; k += (int64_t)gridDim.x * kSortWarps) {
        const int64_t r = mid[k];
        const int64_t base = off[r];
        const int len = (int)(off[r + 1] - base);
        warp_sort_regs<K>(cols + base, len, lane);
    }
}

// Rows of 513 .. kGroupCap values: four groups of 256 threads per block, each
// on its own row and shared-memory quarter (named barriers), so a row of ~1,000
// values does not leave most of a 1,024-thread block idle; longer rows: the
// whole block; rows above kBlockCap are listed for the chunked sort.
constexpr int kGroupThreads = 256;
constexpr int kGroups = kBlockThreads / kGroupThreads;
constexpr int kGroupCap = kBlockCap / kGroups;

__global__ void __launch_bounds__(kBlockThreads)
k_sort_block(const int64_t* __restrict__ off, int32_t* __restrict__ cols, const int32_t* __restrict__ rows,
             const int* __restrict__ nrows_ptr, int32_t* __restrict__ huge, int* __restrict__ nhuge) {
    extern __shared__ int32_t sbuf[];
    const int nrows = *nrows_ptr;
    const int g = threadIdx.x / kGroupThreads, tg = threadIdx.x % kGroupThreads;
    int32_t* gs = sbuf + g * kGroupCap;
    auto gbar = [g] __device__() { asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kGroupThreads) : "memory"); };
    for (int k = blockIdx.x * kGroups + g; k < nrows; k += gridDim.x * kGroups) {
        const int64_t r = rows[k];
        const int64_t base = off[r];
        const int64_t len = off[r + 1] - base;
        if (len > kGroupCap) continue;  // the whole block takes it below
        const int P = max(next_pow2((int)len), kChunkVals);
        for (int i = tg; i < P; i += kGroupThreads) gs[i] = i < len ? cols[base + i] : kInf;
        gbar();
        group_bitonic(gs, P, tg, kGroupThreads, gbar);
        for (int i = tg; i < len; i += kGroupThreads) cols[base + i] = gs[i];
        gbar();
    }
    __syncthreads();
    for (int k = blockIdx.x; k < nrows; k += gridDim.x) {
        const int64_t r = rows[k];
        const int64_t base = off[r];
        const int64_t len = off[r + 1] - base;
        if (len <= kGroupCap) continue;
        if (len > kBlockCap) {
            if (threadIdx.x == 0) huge[atomicAdd(nhuge, 1)] = (int32_t)r;
            continue;
        }
        const int P = max(next_pow2((int)len), kChunkVals);
        for (int i = threadIdx.x; i < P; i += kBlockThreads) sbuf[i] = i < len ? cols[base + i] : kInf;
        __syncthreads();
        block_bitonic(sbuf, P);
        for (int i = threadIdx.x; i < len; i += kBlockThreads) cols[base + i] = sbuf[i];
        __syncthreads();
    }
}

// Sort each kBlockCap chunk of one huge row in place (one block per chunk).
__global__ void __launch_bounds__(kBlockThreads)
k_sort_chunks(int32_t* __restrict__ v, int64_t len) {
    extern __shared__ int32_t sbuf[];
    const int64_t c0 = (int64_t)blockIdx.x * kBlockCap;
    const int64_t cl = (len - c0) < (int64_t)kBlockCap ? (len - c0) : (int64_t)kBlockCap;
    const int P = max(next_pow2((int)cl), kChunkVals);
    for (int i = threadIdx.x; i < P; i += kBlockThreads) sbuf[i] = i < cl ? v[c0 + i] : kInf;
    __syncthreads();
    block_bitonic(sbuf, P);
    for (int i = threadIdx.x; i < cl; i += kBlockThreads) v[c0 + i] = sbuf[i];
}

// Merge adjacent sorted runs of length `run` from src into dst. Each value's
// slot is its rank in its own run plus its rank in the partner run, counted
// stably so that repeated values (candidate rows hold repeats) get distinct
// slots: a value of the first run counts the partner's values below it, a
// value of the second run the partner's values at or below it.
__global__ void k_merge_runs(const int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t len, int64_t run) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pair = i / (2 * run);
        const int64_t a0 = pair * 2 * run;
        const int64_t a1 = min(a0 + run, len);
        const int64_t b0 = a1;
        const int64_t b1 = min(a0 + 2 * run, len);
        const int32_t x = src[i];
        const bool in_a = i < a1;
        int64_t lo = in_a ? b0 : a0, hi = in_a ? b1 : a1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (src[mid] < x || (!in_a && src[mid] == x)) lo = mid + 1; else hi = mid;
        }
        const int64_t rank_partner = lo - (in_a ? b0 : a0);
        const int64_t rank_own = i - (in_a ? a0 : b0);
        dst[a0 + rank_own + rank_partner] = x;
    }
}

}  // namespace

namespace {

// The long classes listed in advance: 65..256 on the first side stream,
// 257..512 then the block class on the second, the short-row kernel on s, all
// started together; s waits for both side streams at the end.
tcrnet_status sort_rows_listed(const int64_t* off, int32_t* cols, int64_t n, cudaStream_t s, int num_sms,
                               int64_t max_len, const SortClasses& pre, const SideStream* side, int32_t* huge_list,
                               int* nhuge) {
    const bool run_wide = max_len < 0 || max_len >= kSortWideMin;
    const bool run_mid = max_len < 0 || max_len >= kSortMidMin;
    const bool run_block = max_len < 0 || max_len >= kSortBigMin;
    TCR_CUDA(cudaEventRecord(side->ev[4], s));
    TCR_CUDA(cudaStreamWaitEvent(side->stream, side->ev[4], 0));
    TCR_CUDA(cudaStreamWaitEvent(side->stream2, side->ev[4], 0));
    if (run_wide) {
        k_sort_warp_wide<<<num_sms * 8, kSortWarps * 32, 0, side->stream>>>(off, cols, pre.wide, pre.counts);
        TCR_LAUNCH_CHECK();
    }
    if (run_mid) {
        k_sort_warp_mid<16><<<num_sms * 4, kSortWarps * 32, 0, side->stream2>>>(off, cols, pre.mid, pre.counts + 1);
        TCR_LAUNCH_CHECK();
    }
    if (run_block) {
        const size_t smem = sizeof(int32_t) * kBlockCap;
        k_sort_block<<<num_sms * 2, kBlockThreads, smem, side->stream2>>>(off, cols, pre.big, pre.counts + 2,
                                                                            huge_list, nhuge);
        TCR_LAUNCH_CHECK();
    }
    // the short rows last: the long classes' kernels take longer, so they are
    // queued first and this one fills the SMs they leave
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 32 * kSortWarps), (int64_t)num_sms * 16);
    k_sort_warp<<<(unsigned)blocks, kSortWarps * 32, 0, s>>>(off, cols, n, nullptr, nullptr, nullptr, nullptr,
                                                               nullptr, nullptr);
    TCR_LAUNCH_CHECK();
    TCR_CUDA(cudaEventRecord(side->ev[5], side->stream));
    TCR_CUDA(cudaEventRecord(side->ev[7], side->stream2));
    TCR_CUDA(cudaStreamWaitEvent(s, side->ev[5], 0));
    TCR_CUDA(cudaStreamWaitEvent(s, side->ev[7], 0));
    return TCRNET_OK;
}

}  // namespace

tcrnet_status sort_rows(const int64_t* off, int32_t* cols, int64_t n, cudaStream_t s, int num_sms, int64_t max_len,
                        const SortClasses* pre) {
    if (n <= 0) return TCRNET_OK;
    // lists: [0, n) rows of 257..512, [n, 2n) rows above 512, [2n, 3n) rows
    // above kBlockCap, [3n, 4n) rows of 65..256; counts in the same order
    DevBuf lists, counts;
    TCR_CHECK(lists.alloc(sizeof(int32_t) * 4 * n, s));
    int* cnt = pre ? pre->zeroed4 : nullptr;  // a caller's zeroed counters save a memset
    if (!cnt) {
        TCR_CHECK(counts.alloc(sizeof(int) * 4, s));
        TCR_CUDA(cudaMemsetAsync(counts.as<void>(), 0, sizeof(int) * 4, s));
        cnt = counts.as<int>();
    }
    int32_t* mid = lists.as<int32_t>();
    int32_t* big = mid + n;
    int32_t* huge_list = big + n;
    int32_t* wide = huge_list + n;
    const bool known = max_len >= 0;  // a known bound skips the kernels of longer classes
    const bool run_mid = !known || max_len > kWideMax;
    const bool run_block = !known || max_len > 2 * kWideMax;
    if (run_block) {
        const size_t smem = sizeof(int32_t) * kBlockCap;
        TCR_CUDA(cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TCR_CUDA(cudaFuncSetAttribute(k_sort_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const SideStream* lside = pre ? leased_side_stream() : nullptr;
    if (lside) {
        TCR_CHECK(sort_rows_listed(off, cols, n, s, num_sms, max_len, *pre, lside, huge_list, cnt + 2));
    } else {
        const int64_t blocks = std::min<int64_t>(ceil_div(n, 32 * kSortWarps), (int64_t)num_sms * 16);
        k_sort_warp<<<(unsigned)blocks, kSortWarps * 32, 0, s>>>(off, cols, n, wide, cnt + 3, mid, cnt, big, cnt + 1);
        TCR_LAUNCH_CHECK();
        // The classes are disjoint rows: rows above 256 are sorted on the second
        // stream of the workspace lease while this stream sorts 65..256.
        const SideStream* side = (run_mid || run_block) ? leased_side_stream() : nullptr;
        cudaStream_t s2 = s;
        if (side) {
            TCR_CUDA(cudaEventRecord(side->ev[4], s));
            TCR_CUDA(cudaStreamWaitEvent(side->stream, side->ev[4], 0));
            s2 = side->stream;
        }
        if (!known || max_len > kShortMax) {
            TCR_CUDA(launch_dependent(k_sort_warp_wide, dim3(num_sms * 8), dim3(kSortWarps * 32), 0, s, off, cols,
                                      wide, cnt + 3));
            note_launch();
        }
        if (run_mid) {
            k_sort_warp_mid<16><<<num_sms * 4, kSortWarps * 32, 0, s2>>>(off, cols, mid, cnt);
            TCR_LAUNCH_CHECK();
        }
        if (run_block) {
            const size_t smem = sizeof(int32_t) * kBlockCap;
            k_sort_block<<<num_sms * 2, kBlockThreads, smem, s2>>>(off, cols, big, cnt + 1, huge_list, cnt + 2);
            TCR_LAUNCH_CHECK();
        }
        if (side) {  // join the second stream back before anything reads the rows
            TCR_CUDA(cudaEventRecord(side->ev[5], s2));
            TCR_CUDA(cudaStreamWaitEvent(s, side->ev[5], 0));
        }
    }
    if (!run_block || (known && max_len <= kBlockCap)) return TCRNET_OK;  // no row can be listed as huge
    const size_t smem = sizeof(int32_t) * kBlockCap;
    int h_huge = 0;
    {
        const void* src[1] = {cnt + 2};
        void* dst[1] = {&h_huge};
        const size_t bytes[1] = {sizeof(int)};
        TCR_CHECK(read_back(s, 1, src, dst, bytes));
    }
    if (h_huge == 0) return TCRNET_OK;
    // Rare: rows longer than one shared-memory block.
    std::vector<int32_t> huge(h_huge);
    TCR_CUDA(cudaMemcpyAsync(huge.data(), huge_list, sizeof(int32_t) * huge.size(), cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> hoff(2);
    TCR_CUDA(cudaStreamSynchronize(s));
    for (int32_t r : huge) {
        TCR_CUDA(cudaMemcpyAsync(hoff.data(), off + r, sizeof(int64_t) * 2, cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        const int64_t len = hoff[1] - hoff[0];
        int32_t* v = cols + hoff[0];
        k_sort_chunks<<<(unsigned)ceil_div(len, kBlockCap), kBlockThreads, smem, s>>>(v, len);
        TCR_LAUNCH_CHECK();
        DevBuf tmp;
        TCR_CHECK(tmp.alloc(sizeof(int32_t) * len, s));
        int32_t* src = v;
        int32_t* dst = tmp.as<int32_t>();
        for (int64_t run = kBlockCap; run < len; run *= 2) {
            k_merge_runs<<<(unsigned)std::min<int64_t>(ceil_div(len, 256), 65535), 256, 0, s>>>(src, dst, len, run);
            TCR_LAUNCH_CHECK();
            std::swap(src, dst);
        }
        if (src != v) TCR_CUDA(cudaMemcpyAsync(v, src, sizeof(int32_t) * len, cudaMemcpyDeviceToDevice, s));
    }
    return TCRNET_OK;
}

}  // namespace tcr
