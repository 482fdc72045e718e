// Deletion-neighbourhood method (hot-path step a7).
//
// The paper computes a Levenshtein DP for every pair of the adjacency matrix
// (Methods "GPU-based network generation"); its cost grows with N^2 while the
// network is sparse for small l_max (the same section notes TCR-NET is only
// efficient when edges are a small fraction of all pairs). For l_max <= 1 the
// neighbours of a string can instead be found by exact key matching on its
// one-deletion variants, in time proportional to the input plus the output:
//   equal length L: lev(a, b) <= 1 <=> a and b agree everywhere except
//     possibly at one position p <=> del_p(a) == del_p(b) for that p;
//   lengths L, L+1: lev(a, b) <= 1 <=> del_p(b) == a for some p.
// Duplicate strings are collapsed first (they are adjacent to each other and
// share every neighbour), so among distinct strings each equal-length pair
// matches at exactly one position (two positions would force a == b), and for
// the indel join only deletions at the first position of a run of equal
// letters are used (deleting any letter of a run gives the same string, and
// deletions from different runs give different strings), so every edge is
// found exactly once and no deduplication pass is needed.
//
// Pipeline:
//  1. dedup: open-addressing hash table of the packed strings (slot claimed by
//     atomicCAS, exact comparison on probe) -> distinct-string ids u,
//     multiplicities m_u, member lists M_u.
//  2. records: per distinct string one full-string record F (tag 63) and one
//     record per deletion position p (with a run-start flag), each a 32-bit
//     word (u << 7 | runstart << 6 | p); they are hash-partitioned by the
//     content they stand for (two passes: count, scatter).
//  3. join: one block per partition loads its records into shared memory,
//     keys each by (56-bit content hash | p), sorts (bitonic), checks that
//     equal hashes are equal contents (exact), and emits edges between
//     distinct strings: every pair inside a run of equal keys (equal length,
//     one substitution), and each run-start deletion record with the full
//     record of the same content (one indel). Count pass, exclusive scan,
//     write pass (a block prefix sum gives each thread its slots). Partitions
//     over capacity or with a hash collision take an exact quadratic fallback.
//  4. degrees: deg(i) = m_u - 1 + sum over distinct neighbours v of m_v.
//  5. fill: all members of u share one row layout (self clique first, then
//     one cursor per distinct string), then rows are sorted (rowsort.cu).
#include <algorithm>
#include <vector>

#include "deletion.cuh"

namespace tcr {
namespace {

constexpr int kThreads = 256;
constexpr int kCap = 2048;        // records per partition joined in shared memory
constexpr int kTargetPart = 256;  // mean records per partition
constexpr uint32_t kTagF = 63;    // position tag of a full-string record
constexpr int kHeavy = 32;        // m_u * m_v above this: a warp fills the edge

// 64-bit finaliser of MurmurHash3 (public domain).
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ uint64_t hash_canon(const Canon& c) {
    uint64_t h = 0x243f6a8885a308d3ULL;
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) h = fmix64(h ^ (c.w[w] + 0x9e3779b97f4a7c15ULL * (uint64_t)(w + 1)));
    return h;
}

__device__ __forceinline__ bool canon_eq(const Canon& a, const Canon& b) {
    return ((a.w[0] ^ b.w[0]) | (a.w[1] ^ b.w[1]) | (a.w[2] ^ b.w[2]) | (a.w[3] ^ b.w[3])) == 0;
}

__device__ __forceinline__ uint64_t word_at(const Canon& c, int w) {
    return w == 0 ? c.w[0] : (w == 1 ? c.w[1] : (w == 2 ? c.w[2] : c.w[3]));
}

__device__ __forceinline__ uint32_t code_at(const Canon& c, int k) {
    return (uint32_t)(word_at(c, k / kCodesPerWord) >> (5 * (k % kCodesPerWord))) & 31u;
}

// The string with position p removed (later positions move down by one).
__device__ __forceinline__ Canon delete_at(const Canon& c, int p) {
    const int wp = p / kCodesPerWord;
    const uint64_t low = (1ull << (5 * (p % kCodesPerWord))) - 1ull;
    Canon o;
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const uint64_t next = (w + 1 < kCanonWords) ? (c.w[w + 1] & 31ull) : 0ull;
        const uint64_t down = (c.w[w] >> 5) | (next << 55);
        o.w[w] = w < wp ? c.w[w] : (w > wp ? down : ((c.w[w] & low) | (down & ~low)));
    }
    return o;
}

__device__ __forceinline__ bool run_start(const Canon& c, int p) {
    return p == 0 || code_at(c, p) != code_at(c, p - 1);
}

__device__ __forceinline__ Canon record_content(uint32_t rec, const Canon* __restrict__ ucanon) {
    const Canon c = load_canon(ucanon + (rec >> 7));
    const int p = (int)(rec & 63u);
    return p == (int)kTagF ? c : delete_at(c, p);
}

__device__ __forceinline__ uint32_t part_of(uint64_t h, uint32_t P) {
    return (uint32_t)(((h >> 32) * (uint64_t)P) >> 32);
}

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

inline unsigned grid_for(int64_t n, int threads = kThreads) {
    int64_t b = ceil_div(n, threads);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 1LL << 30));
}

// Block-wide exclusive scan (kThreads threads) of one int64 per thread.
__device__ __forceinline__ int64_t block_scan(int64_t v, int64_t& excl, int64_t* wtot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < kThreads / 32 ? wtot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, t, d);
            if (lane >= d) t += y;
        }
        if (lane < kThreads / 32) wtot[lane] = t;
    }
    __syncthreads();
    excl = (warp ? wtot[warp - 1] : 0) + x - v;
    const int64_t total = wtot[kThreads / 32 - 1];
    __syncthreads();
    return total;
}

// ---- 1. dedup -------------------------------------------------------------

__global__ void k_dedup_insert(const Canon* __restrict__ canon, int64_t n, int32_t* __restrict__ table,
                               uint32_t mask, int32_t* __restrict__ slot_of, int32_t* __restrict__ scount,
                               int* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Canon c = load_canon(canon + i);
    uint32_t slot = (uint32_t)hash_canon(c) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t r = atomicCAS(&table[slot], -1, (int32_t)i);
        if (r == -1 || canon_eq(load_canon(canon + r), c)) {
            slot_of[i] = (int32_t)slot;
            atomicAdd(&scount[slot], 1);
            return;
        }
        slot = (slot + 1) & mask;
    }
    atomicExch(err, 1);  // unreachable: the table has at least 2n slots
    slot_of[i] = -1;
}

__global__ void k_occupied(const int32_t* __restrict__ scount, int64_t S, int32_t* __restrict__ flag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < S) flag[k] = scount[k] > 0 ? 1 : 0;
}

__global__ void k_unique_compact(const int32_t* __restrict__ scount, const int32_t* __restrict__ table,
                                 const int64_t* __restrict__ ubase, int64_t S, const Canon* __restrict__ canon,
                                 const uint8_t* __restrict__ lens, Canon* __restrict__ ucanon,
                                 uint8_t* __restrict__ ulen, int32_t* __restrict__ umult) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S || scount[k] == 0) return;
    const int64_t u = ubase[k];
    const int32_t rep = table[k];
    store_canon(ucanon + u, load_canon(canon + rep));
    ulen[u] = lens[rep];
    umult[u] = scount[k];
}

__global__ void k_uid(const int32_t* __restrict__ slot_of, const int64_t* __restrict__ ubase, int64_t n,
                      int32_t* __restrict__ uid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t slot = slot_of[i];
        uid[i] = slot >= 0 ? (int32_t)ubase[slot] : 0;  // slot < 0 only with the dedup error flag set
    }
}

__global__ void k_members(const int32_t* __restrict__ uid, int64_t n, const int64_t* __restrict__ mem_off,
                          int32_t* __restrict__ mcur, int32_t* __restrict__ members) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t u = uid[i];
    members[mem_off[u] + atomicAdd(&mcur[u], 1)] = (int32_t)i;
}

// ---- 2. records -----------------------------------------------------------

template <bool SCATTER>
__global__ void k_records(const Canon* __restrict__ ucanon, const uint8_t* __restrict__ ulen, int64_t U, uint32_t P,
                          int32_t* __restrict__ pcnt, const int64_t* __restrict__ poff, uint32_t* __restrict__ recs) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const Canon c = load_canon(ucanon + u);
    const int L = ulen[u];
    for (int p = -1; p < L; ++p) {
        const bool full = p < 0;
        const Canon d = full ? c : delete_at(c, p);
        const uint32_t pid = part_of(hash_canon(d), P);
        if (!SCATTER) {
            atomicAdd(&pcnt[pid], 1);
        } else {
            const uint32_t tag = full ? kTagF : ((run_start(c, p) ? 64u : 0u) | (uint32_t)p);
            const int32_t slot = atomicAdd(&pcnt[pid], 1);
            recs[poff[pid] + slot] = ((uint32_t)u << 7) | tag;
        }
    }
}

// ---- 3. join --------------------------------------------------------------

struct JoinSmem {
    uint64_t key[kCap];
    uint32_t rec[kCap];
    int64_t wtot[kThreads / 32];
    int flag;
};

// Edges initiated by sorted record k (see the file comment); calls emit(a, b).
template <typename Emit>
__device__ __forceinline__ int64_t record_edges(const JoinSmem& sm, int k, int s, int T, Emit emit) {
    const uint64_t key = sm.key[k];
    if ((key & 0xffu) == kTagF) return 0;
    const int32_t u = (int32_t)(sm.rec[k] >> 7);
    int64_t cnt = 0;
    int k2 = k + 1;
    for (; k2 < s && sm.key[k2] == key; ++k2) {  // same content, same deleted position
        emit(u, (int32_t)(sm.rec[k2] >> 7));
        ++cnt;
    }
    if (T >= 1 && ((sm.rec[k] >> 6) & 1u)) {  // run-start deletion: look for the full record
        int g = k2;
        while (g < s && (sm.key[g] >> 8) == (key >> 8)) ++g;
        if ((sm.key[g - 1] & 0xffu) == kTagF) {
            emit((int32_t)(sm.rec[g - 1] >> 7), u);
            ++cnt;
        }
    }
    return cnt;
}

template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_join(const int64_t* __restrict__ poff, int64_t P, const uint32_t* __restrict__ recs,
       const Canon* __restrict__ ucanon, int cap, int T, int64_t* __restrict__ pedges,
       const int64_t* __restrict__ eoff, int2* __restrict__ edges, int32_t* __restrict__ fb_list,
       int* __restrict__ fb_count) {
    __shared__ JoinSmem sm;
    const int tid = threadIdx.x;
    for (int64_t pid = blockIdx.x; pid < P; pid += gridDim.x) {
        const int64_t base = poff[pid];
        const int64_t s64 = poff[pid + 1] - base;
        if (s64 > cap) {
            if (!WRITE && tid == 0) {
                fb_list[atomicAdd(fb_count, 1)] = (int32_t)pid;
                pedges[pid] = 0;
            }
            continue;
        }
        const int s = (int)s64;
        if (s < 2) {
            if (!WRITE && tid == 0) pedges[pid] = 0;
            continue;
        }
        const int Pp = next_pow2(s);
        for (int k = tid; k < Pp; k += kThreads) {
            if (k < s) {
                const uint32_t r = recs[base + k];
                const uint64_t h = hash_canon(record_content(r, ucanon));
                sm.key[k] = (h & ~0xffull) | (r & 63u);
                sm.rec[k] = r;
            } else {
                sm.key[k] = ~0ull;
                sm.rec[k] = 0;
            }
        }
        if (tid == 0) sm.flag = 0;
        __syncthreads();
        // bitonic sort of (key, rec) ascending by key
        for (int kk = 2; kk <= Pp; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < (Pp >> 1); i += kThreads) {
                    const int lo = 2 * j * (i / j) + (i % j);
                    const int hi = lo + j;
                    const bool up = (lo & kk) == 0;
                    const uint64_t x = sm.key[lo], y = sm.key[hi];
                    if ((x > y) == up) {
                        sm.key[lo] = y;
                        sm.key[hi] = x;
                        const uint32_t t = sm.rec[lo];
                        sm.rec[lo] = sm.rec[hi];
                        sm.rec[hi] = t;
                    }
                }
                __syncthreads();
            }
        }
        // equal 56-bit hashes must be equal contents; otherwise the exact fallback
        for (int k = tid + 1; k < s; k += kThreads) {
            if ((sm.key[k] >> 8) == (sm.key[k - 1] >> 8) &&
                !canon_eq(record_content(sm.rec[k], ucanon), record_content(sm.rec[k - 1], ucanon)))
                sm.flag = 1;
        }
        __syncthreads();
        if (sm.flag) {
            if (!WRITE && tid == 0) {
                fb_list[atomicAdd(fb_count, 1)] = (int32_t)pid;
                pedges[pid] = 0;
            }
            __syncthreads();
            continue;
        }
        int64_t mine = 0;
        for (int k = tid; k < s; k += kThreads) mine += record_edges(sm, k, s, T, [](int32_t, int32_t) {});
        int64_t excl;
        const int64_t total = block_scan(mine, excl, sm.wtot);
        if (!WRITE) {
            if (tid == 0) pedges[pid] = total;
        } else {
            int64_t pos = eoff[pid] + excl;
            for (int k = tid; k < s; k += kThreads)
                record_edges(sm, k, s, T, [&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
        }
        __syncthreads();
    }
}

// Exact quadratic join of one partition (over capacity or with a hash collision).
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_join_fallback(const int32_t* __restrict__ fb_list, int nfb, const int64_t* __restrict__ poff,
                const uint32_t* __restrict__ recs, const Canon* __restrict__ ucanon, int T,
                int64_t* __restrict__ pedges, const int64_t* __restrict__ eoff, int2* __restrict__ edges) {
    __shared__ int64_t wtot[kThreads / 32];
    for (int f = blockIdx.x; f < nfb; f += gridDim.x) {
        const int64_t pid = fb_list[f];
        const int64_t base = poff[pid];
        const int64_t s = poff[pid + 1] - base;
        auto scan_pairs = [&](auto emit) {
            int64_t cnt = 0;
            for (int64_t k1 = threadIdx.x; k1 < s; k1 += kThreads) {
                const uint32_t r1 = recs[base + k1];
                const uint32_t p1 = r1 & 63u;
                if (p1 == kTagF) continue;  // deletion records initiate every edge
                const Canon c1 = record_content(r1, ucanon);
                const bool rs1 = (r1 >> 6) & 1u;
                for (int64_t k2 = 0; k2 < s; ++k2) {
                    if (k2 == k1) continue;
                    const uint32_t r2 = recs[base + k2];
                    const uint32_t p2 = r2 & 63u;
                    const bool same = (p2 == p1) && (k2 > k1);
                    const bool indel = (T >= 1) && rs1 && (p2 == kTagF);
                    if (!same && !indel) continue;
                    if (!canon_eq(c1, record_content(r2, ucanon))) continue;
                    if (same) emit((int32_t)(r1 >> 7), (int32_t)(r2 >> 7));
                    else emit((int32_t)(r2 >> 7), (int32_t)(r1 >> 7));
                    ++cnt;
                }
            }
            return cnt;
        };
        const int64_t mine = scan_pairs([](int32_t, int32_t) {});
        int64_t excl;
        const int64_t total = block_scan(mine, excl, wtot);
        if (!WRITE) {
            if (threadIdx.x == 0) pedges[pid] = total;
        } else {
            int64_t pos = eoff[pid] + excl;
            scan_pairs([&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
        }
        __syncthreads();
    }
}

// ---- 4. degrees -----------------------------------------------------------

__global__ void k_weighted_degree(const int2* __restrict__ edges, int64_t E, const int32_t* __restrict__ umult,
                                  int32_t* __restrict__ wsum) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int2 uv = edges[e];
    atomicAdd(&wsum[uv.x], umult[uv.y]);
    atomicAdd(&wsum[uv.y], umult[uv.x]);
}

__global__ void k_node_degree(const int32_t* __restrict__ uid, int64_t n, const int32_t* __restrict__ umult,
                              const int32_t* __restrict__ wsum, int32_t* __restrict__ deg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t u = uid[i];
    deg[i] = umult[u] - 1 + wsum[u];
}

// ---- 5. fill --------------------------------------------------------------

__global__ void k_cursor_init(const int32_t* __restrict__ umult, int64_t U, int32_t* __restrict__ cur) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < U) cur[u] = umult[u] - 1;
}

__global__ void k_fill_self(const int32_t* __restrict__ uid, int64_t n, const int32_t* __restrict__ umult,
                            const int64_t* __restrict__ mem_off, const int32_t* __restrict__ members,
                            const int64_t* __restrict__ off, int32_t* __restrict__ cols) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t u = uid[i];
    const int32_t m = umult[u];
    if (m < 2) return;
    const int64_t b = off[i];
    const int32_t* mem = members + mem_off[u];
    int32_t pos = 0;
    for (int32_t k = 0; k < m; ++k) {
        const int32_t j = mem[k];
        if (j != (int32_t)i) cols[b + pos++] = j;
    }
}

__global__ void k_fill_edges(const int2* __restrict__ edges, int64_t E, const int32_t* __restrict__ umult,
                             const int64_t* __restrict__ mem_off, const int32_t* __restrict__ members,
                             const int64_t* __restrict__ off, int32_t* __restrict__ cur, int32_t* __restrict__ cols,
                             int64_t* __restrict__ heavy, int* __restrict__ nheavy, int* __restrict__ err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * E) return;
    const int2 uv = edges[t >> 1];
    const int32_t a = (t & 1) ? uv.y : uv.x;  // row side
    const int32_t b = (t & 1) ? uv.x : uv.y;  // neighbour side
    const int32_t ma = umult[a], mb = umult[b];
    if ((int64_t)ma * mb > kHeavy) {
        heavy[atomicAdd(nheavy, 1)] = t;
        return;
    }
    const int32_t slot = atomicAdd(&cur[a], mb);
    const int32_t* ra = members + mem_off[a];
    const int32_t* rb = members + mem_off[b];
    for (int32_t x = 0; x < ma; ++x) {
        const int32_t i = ra[x];
        const int64_t o = off[i] + slot;
        if (o + mb > off[i + 1]) {
            atomicExch(err, 1);
            continue;
        }
        for (int32_t y = 0; y < mb; ++y) cols[o + y] = rb[y];
    }
}

__global__ void k_fill_heavy(const int64_t* __restrict__ heavy, const int* __restrict__ nheavy,
                             const int2* __restrict__ edges, const int32_t* __restrict__ umult,
                             const int64_t* __restrict__ mem_off, const int32_t* __restrict__ members,
                             const int64_t* __restrict__ off, int32_t* __restrict__ cur, int32_t* __restrict__ cols,
                             int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nh = *nheavy;
    for (int64_t w = w0; w < nh; w += nw) {
        const int64_t t = heavy[w];
        const int2 uv = edges[t >> 1];
        const int32_t a = (t & 1) ? uv.y : uv.x;
        const int32_t b = (t & 1) ? uv.x : uv.y;
        const int32_t ma = umult[a], mb = umult[b];
        int32_t slot = 0;
        if (lane == 0) slot = atomicAdd(&cur[a], mb);
        slot = __shfl_sync(kFull, slot, 0);
        const int32_t* ra = members + mem_off[a];
        const int32_t* rb = members + mem_off[b];
        const int64_t total = (int64_t)ma * mb;
        for (int64_t idx = lane; idx < total; idx += 32) {
            const int32_t i = ra[idx / mb];
            const int32_t y = (int32_t)(idx % mb);
            const int64_t o = off[i] + slot + y;
            if (o < off[i + 1]) cols[o] = rb[y];
            else atomicExch(err, 1);
        }
    }
}

class Timer {
public:
    Timer(bool on, cudaStream_t s) : on_(on), s_(s) {}
    ~Timer() {
        for (auto e : ev_) cudaEventDestroy(e);
    }
    int mark() {
        if (!on_) return -1;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        cudaEventRecord(e, s_);
        ev_.push_back(e);
        return (int)ev_.size() - 1;
    }
    double ms(int a, int b) {
        if (!on_ || a < 0 || b < 0) return 0.0;
        cudaEventSynchronize(ev_[b]);
        float t = 0.f;
        cudaEventElapsedTime(&t, ev_[a], ev_[b]);
        return (double)t;
    }

private:
    bool on_;
    cudaStream_t s_;
    std::vector<cudaEvent_t> ev_;
};

}  // namespace

tcrnet_status deletion_build(const Packed& pk, int T, DeletionResult& out, cudaStream_t s, int num_sms, bool profile,
                             int partition_cap) {
    const int64_t n = pk.n;
    if (n > kDeletionMaxN) return TCRNET_ENOTSUP;
    const int cap = (partition_cap > 0 && partition_cap < kCap) ? partition_cap : kCap;
    Timer tm(profile, s);
    const int t0 = tm.mark();

    // ---- 1. dedup
    int64_t S = 1024;
    while (S < 2 * n) S <<= 1;
    DevBuf table, slot_of, scount, flag, ubase, errb;
    TCR_CHECK(table.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(slot_of.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(scount.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(flag.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(ubase.alloc(sizeof(int64_t) * (S + 1), s));
    TCR_CHECK(errb.alloc(sizeof(int) * 4, s));  // [0] dedup, [1] fill, [2] fallback count, [3] heavy count
    TCR_CUDA(cudaMemsetAsync(table.as<void>(), 0xff, sizeof(int32_t) * S, s));
    TCR_CUDA(cudaMemsetAsync(scount.as<void>(), 0, sizeof(int32_t) * S, s));
    TCR_CUDA(cudaMemsetAsync(errb.as<void>(), 0, sizeof(int) * 4, s));
    int* d_err = errb.as<int>();
    k_dedup_insert<<<grid_for(n), kThreads, 0, s>>>(pk.canon_in.as<Canon>(), n, table.as<int32_t>(),
                                                    (uint32_t)(S - 1), slot_of.as<int32_t>(), scount.as<int32_t>(),
                                                    d_err);
    TCR_LAUNCH_CHECK();
    k_occupied<<<grid_for(S), kThreads, 0, s>>>(scount.as<int32_t>(), S, flag.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(flag.as<int32_t>(), ubase.as<int64_t>(), S, s));
    int64_t U = 0;
    TCR_CUDA(cudaMemcpyAsync(&U, ubase.as<int64_t>() + S, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    DevBuf ucanon, ulen, umult, uid, mem_off, mcur, members;
    TCR_CHECK(ucanon.alloc(sizeof(Canon) * U, s));
    TCR_CHECK(ulen.alloc(U, s));
    TCR_CHECK(umult.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(uid.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(mem_off.alloc(sizeof(int64_t) * (U + 1), s));
    TCR_CHECK(mcur.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(members.alloc(sizeof(int32_t) * n, s));
    k_unique_compact<<<grid_for(S), kThreads, 0, s>>>(scount.as<int32_t>(), table.as<int32_t>(), ubase.as<int64_t>(),
                                                      S, pk.canon_in.as<Canon>(), pk.lens.as<uint8_t>(),
                                                      ucanon.as<Canon>(), ulen.as<uint8_t>(), umult.as<int32_t>());
    TCR_LAUNCH_CHECK();
    k_uid<<<grid_for(n), kThreads, 0, s>>>(slot_of.as<int32_t>(), ubase.as<int64_t>(), n, uid.as<int32_t>());
    TCR_LAUNCH_CHECK();
    table.reset();
    slot_of.reset();
    scount.reset();
    flag.reset();
    ubase.reset();
    TCR_CHECK(scan_exclusive_i32_to_i64(umult.as<int32_t>(), mem_off.as<int64_t>(), U, s));
    TCR_CUDA(cudaMemsetAsync(mcur.as<void>(), 0, sizeof(int32_t) * U, s));
    k_members<<<grid_for(n), kThreads, 0, s>>>(uid.as<int32_t>(), n, mem_off.as<int64_t>(), mcur.as<int32_t>(),
                                               members.as<int32_t>());
    TCR_LAUNCH_CHECK();
    mcur.reset();
    const int t1 = tm.mark();

    // ---- 2. records and 3. join (l_max >= 1 only; l_max = 0 keeps duplicates only)
    DevBuf edges;
    int64_t E = 0, R = 0, nfb = 0;
    int t2 = t1, t3 = t1, t4 = t1;
    if (T >= 1 && U > 0) {
        int64_t lensum = 0;
        for (int L = 1; L <= kMaxLen; ++L) lensum += (int64_t)L * (pk.bucket_off[L + 1] - pk.bucket_off[L]);
        const double mean_len = n > 0 ? (double)lensum / (double)n : 1.0;
        const int64_t R_est = (int64_t)((double)U * (mean_len + 1.0)) + 1;
        const int64_t P = std::max<int64_t>(1, std::min<int64_t>(R_est / kTargetPart + 1, 1LL << 30));
        DevBuf pcnt, poff, recs, pedges, eoff, fb_list;
        TCR_CHECK(pcnt.alloc(sizeof(int32_t) * P, s));
        TCR_CHECK(poff.alloc(sizeof(int64_t) * (P + 1), s));
        TCR_CUDA(cudaMemsetAsync(pcnt.as<void>(), 0, sizeof(int32_t) * P, s));
        k_records<false><<<grid_for(U), kThreads, 0, s>>>(ucanon.as<Canon>(), ulen.as<uint8_t>(), U, (uint32_t)P,
                                                          pcnt.as<int32_t>(), nullptr, nullptr);
        TCR_LAUNCH_CHECK();
        TCR_CHECK(scan_exclusive_i32_to_i64(pcnt.as<int32_t>(), poff.as<int64_t>(), P, s));
        TCR_CUDA(cudaMemcpyAsync(&R, poff.as<int64_t>() + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        TCR_CHECK(recs.alloc(sizeof(uint32_t) * R, s));
        TCR_CUDA(cudaMemsetAsync(pcnt.as<void>(), 0, sizeof(int32_t) * P, s));
        k_records<true><<<grid_for(U), kThreads, 0, s>>>(ucanon.as<Canon>(), ulen.as<uint8_t>(), U, (uint32_t)P,
                                                         pcnt.as<int32_t>(), poff.as<int64_t>(), recs.as<uint32_t>());
        TCR_LAUNCH_CHECK();
        pcnt.reset();
        t2 = tm.mark();
        TCR_CHECK(pedges.alloc(sizeof(int64_t) * P, s));
        TCR_CHECK(eoff.alloc(sizeof(int64_t) * (P + 1), s));
        TCR_CHECK(fb_list.alloc(sizeof(int32_t) * P, s));
        const int jgrid = (int)std::min<int64_t>(P, (int64_t)num_sms * 8);
        k_join<false><<<jgrid, kThreads, 0, s>>>(poff.as<int64_t>(), P, recs.as<uint32_t>(), ucanon.as<Canon>(), cap,
                                                 T, pedges.as<int64_t>(), nullptr, nullptr, fb_list.as<int32_t>(),
                                                 d_err + 2);
        TCR_LAUNCH_CHECK();
        int h_nfb = 0;
        TCR_CUDA(cudaMemcpyAsync(&h_nfb, d_err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        nfb = h_nfb;
        if (h_nfb > 0) {
            k_join_fallback<false><<<std::min(h_nfb, num_sms * 4), kThreads, 0, s>>>(
                fb_list.as<int32_t>(), h_nfb, poff.as<int64_t>(), recs.as<uint32_t>(), ucanon.as<Canon>(), T,
                pedges.as<int64_t>(), nullptr, nullptr);
            TCR_LAUNCH_CHECK();
        }
        TCR_CHECK(scan_exclusive_i64(pedges.as<int64_t>(), eoff.as<int64_t>(), P, s));
        TCR_CUDA(cudaMemcpyAsync(&E, eoff.as<int64_t>() + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        t3 = tm.mark();
        TCR_CHECK(edges.alloc(sizeof(int2) * E, s));
        if (E > 0) {
            k_join<true><<<jgrid, kThreads, 0, s>>>(poff.as<int64_t>(), P, recs.as<uint32_t>(), ucanon.as<Canon>(),
                                                    cap, T, nullptr, eoff.as<int64_t>(), edges.as<int2>(), nullptr,
                                                    nullptr);
            TCR_LAUNCH_CHECK();
            if (h_nfb > 0) {
                k_join_fallback<true><<<std::min(h_nfb, num_sms * 4), kThreads, 0, s>>>(
                    fb_list.as<int32_t>(), h_nfb, poff.as<int64_t>(), recs.as<uint32_t>(), ucanon.as<Canon>(), T,
                    nullptr, eoff.as<int64_t>(), edges.as<int2>());
                TCR_LAUNCH_CHECK();
            }
        }
        t4 = tm.mark();
    }

    // ---- 4. degrees
    DevBuf wsum, deg, off64;
    TCR_CHECK(wsum.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(deg.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(off64.alloc(sizeof(int64_t) * (n + 1), s));
    TCR_CUDA(cudaMemsetAsync(wsum.as<void>(), 0, sizeof(int32_t) * U, s));
    if (E > 0) {
        k_weighted_degree<<<grid_for(E), kThreads, 0, s>>>(edges.as<int2>(), E, umult.as<int32_t>(),
                                                           wsum.as<int32_t>());
        TCR_LAUNCH_CHECK();
    }
    k_node_degree<<<grid_for(n), kThreads, 0, s>>>(uid.as<int32_t>(), n, umult.as<int32_t>(), wsum.as<int32_t>(),
                                                   deg.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(deg.as<int32_t>(), off64.as<int64_t>(), n, s));
    int64_t nnz = 0;
    TCR_CUDA(cudaMemcpyAsync(&nnz, off64.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    wsum.reset();
    const int t5 = tm.mark();

    // ---- 5. fill
    DevBuf cols, cur, heavy;
    TCR_CHECK(cols.alloc(sizeof(int32_t) * nnz, s));
    TCR_CHECK(cur.alloc(sizeof(int32_t) * U, s));
    k_cursor_init<<<grid_for(U), kThreads, 0, s>>>(umult.as<int32_t>(), U, cur.as<int32_t>());
    TCR_LAUNCH_CHECK();
    k_fill_self<<<grid_for(n), kThreads, 0, s>>>(uid.as<int32_t>(), n, umult.as<int32_t>(), mem_off.as<int64_t>(),
                                                 members.as<int32_t>(), off64.as<int64_t>(), cols.as<int32_t>());
    TCR_LAUNCH_CHECK();
    if (E > 0) {
        TCR_CHECK(heavy.alloc(sizeof(int64_t) * 2 * E, s));
        k_fill_edges<<<grid_for(2 * E), kThreads, 0, s>>>(edges.as<int2>(), E, umult.as<int32_t>(),
                                                          mem_off.as<int64_t>(), members.as<int32_t>(),
                                                          off64.as<int64_t>(), cur.as<int32_t>(), cols.as<int32_t>(),
                                                          heavy.as<int64_t>(), d_err + 3, d_err + 1);
        TCR_LAUNCH_CHECK();
        k_fill_heavy<<<num_sms * 8, kThreads, 0, s>>>(heavy.as<int64_t>(), d_err + 3, edges.as<int2>(),
                                                      umult.as<int32_t>(), mem_off.as<int64_t>(),
                                                      members.as<int32_t>(), off64.as<int64_t>(), cur.as<int32_t>(),
                                                      cols.as<int32_t>(), d_err + 1);
        TCR_LAUNCH_CHECK();
    }
    const int t6 = tm.mark();
    TCR_CHECK(sort_rows(off64.as<int64_t>(), cols.as<int32_t>(), n, s, num_sms));
    const int t7 = tm.mark();
    int h_err[4] = {0, 0, 0, 0};
    TCR_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    if (h_err[0] || h_err[1]) return TCRNET_EDEVICE;

    out.off64 = std::move(off64);
    out.cols = std::move(cols);
    out.degree = std::move(deg);
    out.nnz = nnz;
    out.n_unique = U;
    out.n_records = R;
    out.unique_edges = E;
    out.n_fallback = nfb;
    out.ms_phase[0] = tm.ms(t0, t1);
    out.ms_phase[1] = tm.ms(t1, t2);
    out.ms_phase[2] = tm.ms(t2, t3);
    out.ms_phase[3] = tm.ms(t3, t4);
    out.ms_phase[4] = tm.ms(t4, t5);
    out.ms_phase[5] = tm.ms(t5, t6);
    out.ms_phase[6] = tm.ms(t6, t7);
    out.ms_phase[7] = tm.ms(t0, t7);
    out.ms_join = tm.ms(t2, t3) + tm.ms(t3, t4);
    out.ms_scan = tm.ms(t4, t5);
    out.ms_fill = tm.ms(t5, t6);
    out.ms_sort = tm.ms(t6, t7);
    return TCRNET_OK;
}

}  // namespace tcr
