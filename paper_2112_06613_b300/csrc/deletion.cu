// Deletion-neighbourhood method: the network of Methods "TCR network" (edges at
// Levenshtein distance <= l_max) without testing all pairs.
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
//     atomicCAS, exact comparison on probe; the claiming thread numbers the
//     new distinct string) -> distinct-string ids u,
//     multiplicities m_u, member lists M_u.
//  2. records: per distinct string one full-string record (tag p = 63) and one
//     record per deletion position p; each is one 64-bit word
//       bits 63..32  low 32 bits of the content hash
//       bits 31..26  p (63: the full string)
//       bit  25      p starts a run of equal letters
//       bits 24..0   u
//     hash-partitioned (high hash bits, 24 or 32 records per partition on
//     average) in two passes (count, scatter).
//  3. join: windows of whole consecutive partitions with at most 32 records
//     are joined by one warp step without sorting (lane k holds record k;
//     warp match on the hash gives each record its group, on (hash, p) its
//     run); partitions of 33..128 records by a warp that sorts its words in
//     registers (bitonic network), larger ones by a quadratic block pass. The
//     candidate pairs are every pair inside a run of equal (hash, p) (equal
//     length, one substitution) and each run-start deletion record with each
//     full record of its hash group (one indel); they go into a buffer of
//     2 x (records bound) entries (staged per warp in shared memory) or, if
//     they do not fit, a second pass writes them at positions scanned from
//     the per-partition counts. A confirmation pass then compares the two
//     contents of every candidate (exact: equal contents make equal hashes,
//     so no edge is missed, and a hash collision is rejected there) and adds
//     m_v to W_u (and m_u to W_v) for every edge {u, v}.
//  4. closed neighbourhoods: D_u = m_u + W_u; S_u = M_u followed by every
//     M_v (appended at a slot taken from a per-string cursor; long member
//     lists are copied by a whole warp), written once per distinct string and
//     sorted (rowsort.cu). A node i of u has degree D_u - 1.
//  5. expand: row i of the CSR is S_u without i (a streaming copy), so the
//     long rows of frequent strings are sorted once, not once per copy.
// l_max = 2 replaces steps 2-3 (section 3' below): candidates from shared
// variants with up to two deletions, checked with the exact distance.
#include <algorithm>
#include <vector>

#include "deletion.cuh"
#include "lookback.cuh"

namespace tcr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpCap = 128;     // records per partition joined by one warp
// Default mean records per partition. Fewer records per partition fill the
// join's 32-lane windows better (a window ends at a partition boundary) and
// send fewer partitions to the sorted join; more partitions make the counters
// of the record scatter colder. Measured on one B300 at 8e5 strings (build
// 0.827 ms at 12, 0.830 at 16, 0.837 at 8, 0.852 at 24); 8.9e6 strings: 32
// (an earlier join; 14.5 vs 14.8 ms at 24).
constexpr int kTargetPartSmall = 12;
constexpr int kTargetPartLarge = 32;
constexpr int64_t kTargetSwitchRecords = 1LL << 25;
constexpr uint32_t kTagF = 63;    // position tag of a full-string record
constexpr uint64_t kUMask = (1ull << 25) - 1;
constexpr int kEdgeSegs = 64;     // edge buffer segments (one cursor each), by partition id

__device__ __forceinline__ uint32_t rec_u(uint64_t r) { return (uint32_t)(r & kUMask); }
__device__ __forceinline__ uint32_t rec_p(uint64_t r) { return (uint32_t)(r >> 26) & 63u; }
__device__ __forceinline__ bool rec_runstart(uint64_t r) { return (r >> 25) & 1ull; }

// 64-bit finaliser of MurmurHash3 (public domain).
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// Content hash: odd-multiplier combination of the four words, then one
// finaliser. Only the partition choice and the in-partition order depend on
// it; equal hashes are always confirmed by comparing contents.
// The repertoire tag (top nibble of each word) enters through its own term:
// in the word combination a top-nibble difference only reaches bits 60..63 of
// x, so strings equal up to their tag would collide for 1 in 16 tag pairs.
// The gathered 16-bit tag times an odd constant keeps its lowest set bit below
// bit 16, so a pure tag difference can never cancel.
constexpr uint64_t kHashMul1 = 0x9e3779b97f4a7c15ULL;
constexpr uint64_t kHashMul2 = 0xc2b2ae3d27d4eb4fULL;
constexpr uint64_t kHashMul3 = 0x165667b19e3779f9ULL;
constexpr uint64_t kHashMulTag = 0xd6e8feb86659fd93ULL;
constexpr uint64_t kHashSeed = 0x243f6a8885a308d3ULL;

__device__ __forceinline__ uint64_t canon_tag(const Canon& c) {
    return (c.w[0] >> 60) | ((c.w[1] >> 56) & 0xF0ull) | ((c.w[2] >> 52) & 0xF00ull) | ((c.w[3] >> 48) & 0xF000ull);
}

__device__ __forceinline__ uint64_t hash_canon(const Canon& c) {
    const uint64_t x = c.w[0] + kHashMul1 * c.w[1] + kHashMul2 * c.w[2] + kHashMul3 * c.w[3] +
                       kHashMulTag * canon_tag(c);
    return fmix64(x ^ kHashSeed);
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

// The string with position p removed (later positions move down by one); the
// repertoire tag bits stay where they are.
__device__ __forceinline__ Canon delete_at(const Canon& c, int p) {
    const int wp = p / kCodesPerWord;
    const uint64_t low = (1ull << (5 * (p % kCodesPerWord))) - 1ull;
    Canon o;
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const uint64_t cw = c.w[w] & ~kTagBits;
        const uint64_t next = (w + 1 < kCanonWords) ? (c.w[w + 1] & 31ull) : 0ull;
        const uint64_t down = (cw >> 5) | (next << 55);
        o.w[w] = (w < wp ? cw : (w > wp ? down : ((cw & low) | (down & ~low)))) | (c.w[w] & kTagBits);
    }
    return o;
}

__device__ __forceinline__ bool run_start(const Canon& c, int p) {
    return p == 0 || code_at(c, p) != code_at(c, p - 1);
}

// fn(p, h, rs) for the full string (p = -1) and for each deletion position p
// of a string of L letters, with h = hash_canon(p < 0 ? c : delete_at(c, p))
// and rs = run_start(c, p), at a fraction of the work of those calls: the word
// combination inside the hash is linear, and deleting p keeps the words before
// p's word, shifts every word after it down by one letter and mixes the two
// forms inside p's word. So the sum over the kept prefix and the sum over the
// shifted suffix are formed once per string; a variant adds its mixed word
// (two logic operations, one multiply) and runs the finaliser.
template <typename Fn>
__device__ __forceinline__ void for_each_variant_hash(const Canon& c, int L, Fn fn) {
    uint64_t down[kCanonWords];  // word w shifted down one letter, the next word's first letter on top
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const uint64_t cw = c.w[w] & ~kTagBits;
        const uint64_t next = (w + 1 < kCanonWords) ? (c.w[w + 1] & 31ull) : 0ull;
        down[w] = (cw >> 5) | (next << 55) | (c.w[w] & kTagBits);
    }
    const uint64_t mul[kCanonWords] = {1ull, kHashMul1, kHashMul2, kHashMul3};
    const uint64_t t = kHashMulTag * canon_tag(c);
    fn(-1, fmix64((c.w[0] + kHashMul1 * c.w[1] + kHashMul2 * c.w[2] + kHashMul3 * c.w[3] + t) ^ kHashSeed), false);
    uint64_t pre = 0;  // words before w as they are
    uint64_t suf = kHashMul1 * down[1] + kHashMul2 * down[2] + kHashMul3 * down[3] + t;  // words after w, shifted
    uint32_t prev = 32u;  // letter before the position (none before 0; codes are < 32)
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const int p0 = w * kCodesPerWord;
        const int pend = L < p0 + kCodesPerWord ? L : p0 + kCodesPerWord;
        uint64_t low = 0;  // positions of the word before p
        uint64_t cur = c.w[w];
        for (int p = p0; p < pend; ++p) {
            const uint32_t code = (uint32_t)cur & 31u;
            cur >>= 5;
            const uint64_t mixed = (c.w[w] & low) | (down[w] & ~low);
            fn(p, fmix64((pre + mul[w] * mixed + suf) ^ kHashSeed), code != prev);
            prev = code;
            low = (low << 5) | 31ull;
        }
        pre += mul[w] * c.w[w];
        if (w + 1 < kCanonWords) suf -= mul[w + 1] * down[w + 1];
    }
}

__device__ __forceinline__ Canon record_content(uint64_t rec, const Canon* __restrict__ ucanon) {
    const Canon c = load_canon(ucanon + rec_u(rec));
    const uint32_t p = rec_p(rec);
    return p == kTagF ? c : delete_at(c, (int)p);
}

__device__ __forceinline__ uint32_t part_of(uint64_t h, uint32_t P) {
    return (uint32_t)(((h >> 32) * (uint64_t)P) >> 32);
}

// Blocks per edge segment of k_confirm (grid-stride loop; the candidate counts
// are not known on the host when it is launched): about eight blocks per SM.
inline unsigned confirm_blocks_x(int num_sms) {
    return (unsigned)std::max(1, num_sms * 8 / kEdgeSegs);
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
        int64_t t = lane < kWarps ? wtot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, t, d);
            if (lane >= d) t += y;
        }
        if (lane < kWarps) wtot[lane] = t;
    }
    __syncthreads();
    excl = (warp ? wtot[warp - 1] : 0) + x - v;
    const int64_t total = wtot[kWarps - 1];
    __syncthreads();
    return total;
}

// Warp-wide exclusive scan of one int64 per lane; returns the warp total.
__device__ __forceinline__ int64_t warp_scan(int64_t v, int64_t& excl, int lane) {
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    excl = x - v;
    return __shfl_sync(kFull, x, 31);
}

// ---- 1. dedup -------------------------------------------------------------

// Claim or find the table slot of each string. The claiming thread numbers
// the new distinct string (u = running count; the numbering depends on the
// schedule, the network does not) and copies it to ucanon/ulen.
__global__ void k_dedup_insert(const Canon* __restrict__ canon, const uint8_t* __restrict__ lens, int64_t n,
                               int32_t* __restrict__ table, uint32_t mask, int32_t* __restrict__ slot_of,
                               int32_t* __restrict__ slot_u, unsigned long long* __restrict__ U,
                               Canon* __restrict__ ucanon, uint8_t* __restrict__ ulen, int* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Canon c = load_canon(canon + i);
    uint32_t slot = (uint32_t)hash_canon(c) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t r = atomicCAS(&table[slot], -1, (int32_t)i);
        if (r == -1) {
            const int32_t u = (int32_t)atomicAdd(U, 1ull);
            slot_u[slot] = u;
            store_canon(ucanon + u, c);
            ulen[u] = lens[i];
            slot_of[i] = (int32_t)slot;
            return;
        }
        if (canon_eq(load_canon(canon + r), c)) {
            slot_of[i] = (int32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    atomicExch(err, 1);  // unreachable: the table has at least 2n slots
    slot_of[i] = -1;
}

// Every array of a build that starts at a fixed value, set in one launch before
// the dedup (in place of five memsets, four of them between the dedup and the
// kernels after it): the counter block, the dedup table (-1), the
// multiplicities and weights (0) and, for the l_max = 1 join, the partition
// counts (0).
__global__ void k_build_clear(unsigned long long* __restrict__ zeroed, int64_t zwords, int32_t* __restrict__ table,
                              int64_t S, int32_t* __restrict__ umult, int32_t* __restrict__ wsum, int64_t n,
                              int32_t* __restrict__ pcnt, int64_t P) {
    const int64_t total = zwords + S + 2 * n + P;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = t;
        if (k < zwords) {
            zeroed[k] = 0ull;
        } else if ((k -= zwords) < S) {
            table[k] = -1;
        } else if ((k -= S) < n) {
            umult[k] = 0;
        } else if ((k -= n) < n) {
            wsum[k] = 0;
        } else {
            pcnt[k - n] = 0;  // k - n < P
        }
    }
}

// Distinct-string id of every node and the multiplicities m_u.
__global__ void k_uid(const int32_t* __restrict__ slot_of, const int32_t* __restrict__ slot_u, int64_t n,
                      int32_t* __restrict__ uid, int32_t* __restrict__ umult) {
    dep_entry();  // launched dependent on the kernel before it
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t slot = slot_of[i];
        const int32_t u = slot >= 0 ? slot_u[slot] : 0;  // slot < 0 only with the dedup error flag set
        uid[i] = u;
        atomicAdd(&umult[u], 1);
    }
}

// Member lists M_u (arrival order) and each node's position inside its list.
__global__ void k_members(const int32_t* __restrict__ uid, int64_t n, const int64_t* __restrict__ mem_off,
                          int32_t* __restrict__ mcur, int32_t* __restrict__ members, int32_t* __restrict__ mpos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t u = uid[i];
    const int32_t k = atomicAdd(&mcur[u], 1);
    members[mem_off[u] + k] = (int32_t)i;
    mpos[i] = k;
}

// ---- 2. records -----------------------------------------------------------

constexpr int kRecBatch = 4;  // records of the scatter in flight per thread (8 measured slower)

// Stores of the record scatter carry an L2 evict-last hint: the ~1e6 partition
// write fronts each fill a 32-byte sector a few records at a time, and a line
// the L2 evicts before its sector is complete makes the DRAM read it back and
// merge it. (A per-instruction priority; no cache setting is changed.)
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void st_keep(uint64_t* p, uint64_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// The scatter takes each record's absolute position from its partition's
// cursor (pcnt, seeded with the partition start by the scan: one atomic and
// one store per record, no offset load). It writes nothing when the records
// counted exceed R_cap, the size the record array was given (only invalid
// input, whose error the build reports at its first readback, can get there).
template <bool SCATTER>
__global__ void k_records(const Canon* __restrict__ ucanon, const uint8_t* __restrict__ ulen,
                          const int64_t* __restrict__ U_ptr, int64_t n, uint32_t P, int32_t* __restrict__ pcnt,
                          const int64_t* __restrict__ poff, uint64_t* __restrict__ recs, uint32_t u0 = 0,
                          int64_t R_cap = INT64_MAX, uint64_t hash_mask = 0xffffffffull) {
    dep_entry();  // launched dependent on the kernel before it
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || u >= *U_ptr) return;
    if (SCATTER && poff[P] > R_cap) return;
    const Canon c = load_canon(ucanon + u);
    const int L = ulen[u];
    const uint64_t uid = (uint64_t)(u0 + (uint32_t)u);  // ids of a slice start at u0
    if constexpr (!SCATTER) {
        for_each_variant_hash(c, L, [&](int, uint64_t h, bool) { atomicAdd(&pcnt[part_of(h, P)], 1); });
    } else {
        // kRecBatch records at a time (a shift register of pending ones): their
        // slot atomics and offset loads are independent, so they are in flight
        // together rather than one round trip each
        const uint64_t pol = l2_keep_policy();
        uint64_t r[kRecBatch];
        uint32_t q[kRecBatch];
#pragma unroll
        for (int j = 0; j < kRecBatch; ++j) {
            r[j] = 0;
            q[j] = 0;
        }
        int pending = 0;
        auto issue = [&](int k) {  // the k newest pending records (k <= kRecBatch)
            int32_t sl[kRecBatch];
#pragma unroll
            for (int j = 0; j < kRecBatch; ++j) sl[j] = j < k ? atomicAdd(&pcnt[q[j]], 1) : 0;
#pragma unroll
            for (int j = 0; j < kRecBatch; ++j)
                if (j < k) st_keep(recs + sl[j], r[j], pol);
        };
        for_each_variant_hash(c, L, [&](int p, uint64_t h, bool rs) {
            const uint64_t tag = p < 0 ? ((uint64_t)kTagF << 26) : (((uint64_t)p << 26) | (rs ? (1ull << 25) : 0ull));
#pragma unroll
            for (int j = kRecBatch - 1; j > 0; --j) {
                r[j] = r[j - 1];
                q[j] = q[j - 1];
            }
            r[0] = ((h & hash_mask) << 32) | tag | uid;  // (hash_mask: testing, fewer hash bits kept)
            q[0] = part_of(h, P);
            if (++pending == kRecBatch) {
                issue(kRecBatch);
                pending = 0;
            }
        });
        issue(pending);
    }
}

// ---- 3. join --------------------------------------------------------------

// Bitonic sort of 32*K words held K per lane (network position lane*K + r).
template <int K>
__device__ __forceinline__ void warp_sort_u64(uint64_t (&v)[K], int lane) {
    constexpr int P = 32 * K;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    if ((r & j) == 0) {
                        const int r2 = r | j;
                        const bool up = ((lane * K + r) & k) == 0;
                        const uint64_t a = v[r], b = v[r2];
                        const bool sw = (a > b) == up;
                        v[r] = sw ? b : a;
                        v[r2] = sw ? a : b;
                    }
                }
            } else {
                const int jl = j / K;
                const bool lower = (lane & jl) == 0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const uint64_t p = __shfl_xor_sync(kFull, v[r], jl);
                    const bool up = ((lane * K + r) & k) == 0;
                    const uint64_t mn = v[r] < p ? v[r] : p;
                    const uint64_t mx = v[r] < p ? p : v[r];
                    v[r] = (lower == up) ? mn : mx;
                }
            }
        }
    }
}

template <int K>
__device__ __forceinline__ void load_sort_store(const uint64_t* __restrict__ src, int s, uint64_t* buf, int lane) {
    uint64_t v[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = r * 32 + lane;
        v[r] = e < s ? src[e] : ~0ull;  // ~0 is never a record (full records have no run-start bit)
    }
    warp_sort_u64<K>(v, lane);
#pragma unroll
    for (int r = 0; r < K; ++r) buf[lane * K + r] = v[r];
}

// A candidate pair of the join, one side per int32: the distinct string u in
// bits 24..0 and the variant of it that matched in bits 30..25 (the deleted
// position p, or kTagF for the full string). k_confirm compares the two
// variants' contents and rewrites the entry as the plain edge (u, v), or as
// (-1, -1) when the 32-bit hashes matched by accident.
__device__ __forceinline__ int32_t cand_side(uint64_t rec) {
    return (int32_t)(rec_u(rec) | (rec_p(rec) << 25));
}

// Candidates initiated by sorted record k (see the file comment); calls
// emit(a, b) with encoded sides. Same-position partners are the later records
// of k's run of equal (hash, p); a run-start deletion pairs with every full
// record of its hash group (these sort to the group's end; more than one only
// under a hash collision, which the confirmation sorts out).
template <typename Emit>
__device__ __forceinline__ int64_t record_cands(const uint64_t* buf, int k, int s, int T, Emit emit) {
    const uint64_t key = buf[k];
    if (rec_p(key) == kTagF) return 0;
    const int32_t a = cand_side(key);
    int64_t cnt = 0;
    int k2 = k + 1;
    for (; k2 < s && (buf[k2] >> 26) == (key >> 26); ++k2) {  // same hash, same deleted position
        emit(a, cand_side(buf[k2]));
        ++cnt;
    }
    if (T >= 1 && rec_runstart(key)) {
        int g = k2;
        while (g < s && (buf[g] >> 32) == (key >> 32)) ++g;
        for (int f = g - 1; f >= k2 && rec_p(buf[f]) == kTagF; --f) {
            emit(cand_side(buf[f]), a);
            ++cnt;
        }
    }
    return cnt;
}

// W_u += m_v and W_v += m_u for an edge {u, v}.
struct Weigh {
    const int32_t* umult;
    int32_t* wsum;
    __device__ __forceinline__ void operator()(int32_t a, int32_t b) const {
        atomicAdd(&wsum[a], umult[b]);
        atomicAdd(&wsum[b], umult[a]);
    }
};

// The partitions that k_join_small leaves to the other two joins, listed
// before it runs (from the partition offsets, while the records are
// scattered): more than cap records for k_join_fallback, 33..cap for
// k_join_sorted, so that those joins can run beside k_join_small on a side
// stream. One atomic per warp and list.
__global__ void k_part_classes(const int64_t* __restrict__ poff, int64_t P, int cap, int32_t* __restrict__ big_list,
                               int* __restrict__ big_count, int32_t* __restrict__ fb_list, int* __restrict__ fb_count) {
    const int lane = threadIdx.x & 31;
    for (int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; p0 < P;
         p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + lane;
        const int64_t sz = p < P ? poff[p + 1] - poff[p] : 0;
        const bool fb = sz > cap, big = !fb && sz > 32;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool mine = l ? fb : big;
            const uint32_t m = __ballot_sync(kFull, mine);
            if (m) {
                const int lead = __ffs(m) - 1;
                int base = 0;
                if (lane == lead) base = atomicAdd(l ? fb_count : big_count, __popc(m));
                base = __shfl_sync(kFull, base, lead);
                if (mine) (l ? fb_list : big_list)[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
            }
        }
    }
}

// Join of the partitions of at most 32 records, without sorting. The records
// of consecutive partitions are adjacent, so a warp step takes a window of
// whole consecutive partitions holding at most 32 records: lane k holds record
// k of the window. __match_any_sync on the 32-bit hash, restricted to the
// lanes of the record's own partition, gives each lane its hash group G, and
// G intersected with a match on p its run M of equal (hash, p) (two 32-bit
// matches cost less than one on the 38-bit pair, measured). Same-position
// candidates are the lanes of M above this one (each pair once); a run-start
// deletion pairs with every full record of G. No content is read here: the
// candidates are confirmed by k_confirm, so this pass streams the records and
// issues only shuffles, votes and stores. Larger partitions are listed for
// k_join_sorted / k_join_fallback (first pass) and skipped here; both passes
// form the same windows, so their counts agree.
// First pass (WRITE = false): candidate counts (a window's total at its first
// partition, 0 at the others) and every candidate written into the capped
// segmented buffer when it fits; a warp gathers its candidates in shared
// memory and moves them out kStage at a time (one cursor update per flush,
// coalesced stores). Second pass (WRITE = true, only after an overflow):
// candidates written at the scanned positions eoff. The records of the next
// window are loaded while the current one is joined.
constexpr int kStage = 256;

template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_join_small(const int64_t* __restrict__ poff, int64_t P, const uint64_t* __restrict__ recs, int cap, int T,
             int64_t* __restrict__ pedges, const int64_t* __restrict__ eoff, int2* __restrict__ edges,
             unsigned long long* __restrict__ ecur, int64_t seg_cap, int32_t* __restrict__ big_list,
             int* __restrict__ big_count, int32_t* __restrict__ fb_list, int* __restrict__ fb_count,
             int64_t R_cap = INT64_MAX) {
    dep_entry();  // launched dependent on the kernel before it
    if (poff[P] > R_cap) return;  // records beyond the array (invalid input): nothing is joined
    __shared__ uint64_t sbuf[kWarps][32];
    __shared__ int2 sstage[WRITE ? 1 : kWarps][WRITE ? 1 : kStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* buf = sbuf[warp];
    int2* stage = sstage[WRITE ? 0 : warp];
    const uint32_t above = lane == 31 ? 0u : ~((2u << lane) - 1u);
    const uint32_t upto = lane == 31 ? kFull : ((2u << lane) - 1u);  // lanes 0 .. lane
    const uint32_t below = (1u << lane) - 1u;
    const int64_t wid = (int64_t)blockIdx.x * kWarps + warp;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    const int seg = (int)(wid & (kEdgeSegs - 1));
    const int small_max = cap < 32 ? cap : 32;
    int fillc = 0;  // staged candidates of this warp
    auto flush = [&]() {
        __syncwarp();
        if (fillc) {
            unsigned long long eb = 0;
            if (lane == 0) eb = atomicAdd(&ecur[seg], (unsigned long long)fillc);
            eb = __shfl_sync(kFull, eb, 0);
            if ((int64_t)(eb + fillc) <= seg_cap) {
                int2* dst = edges + seg * seg_cap + (int64_t)eb;
                for (int k = lane; k < fillc; k += 32) dst[k] = stage[k];
            }
            fillc = 0;
        }
        __syncwarp();
    };
    for (int64_t p0 = wid * 32; p0 < P; p0 += nwarps * 32) {
        // lane k: partition p0 + k
        int64_t my_base = 0;
        int my_size = 0;
        if (p0 + lane < P) {
            my_base = poff[p0 + lane];
            const int64_t sz = poff[p0 + lane + 1] - my_base;
            my_size = sz > 0x7fffffff ? 0x7fffffff : (int)sz;
        }
        const bool wable = p0 + lane < P && my_size <= small_max;  // joined in a window here
        if (!WRITE && p0 + lane < P) {  // lane-parallel hand-off of the other partitions (unless listed before)
            if (my_size > cap) {
                if (fb_list) fb_list[atomicAdd(fb_count, 1)] = (int32_t)(p0 + lane);
            } else if (my_size > 32) {
                if (big_list) big_list[atomicAdd(big_count, 1)] = (int32_t)(p0 + lane);
            } else {
                pedges[p0 + lane] = 0;  // a window's first partition overwrites it with the window's count
            }
        }
        const uint32_t wmask = __ballot_sync(kFull, wable);
        const int wsize = wable ? my_size : 0;
        int incl = wsize;  // inclusive prefix of the window-able sizes (each <= 32)
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        // the window starting at the first window-able lane >= from: partitions
        // j .. e (consecutive, all window-able, at most 32 records), records
        // [rb, rb + tot); false when no lane is left
        auto window = [&](int from, int& j, int& e, int& tot, int64_t& rb) -> bool {
            const uint32_t cand = from >= 32 ? 0u : (wmask & ~((1u << from) - 1u));
            if (!cand) return false;
            j = __ffs(cand) - 1;
            const uint32_t stops = ~wmask & (j == 31 ? 0u : ~((2u << j) - 1u));
            const int nb = stops ? __ffs(stops) - 1 : 32;  // first partition over the window size after j
            const int excl_j = __shfl_sync(kFull, incl - wsize, j);
            const uint32_t fit = __ballot_sync(kFull, lane >= j && lane < nb && incl - excl_j <= 32);
            e = 31 - __clz(fit);
            tot = __shfl_sync(kFull, incl, e) - excl_j;
            rb = __shfl_sync(kFull, my_base, j);
            return true;
        };
        int j = 0, e = 0, tot = 0;
        int64_t rb = 0;
        bool have = window(0, j, e, tot, rb);
        uint64_t rec_next = (have && lane < tot) ? recs[rb + lane] : ~0ull;
        while (have) {
            const int wj = j, we = e, s = tot;
            const uint64_t rec = rec_next;
            // record lanes of each partition: bit (start offset) of every non-empty one
            const int excl_j = __shfl_sync(kFull, incl - wsize, wj);
            const uint32_t starts = __reduce_or_sync(
                kFull, (lane >= wj && lane <= we && wsize > 0) ? (1u << (incl - wsize - excl_j)) : 0u);
            have = window(we + 1, j, e, tot, rb);
            rec_next = (have && lane < tot) ? recs[rb + lane] : ~0ull;  // prefetch the next window
            if (s < 2) continue;  // no pair in this window (its partitions' counts stay 0)
            const bool act = lane < s;
            // lanes [a, b) hold this record's partition
            const uint32_t st_upto = starts & upto;
            const int a = st_upto ? 31 - __clz(st_upto) : 0;
            const uint32_t st_above = starts & above;
            const int b = st_above ? __ffs(st_above) - 1 : s;
            const uint32_t pmask = (b >= 32 ? kFull : ((1u << b) - 1u)) & ~((1u << a) - 1u);
            buf[lane] = rec;
            const uint32_t amask = (s >= 32) ? kFull : ((1u << s) - 1u);
            const uint32_t G = __match_any_sync(kFull, (uint32_t)(rec >> 32)) & amask & pmask;
            // no two records of a partition share a hash: the window has no candidate
            // (its partitions' counts stay 0)
            if (!__any_sync(kFull, (G & ~(1u << lane)) != 0u)) continue;
            const uint32_t M = G & __match_any_sync(kFull, rec_p(rec));  // same hash and same p
            const bool isF = rec_p(rec) == kTagF;
            const uint32_t Gf = G & __ballot_sync(kFull, act && isF);
            const uint32_t partners = (act && !isF) ? (M & above) : 0u;
            const uint32_t fulls = (act && !isF && T >= 1 && rec_runstart(rec)) ? Gf : 0u;
            // prefix sum of the per-lane counts (<= 63) by bit planes: votes and
            // population counts instead of shuffles
            const int mine = __popc(partners) + __popc(fulls);
            int excl = 0, total = 0;
#pragma unroll
            for (int bp = 0; bp < 6; ++bp) {
                const uint32_t plane = __ballot_sync(kFull, (mine >> bp) & 1);
                excl += __popc(plane & below) << bp;
                total += __popc(plane) << bp;
            }
            __syncwarp();  // buf written by every lane
            const int32_t me = cand_side(rec);
            if (!WRITE) {
                if (lane == wj) pedges[p0 + wj] = total;
                if (total) {
                    // staged (total <= kStage) or written directly with its own cursor update
                    if (fillc + total > kStage) flush();
                    int2* dst = stage + fillc + excl;
                    bool fits = true;
                    if (total > kStage) {
                        unsigned long long eb = 0;
                        if (lane == 0) eb = atomicAdd(&ecur[seg], (unsigned long long)total);
                        eb = __shfl_sync(kFull, eb, 0);
                        fits = (int64_t)(eb + total) <= seg_cap;
                        dst = edges + seg * seg_cap + (int64_t)eb + excl;
                    } else {
                        fillc += total;
                    }
                    if (fits) {
                        for (uint32_t m = partners; m; m &= m - 1) *dst++ = make_int2(me, cand_side(buf[__ffs(m) - 1]));
                        for (uint32_t m = fulls; m; m &= m - 1) *dst++ = make_int2(cand_side(buf[__ffs(m) - 1]), me);
                    }
                }
            } else if (mine) {
                int64_t pos = eoff[p0 + wj] + excl;
                for (uint32_t m = partners; m; m &= m - 1) edges[pos++] = make_int2(me, cand_side(buf[__ffs(m) - 1]));
                for (uint32_t m = fulls; m; m &= m - 1) edges[pos++] = make_int2(cand_side(buf[__ffs(m) - 1]), me);
            }
            __syncwarp();
        }
    }
    if (!WRITE) flush();
}

// Join of the listed partitions of 33 .. cap records: warp per partition,
// register bitonic sort, runs of equal (hash, p) and hash groups scanned in
// order (record_cands); candidates as in k_join_small.
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_join_sorted(const int32_t* __restrict__ list, const int* __restrict__ count, const int64_t* __restrict__ poff,
              const uint64_t* __restrict__ recs, int T, int64_t* __restrict__ pedges,
              const int64_t* __restrict__ eoff, int2* __restrict__ edges, unsigned long long* __restrict__ ecur,
              int64_t seg_cap) {
    dep_entry();  // launched dependent on the kernel before it
    __shared__ uint64_t sbuf[kWarps][kWarpCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* buf = sbuf[warp];
    const int nlist = *count;
    for (int f = blockIdx.x * kWarps + warp; f < nlist; f += gridDim.x * kWarps) {
        const int64_t pid = list[f];
        const int64_t base = poff[pid];
        const int s = (int)(poff[pid + 1] - base);
        if (s <= 64) load_sort_store<2>(recs + base, s, buf, lane);
        else load_sort_store<4>(recs + base, s, buf, lane);
        __syncwarp();
        int64_t mine = 0;
        for (int k = lane; k < s; k += 32) mine += record_cands(buf, k, s, T, [](int32_t, int32_t) {});
        int64_t excl;
        const int64_t total = warp_scan(mine, excl, lane);
        if (!WRITE) {
            if (lane == 0) pedges[pid] = total;
            if (total) {
                const int seg = (int)(pid & (kEdgeSegs - 1));
                unsigned long long eb = 0;
                if (lane == 0) eb = atomicAdd(&ecur[seg], (unsigned long long)total);
                eb = __shfl_sync(kFull, eb, 0);
                if ((int64_t)(eb + total) <= seg_cap) {
                    int64_t pos = seg * seg_cap + (int64_t)eb + excl;
                    for (int k = lane; k < s; k += 32)
                        record_cands(buf, k, s, T, [&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
                }
            }
        } else {
            int64_t pos = eoff[pid] + excl;
            for (int k = lane; k < s; k += 32)
                record_cands(buf, k, s, T, [&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
        }
        __syncwarp();
    }
}

// Join of one partition over the warp capacity (cap records): a block tests
// every pair of its records for the candidate conditions (equal 32-bit hash
// and equal p, or a run-start deletion and a full record of equal hash),
// without sorting; candidates as in k_join_small.
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_join_fallback(const int32_t* __restrict__ fb_list, const int* __restrict__ fb_count, const int64_t* __restrict__ poff,
                const uint64_t* __restrict__ recs, int T, int64_t* __restrict__ pedges,
                const int64_t* __restrict__ eoff, int2* __restrict__ edges, unsigned long long* __restrict__ ecur,
                int64_t seg_cap) {
    dep_entry();  // launched dependent on the kernel before it
    __shared__ int64_t wtot[kWarps];
    __shared__ unsigned long long sbase;
    const int nfb = *fb_count;
    for (int f = blockIdx.x; f < nfb; f += gridDim.x) {
        const int64_t pid = fb_list[f];
        const int64_t base = poff[pid];
        const int64_t s = poff[pid + 1] - base;
        auto scan_pairs = [&](auto emit) {
            int64_t cnt = 0;
            for (int64_t k1 = threadIdx.x; k1 < s; k1 += kThreads) {
                const uint64_t r1 = recs[base + k1];
                if (rec_p(r1) == kTagF) continue;  // deletion records initiate every candidate
                const bool rs1 = T >= 1 && rec_runstart(r1);
                for (int64_t k2 = 0; k2 < s; ++k2) {
                    const uint64_t r2 = recs[base + k2];
                    if ((r2 >> 32) != (r1 >> 32) || k2 == k1) continue;
                    const uint32_t p2 = rec_p(r2);
                    if (p2 == rec_p(r1) && k2 > k1) {
                        emit(cand_side(r1), cand_side(r2));
                        ++cnt;
                    } else if (rs1 && p2 == kTagF) {
                        emit(cand_side(r2), cand_side(r1));
                        ++cnt;
                    }
                }
            }
            return cnt;
        };
        const int64_t mine = scan_pairs([](int32_t, int32_t) {});
        int64_t excl;
        const int64_t total = block_scan(mine, excl, wtot);
        if (!WRITE) {
            if (threadIdx.x == 0) pedges[pid] = total;
            if (total) {
                const int seg = (int)(pid & (kEdgeSegs - 1));
                if (threadIdx.x == 0) sbase = atomicAdd(&ecur[seg], (unsigned long long)total);
                __syncthreads();
                if ((int64_t)(sbase + total) <= seg_cap) {
                    int64_t pos = seg * seg_cap + (int64_t)sbase + excl;
                    scan_pairs([&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
                }
            }
        } else {
            int64_t pos = eoff[pid] + excl;
            scan_pairs([&](int32_t a, int32_t b) { edges[pos++] = make_int2(a, b); });
        }
        __syncthreads();
    }
}

// Confirmation of the join's candidates: the two variants an entry names are
// compared by content; a match becomes the plain edge (u, v) and adds
// W_u += m_v, W_v += m_u, a mismatch (equal 32-bit hashes of different
// contents) becomes (-1, -1) and is counted. One thread per entry, so the
// random reads of the two strings are many in flight at once. Over the
// segmented one-pass buffer (grid.y = segment) nothing is done when a segment
// overflowed: the second join pass then writes the complete list and this
// kernel runs on it.
__global__ void k_confirm(int2* __restrict__ edges, int64_t seg_cap, const unsigned long long* __restrict__ seg_count,
                          int check_overflow, const Canon* __restrict__ ucanon, Weigh weigh,
                          int* __restrict__ false_count) {
    dep_entry();  // launched dependent on the kernel before it
    if (check_overflow) {
        __shared__ int over;
        if (threadIdx.x == 0) over = 0;
        __syncthreads();
        if (threadIdx.x < kEdgeSegs && (int64_t)seg_count[threadIdx.x] > seg_cap) over = 1;
        __syncthreads();
        if (over) return;
    }
    const int64_t E = (int64_t)seg_count[blockIdx.y];
    int2* seg = edges + blockIdx.y * seg_cap;
    // two entries per step: their loads are in flight together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < E; t += 2 * stride) {
        const int64_t t2 = t + stride;
        const bool two = t2 < E;
        const int2 e1 = seg[t];
        const int2 e2 = two ? seg[t2] : e1;
        const int32_t a1 = e1.x & (int32_t)kUMask, b1 = e1.y & (int32_t)kUMask;
        const int32_t a2 = e2.x & (int32_t)kUMask, b2 = e2.y & (int32_t)kUMask;
        Canon ca1 = load_canon(ucanon + a1), cb1 = load_canon(ucanon + b1);
        Canon ca2 = load_canon(ucanon + a2), cb2 = load_canon(ucanon + b2);
        auto variant = [](Canon& c, int32_t side) {
            const uint32_t p = (uint32_t)side >> 25;
            if (p != kTagF) c = delete_at(c, (int)p);
        };
        variant(ca1, e1.x);
        variant(cb1, e1.y);
        variant(ca2, e2.x);
        variant(cb2, e2.y);
        auto finish = [&](int64_t k, int32_t a, int32_t b, bool same) {
            if (same) {
                weigh(a, b);
                seg[k] = make_int2(a, b);
            } else {
                seg[k] = make_int2(-1, -1);
                atomicAdd(false_count, 1);
            }
        };
        finish(t, a1, b1, canon_eq(ca1, cb1));
        if (two) finish(t2, a2, b2, canon_eq(ca2, cb2));
    }
}

// ---- 3'. l_max = 2: candidates from shared variants of up to two deletions --
//
// lev(a, b) <= 2 is at most two edits; a substitution at position i is the
// deletion of i from both strings and an insertion into one the deletion of a
// letter of the other, so a and b have equal variants with at most two
// deletions each. Every pair of distinct strings with a variant of equal
// 32-bit hash in the same partition is a candidate (a hash collision only
// adds a candidate); candidates are deduplicated and each one is checked with
// the exact bit-parallel distance, so the edges are exact. Deletions inside a
// run of equal letters start at the run (two from one run: its first two),
// which drops most repeated variants of a string.

// fn(v) for the full string, every run-start deletion and every canonical
// pair of deletions of c (length L).
template <typename Fn>
__device__ __forceinline__ void for_variants2(const Canon& c, int L, Fn fn) {
    fn(c);
    for (int p = 0; p < L; ++p) {
        if (!run_start(c, p)) continue;
        const Canon d = delete_at(c, p);
        fn(d);
        for (int q = p + 1; q < L; ++q)
            if (q == p + 1 || run_start(c, q)) fn(delete_at(d, q - 1));  // position q of c is q - 1 of d
    }
}

// Variants per distinct string (their sum sizes the records).
__global__ void k_var2_count(const Canon* __restrict__ ucanon, const uint8_t* __restrict__ ulen,
                             const int64_t* __restrict__ U_ptr, int64_t n, unsigned long long* __restrict__ total) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (u < n && u < *U_ptr) {
        const Canon c = load_canon(ucanon + u);
        const int L = ulen[u];
        cnt = 1;
        for (int p = 0; p < L; ++p) {
            if (!run_start(c, p)) continue;
            ++cnt;
            for (int q = p + 1; q < L; ++q) cnt += (q == p + 1 || run_start(c, q)) ? 1 : 0;
        }
    }
    // one atomic per warp
    int x = cnt;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(total, (unsigned long long)x);
}

// Records (low 32 hash bits | u) of every variant: count per partition, or
// scatter at slots from per-partition cursors.
template <bool SCATTER>
__global__ void k_var2_records(const Canon* __restrict__ ucanon, const uint8_t* __restrict__ ulen,
                               const int64_t* __restrict__ U_ptr, int64_t n, uint32_t P, int32_t* __restrict__ pcnt,
                               const int64_t* __restrict__ poff, uint64_t* __restrict__ recs) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || u >= *U_ptr) return;
    const Canon c = load_canon(ucanon + u);
    for_variants2(c, ulen[u], [&](const Canon& v) {
        const uint64_t h = hash_canon(v);
        const uint32_t pid = part_of(h, P);
        if constexpr (!SCATTER) {
            atomicAdd(&pcnt[pid], 1);
        } else {
            recs[poff[pid] + atomicAdd(&pcnt[pid], 1)] = (h << 32) | (uint64_t)u;
        }
    });
}

// Candidate pairs of every partition: records of equal hash and different
// strings, filed under the smaller string. COUNT adds one to rcnt[u] per
// candidate {u, v} (u < v); WRITE stores v at coff[u] + a slot taken from
// rcnt[u], so rows fill without a shared cursor. A warp takes a partition:
// up to 32 records at once with two match steps (equal hash, equal record),
// larger ones 32 by 32 records.
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_var2_pairs(const int64_t* __restrict__ poff, int64_t P, const uint64_t* __restrict__ recs,
             int32_t* __restrict__ rcnt, const int64_t* __restrict__ coff, int32_t* __restrict__ ccols) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto emit = [&](uint32_t a, uint32_t b) {
        const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
        if constexpr (!WRITE) atomicAdd(&rcnt[lo], 1);
        else ccols[coff[lo] + atomicAdd(&rcnt[lo], 1)] = (int32_t)hi;
    };
    for (int64_t pid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pid < P; pid += nw) {
        const int64_t b0 = poff[pid], b1 = poff[pid + 1];
        if (b1 - b0 < 2) continue;
        if (b1 - b0 <= 32) {
            const bool valid = b0 + lane < b1;
            const uint64_t r = valid ? recs[b0 + lane] : 0;
            const unsigned vmask = __ballot_sync(kFull, valid);
            const unsigned peers = __match_any_sync(kFull, (uint32_t)(r >> 32)) & vmask;
            const unsigned same = __match_any_sync(kFull, (unsigned long long)r) & vmask;
            // lanes above this one with the same hash and another string
            unsigned bits = valid ? peers & ~same & ((~0u << lane) << 1) : 0u;
            const uint32_t u = (uint32_t)r;
            while (__any_sync(kFull, bits)) {
                const int j = bits ? __ffs(bits) - 1 : lane;
                const uint32_t uj = __shfl_sync(kFull, u, j);
                if (bits) {
                    emit(u, uj);
                    bits &= bits - 1;
                }
            }
            continue;
        }
        for (int64_t i0 = b0; i0 < b1; i0 += 32) {
            const int64_t i = i0 + lane;
            const uint64_t ri = i < b1 ? recs[i] : ~0ull;
            for (int64_t j0 = i0; j0 < b1; j0 += 32) {
                const uint64_t rj = j0 + lane < b1 ? recs[j0 + lane] : ~0ull;
                for (int t = 0; t < 32; ++t) {
                    const uint64_t r = __shfl_sync(kFull, rj, t);
                    const int64_t j = j0 + t;
                    if (i < b1 && j < b1 && j > i && (r >> 32) == (ri >> 32) && (uint32_t)r != (uint32_t)ri)
                        emit((uint32_t)ri, (uint32_t)r);
                }
            }
        }
    }
}

// Each distinct candidate (row u sorted, repeats adjacent) checked with the
// bit-parallel distance (Myers 1999, Hyyro 2001). A warp walks rows and
// queues their distinct candidates; each full queue of 32 is checked with one
// pair per lane: the lane builds the letter masks of its u in its own column
// of shared memory and runs the recurrence over v. Pairs within l_max = 2 (and
// of one repertoire) become edges {u, v} with their weights; a warp gathers
// its edges in shared memory and appends them at *ecur a hundred or so at a
// time (one atomic each).
constexpr int kVerifyWarps = 4;
constexpr int kVerifyBuf = 128;
constexpr int kSigma = 20;  // letter codes 1..20
__global__ void __launch_bounds__(32 * kVerifyWarps)
k_cand_verify(const int64_t* __restrict__ coff, const int32_t* __restrict__ ccols, const int64_t* __restrict__ U_ptr,
              const Canon* __restrict__ ucanon, const uint8_t* __restrict__ ulen, Weigh weigh, int2* __restrict__ edges,
              unsigned long long* __restrict__ ecur, int64_t cap, int* __restrict__ err) {
    __shared__ uint64_t peq[kVerifyWarps][kSigma][32];
    __shared__ int2 queue[kVerifyWarps][64];
    __shared__ int2 ebuf[kVerifyWarps][kVerifyBuf];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t U = *U_ptr;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int qn = 0, fill = 0;  // queued pairs, buffered edges (warp-uniform)
    auto flush = [&]() {
        unsigned long long base = 0;
        if (lane == 0 && fill) base = atomicAdd(ecur, (unsigned long long)fill);
        base = __shfl_sync(kFull, base, 0);
        for (int k = lane; k < fill; k += 32) {
            const unsigned long long slot = base + (unsigned long long)k;
            if ((int64_t)slot < cap) edges[slot] = ebuf[w][k];
            else atomicExch(err, 1);
        }
        __syncwarp();
        fill = 0;
    };
    auto check = [&](int cnt) {  // queue[0 .. cnt), cnt <= 32
        bool edge = false;
        int2 uv = make_int2(0, 0);
        if (lane < cnt) {
            uv = queue[w][lane];
            const Canon cu = load_canon(ucanon + uv.x), cv = load_canon(ucanon + uv.y);
            const int Lu = ulen[uv.x], Lv = ulen[uv.y];
            const uint64_t tags = ((cu.w[0] ^ cv.w[0]) | (cu.w[1] ^ cv.w[1]) | (cu.w[2] ^ cv.w[2]) |
                                   (cu.w[3] ^ cv.w[3])) & kTagBits;
            if (tags == 0 && Lv - Lu <= 2 && Lu - Lv <= 2) {
#pragma unroll
                for (int c = 0; c < kSigma; ++c) peq[w][c][lane] = 0;
                for (int k = 0; k < Lu; ++k) peq[w][code_at(cu, k) - 1][lane] |= 1ull << k;
                const uint64_t top = 1ull << (Lu - 1);
                uint64_t vp = ~0ull, vn = 0;
                int score = Lu;
                for (int k = 0; k < Lv; ++k) {
                    const uint64_t eq = peq[w][code_at(cv, k) - 1][lane];
                    const uint64_t xv = eq | vn;
                    const uint64_t xh = (((eq & vp) + vp) ^ vp) | eq;
                    uint64_t hp = vn | ~(xh | vp);
                    uint64_t hn = vp & xh;
                    score += ((hp & top) ? 1 : 0) - ((hn & top) ? 1 : 0);
                    hp = (hp << 1) | 1ull;
                    hn <<= 1;
                    vp = hn | ~(xv | hp);
                    vn = hp & xv;
                }
                edge = score <= 2;
            }
        }
        const unsigned hits = __ballot_sync(kFull, edge);
        if (edge) {
            ebuf[w][fill + __popc(hits & lanemask_lt())] = uv;
            weigh(uv.x, uv.y);
        }
        fill += __popc(hits);
        __syncwarp();
        if (fill > kVerifyBuf - 32) flush();
    };
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < U; u += nw) {
        const int64_t a = coff[u], b = coff[u + 1];
        for (int64_t e0 = a; e0 < b; e0 += 32) {
            const int64_t e = e0 + lane;
            int32_t v = -1;
            bool first = false;
            if (e < b) {
                v = ccols[e];
                first = e == a || ccols[e - 1] != v;  // first of its repeats
            }
            const unsigned m = __ballot_sync(kFull, first);
            if (first) queue[w][qn + __popc(m & lanemask_lt())] = make_int2((int32_t)u, v);
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                check(32);
                const int rest = qn - 32;
                const int2 t = lane < rest ? queue[w][32 + lane] : make_int2(0, 0);
                __syncwarp();
                if (lane < rest) queue[w][lane] = t;
                __syncwarp();
                qn = rest;
            }
        }
    }
    if (qn) check(qn);
    __syncwarp();
    flush();
}

// ---- 4. closed neighbourhoods ---------------------------------------------

// D_u = m_u + W_u (written into wsum in place); the largest D_u into *dmax.
__global__ void k_closed_size(const int32_t* __restrict__ umult, int64_t U, int32_t* __restrict__ wsum,
                              int* __restrict__ dmax) {
    dep_entry();  // launched dependent on the kernel before it
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int d = 0;
    if (u < U) {
        d = wsum[u] + umult[u];
        wsum[u] = d;
    }
    // block maximum, then one atomic per block
    __shared__ int wmax[kWarps];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(kFull, d, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x < 32) {
        d = threadIdx.x < kWarps ? wmax[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(kFull, d, o));
        if (threadIdx.x == 0 && d > 0) atomicMax(dmax, d);
    }
}

// Sizes of the closed lists and of the CSR rows with both offset scans, in
// one launch of two independent look-back chains (lookback.cuh), blockIdx.y:
// (chain 0 also lists the long lists by row-sort class into cls_lists[c * n
// + k], counts cls_cnt[c], for a list sort whose classes then start together)
// chain 0 scans D_u = m_u + W_u over the string ids u < n (list offsets uoff;
// the list cursors start after the own members, at the absolute position
// ucur_u = uoff_u + m_u (64-bit: the appends' atomics return positions in S,
// no offset load); the largest D_u
// into *dmax), chain 1 scans d(i) = D_{u(i)} - 1 over the nodes (CSR offsets
// off64, and the degree array). In place of k_closed_size, k_node_degree and
// two scans (four launches, two look-back latencies in a row).
__global__ void __launch_bounds__(kScanThreads)
k_fill_sizes(const int32_t* __restrict__ wsum, const int32_t* __restrict__ umult, const int32_t* __restrict__ uid,
             int64_t n, unsigned long long* __restrict__ ucur, int* __restrict__ dmax, int32_t* __restrict__ deg,
             int64_t* __restrict__ uoff, int64_t* __restrict__ off64, unsigned long long* st_u,
             unsigned long long* st_n, int64_t tiles, int32_t* __restrict__ cls_lists, int* __restrict__ cls_cnt) {
    dep_entry();  // launched dependent on the kernel before it
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t stage[kScanStage];
    __shared__ int64_t s_prefix;
    __shared__ int64_t s_tile;
    __shared__ int s_max[kScanThreads / 32];
    const bool nodes = blockIdx.y == 1;
    unsigned long long* status = nodes ? st_n : st_u;
    int64_t* out = nodes ? off64 : uoff;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(status + tiles, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile;
    int dm = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = k * kScanThreads + threadIdx.x;
        const int64_t i = base + idx;
        int32_t v = 0;
        if (i < n) {
            if (nodes) {
                const int32_t u = uid[i];
                v = wsum[u] + umult[u] - 1;
                deg[i] = v;
            } else {
                v = wsum[i] + umult[i];
                dm = max(dm, v);
            }
        }
        if (!nodes && cls_cnt) {  // long lists listed for their sort class, one atomic per warp and class
            const int c = (i < n && v >= kSortWideMin) ? (v >= kSortBigMin ? 2 : (v >= kSortMidMin ? 1 : 0)) : -1;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const uint32_t m = __ballot_sync(kFull, c == cc);
                if (m) {
                    const int lead = __ffs(m) - 1;
                    int base = 0;
                    if ((int)(threadIdx.x & 31) == lead) base = atomicAdd(&cls_cnt[cc], __popc(m));
                    base = __shfl_sync(kFull, base, lead);
                    if (c == cc) cls_lists[cc * n + base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = (int32_t)i;
                }
            }
        }
        stage[scan_slot(idx)] = v;
    }
    if (!nodes) {  // block maximum of D_u, one atomic per block
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dm = max(dm, __shfl_xor_sync(kFull, dm, o));
        if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = dm;
    }
    __syncthreads();
    if (!nodes && threadIdx.x < 32) {
        int d = threadIdx.x < kScanThreads / 32 ? s_max[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(kFull, d, o));
        if (threadIdx.x == 0 && d > 0) atomicMax(dmax, d);
    }
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = stage[scan_slot(threadIdx.x * kScanItems + k)];
        sum += v[k];
    }
    int64_t excl;
    const int64_t tot = scan_block_exclusive(sum, excl, warp_tot);
    if (threadIdx.x < 32) {
        const int64_t prefix = scan_lookback(tile, tot, status, tiles);
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    int64_t run = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        stage[scan_slot(threadIdx.x * kScanItems + k)] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) {
            const int64_t o = stage[scan_slot(k * kScanThreads + threadIdx.x)];
            out[i] = o;
            if (!nodes) ucur[i] = (unsigned long long)(o + umult[i]);
        }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) out[n] = s_prefix + tot;  // the grand total
}

// List cursors after the own members (the single-tile path of the sizes).
__global__ void k_list_cursors(const int64_t* __restrict__ uoff, const int32_t* __restrict__ umult, int64_t n,
                               unsigned long long* __restrict__ ucur) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) ucur[u] = (unsigned long long)(uoff[u] + umult[u]);
}

__global__ void k_node_degree(const int32_t* __restrict__ uid, int64_t n, const int32_t* __restrict__ dsize,
                              int32_t* __restrict__ deg) {
    dep_entry();  // launched dependent on the kernel before it
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) deg[i] = dsize[uid[i]] - 1;
}

// Edges of the segmented join buffer moved next to each other (kept by a
// build handle: the network of distinct strings).
struct SegBases {
    int64_t base[kEdgeSegs + 1];
};

__global__ void k_compact_edges(const int2* __restrict__ edges, int64_t seg_cap, SegBases b, int2* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (t < b.base[g + 1] - b.base[g]) out[b.base[g] + t] = edges[(int64_t)g * seg_cap + t];
}

// The confirmed edges of a list that holds rejected candidates ((-1, -1)),
// gathered at a shared cursor (grid.y = segment).
__global__ void k_gather_edges(const int2* __restrict__ edges, int64_t seg_cap,
                               const unsigned long long* __restrict__ seg_count, int2* __restrict__ out,
                               unsigned long long* __restrict__ cursor) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)seg_count[blockIdx.y]) return;
    const int2 e = edges[(int64_t)blockIdx.y * seg_cap + t];
    if (e.x >= 0) out[atomicAdd(cursor, 1ull)] = e;
}

__global__ void k_closed_self(const int32_t* __restrict__ uid, const int32_t* __restrict__ mpos, int64_t n,
                              const int64_t* __restrict__ uoff, int32_t* __restrict__ S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) S[uoff[uid[i]] + mpos[i]] = (int32_t)i;
}

// Append M_b to the list of a for both directions of every edge. Lanes copy
// short member lists themselves; long ones are copied by the whole warp.
__global__ void __launch_bounds__(kThreads)
k_closed_edges(const int2* __restrict__ edges, int64_t seg_cap, const unsigned long long* __restrict__ seg_count,
               const int32_t* __restrict__ umult,
               const int64_t* __restrict__ mem_off, const int32_t* __restrict__ members,
               unsigned long long* __restrict__ ucur, int32_t* __restrict__ S, int64_t SD, int* __restrict__ err) {
    constexpr int kShort = 8;  // (4: list fill 0.102 ms at 8e5; 8: 0.099; 16: 0.100)
    const int lane = threadIdx.x & 31;
    // grid.y = edge segment; t = direction-expanded index inside the segment
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t E = (int64_t)seg_count[blockIdx.y];
    bool have = t < 2 * E;
    int32_t a = 0, b = 0, mb = 0;
    int64_t o = 0;
    int2 uv = make_int2(-1, -1);
    if (have) uv = edges[blockIdx.y * seg_cap + (t >> 1)];
    have = have && uv.x >= 0;  // a rejected candidate of the join is no edge
    if (have) {
        a = (t & 1) ? uv.y : uv.x;  // list owner
        b = (t & 1) ? uv.x : uv.y;  // neighbour whose members are appended
        mb = umult[b];
        // a short member list is loaded before the slot atomic returns
        const int32_t* rb = members + mem_off[b];
        int32_t mv[kShort];
#pragma unroll
        for (int y = 0; y < kShort; ++y) mv[y] = y < mb ? rb[y] : 0;
        o = (int64_t)atomicAdd(&ucur[a], (unsigned long long)mb);
        if (o + mb > SD) {  // (weights that disagree with the list: an error, never a write past S)
            atomicExch(err, 1);
            mb = 0;
        }
        if (mb <= kShort) {
#pragma unroll
            for (int y = 0; y < kShort; ++y)
                if (y < mb) S[o + y] = mv[y];
        }
    }
    unsigned longs = __ballot_sync(kFull, have && mb > kShort);
    while (longs) {
        const int src = __ffs(longs) - 1;
        longs &= longs - 1;
        const int32_t lb = __shfl_sync(kFull, b, src);
        const int32_t lm = __shfl_sync(kFull, mb, src);
        const int64_t lo = __shfl_sync(kFull, o, src);
        const int32_t* rb = members + mem_off[lb];
        for (int32_t y = lane; y < lm; y += 32) S[lo + y] = rb[y];
    }
}

// ---- 5. expand --------------------------------------------------------------

// Row i = sorted S_u without i. A warp takes 32 rows: each lane fetches one
// row's list bounds (independent loads in parallel); rows of at most
// kLaneRow entries are copied by their own lane, longer ones by the whole warp
// one after another, lanes along the row. S_u is sorted and contains i once,
// so element x at position k goes to k - (x > i).
constexpr int kLaneRow = 16;
constexpr int kExpVec = 4;  // entries per lane of a long row in flight (8 measured slower)
constexpr int kExpChunk = 32 * kExpVec;

__global__ void k_expand(const int32_t* __restrict__ uid, int64_t n, const int64_t* __restrict__ uoff,
                         const int32_t* __restrict__ S, const int64_t* __restrict__ off, int32_t* __restrict__ cols) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = w0 * 32; r0 < n; r0 += nw * 32) {
        const int64_t my = r0 + lane;
        int64_t s0 = 0, D = 0, o = 0;
        if (my < n) {
            const int32_t u = uid[my];
            s0 = uoff[u];
            D = uoff[u + 1] - s0;
            o = off[my];
        }
        if (D >= 2 && D <= kLaneRow + 1) {
            // S_u is sorted and holds i: an entry above i moves one slot left,
            // so the slots are known and eight loads go out before their stores
            const int32_t me = (int32_t)my;
            const int32_t* su = S + s0;
            int32_t* row = cols + o;
            const int iD = (int)D;
            for (int k0 = 0; k0 < iD; k0 += 8) {
                int32_t y[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) y[t] = k0 + t < iD ? su[k0 + t] : me;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int q = k0 + t - (y[t] > me ? 1 : 0);
                    if (y[t] != me && q < iD - 1) row[q] = y[t];
                }
            }
        }
        // long rows, one per step with the whole warp: the first kExpChunk entries of
        // the next row are loaded before this row's are stored (eight loads per
        // lane in flight)
        uint32_t todo = __ballot_sync(kFull, D > kLaneRow + 1);
        int j = todo ? __ffs(todo) - 1 : -1;
        int64_t js0 = 0, jo = 0;
        int iD = 0;
        int32_t x[kExpVec];
        auto fetch = [&](int jj, int64_t& s0_, int64_t& o_, int& d_, int32_t (&v)[kExpVec]) {
            s0_ = __shfl_sync(kFull, s0, jj);
            d_ = (int)__shfl_sync(kFull, D, jj);
            o_ = __shfl_sync(kFull, o, jj);
            const int32_t me_ = (int32_t)(r0 + jj);
#pragma unroll
            for (int t = 0; t < kExpVec; ++t) {
                const int k = lane + 32 * t;
                v[t] = k < d_ ? S[s0_ + k] : me_;
            }
        };
        if (j >= 0) fetch(j, js0, jo, iD, x);
        while (j >= 0) {
            todo &= todo - 1;
            const int nj = todo ? __ffs(todo) - 1 : -1;
            int64_t ns0 = 0, no = 0;
            int nD = 0;
            int32_t nx[kExpVec];
            if (nj >= 0) fetch(nj, ns0, no, nD, nx);
            const int32_t me = (int32_t)(r0 + j);
            int32_t* row = cols + jo;
#pragma unroll
            for (int t = 0; t < kExpVec; ++t) {
                const int k = lane + 32 * t;
                const int q = k - (x[t] > me ? 1 : 0);
                if (x[t] != me && q < iD - 1) row[q] = x[t];  // q < D - 1 always holds when i is in S_u
            }
            const int32_t* su = S + js0;
            if (iD > kExpChunk) {  // the rest of a long row: each chunk's loads go out before the previous chunk's stores
                int32_t y[kExpVec];
#pragma unroll
                for (int t = 0; t < kExpVec; ++t) {
                    const int k = kExpChunk + lane + 32 * t;
                    y[t] = k < iD ? su[k] : me;
                }
                for (int k0 = kExpChunk; k0 < iD; k0 += kExpChunk) {
                    int32_t z[kExpVec];
#pragma unroll
                    for (int t = 0; t < kExpVec; ++t) {
                        const int k = k0 + kExpChunk + lane + 32 * t;
                        z[t] = k < iD ? su[k] : me;
                    }
#pragma unroll
                    for (int t = 0; t < kExpVec; ++t) {
                        const int k = k0 + lane + 32 * t;
                        const int q = k - (y[t] > me ? 1 : 0);
                        if (y[t] != me && q < iD - 1) row[q] = y[t];
                    }
#pragma unroll
                    for (int t = 0; t < kExpVec; ++t) y[t] = z[t];
                }
            }
            j = nj;
            js0 = ns0;
            jo = no;
            iD = nD;
#pragma unroll
            for (int t = 0; t < kExpVec; ++t) x[t] = nx[t];
        }
    }
}

using Timer = EventMarks;

// Readbacks of the build, written by one small kernel straight into mapped
// page-locked host memory (pinned_scratch_device): the sizes of the closed
// lists and of the CSR, the per-segment edge counts, the longest list and the
// encoder's error word in mid-build; the error counters and totals at the end.
struct MidReadback {
    int64_t sizes[2];                        // sum of D_u, nnz
    unsigned long long segs[kEdgeSegs + 1];  // per-segment edge counts, then the single-list count
    unsigned long long pack_error;           // encoder's first error word (0: none)
    int dmax;
    int nfalse;                              // candidates the confirmation rejected
};

struct EndReadback {
    int64_t U, R;
    int err[4];  // the first four device counters
};

__global__ void k_mid_readback(const int64_t* __restrict__ sd, const int64_t* __restrict__ nnz,
                               const unsigned long long* __restrict__ ecur, const int* __restrict__ dmax,
                               const unsigned long long* __restrict__ pack_flags, MidReadback* dst) {
    dep_entry();  // launched dependent on the kernel before it
    const int t = threadIdx.x;
    if (t <= kEdgeSegs) dst->segs[t] = ecur[t];
    if (t == 0) {
        dst->sizes[0] = *sd;
        dst->sizes[1] = *nnz;
        dst->dmax = dmax[0];
        dst->nfalse = dmax[1];  // the counter after the longest-list maximum
        dst->pack_error = pack_flags ? *pack_flags : 0ull;
    }
}

__global__ void k_end_readback(const int* __restrict__ err, const int64_t* __restrict__ U,
                               const int64_t* __restrict__ R, EndReadback* dst) {
    dep_entry();  // launched dependent on the kernel before it
    const int t = threadIdx.x;
    if (t < 4) dst->err[t] = err[t];
    if (t == 0) {
        dst->U = *U;
        dst->R = R ? *R : 0;
    }
}

}  // namespace

tcrnet_status deletion_build(const Packed& pk, int T, DeletionResult& out, cudaStream_t s, int num_sms, bool profile,
                             int partition_cap, bool keep_index, int partition_target, bool force_off64,
                             int record_hash_bits) {
    const int64_t n = pk.n;
    if (n > kDeletionMaxN || T > 2) return TCRNET_ENOTSUP;
    const int cap = (partition_cap > 0 && partition_cap < kWarpCap) ? partition_cap : kWarpCap;
    Timer tm(profile, s);
    const int t0 = tm.mark();
    // Arrays over distinct strings are sized by n (an upper bound) and the
    // record array by n + total length, so no host round trip is needed until
    // the output sizes are known.
    const int64_t R_max = n + pk.lensum;

    const bool join = T == 1;   // the deletion join (l_max = 1)
    const bool cand2 = T == 2;  // candidates of shared variants + exact check (l_max = 2)
    // partitions of the l_max = 1 join, sized from the record bound
    int64_t P = 1;
    if (join) {
        const int target = partition_target > 0 ? partition_target
                                                 : (R_max <= kTargetSwitchRecords ? kTargetPartSmall : kTargetPartLarge);
        P = std::max<int64_t>(1, std::min<int64_t>(R_max / target + 1, 1LL << 30));
    }
    // Every counter of the build that starts at zero, cleared by one memset
    // (u64 words): the edge cursors ([kEdgeSegs]: single-segment count), the
    // distinct-string count, the device counters ([0] dedup error, [1] fill
    // error, [2] partitions for the quadratic join, [3] partitions for the
    // sorted join, [4] largest closed list, [5] rejected candidates, [6..8]
    // lists of the long sort classes, [10..13] the list sort's own counters),
    // and the status words of the build's scans.
    const int64_t w_scan_n = scan_status_words(n);
    const int64_t w_scan_p = join ? scan_status_words(P) : 0;
    const int64_t w_fixed = (kEdgeSegs + 1) + 1 + 7;
    DevBuf zeroed;
    TCR_CHECK(zeroed.alloc(sizeof(unsigned long long) * (w_fixed + 3 * w_scan_n + w_scan_p), s));
    unsigned long long* d_ecur = zeroed.as<unsigned long long>();  // cleared by k_build_clear
    unsigned long long* d_ucount = d_ecur + (kEdgeSegs + 1);
    int* d_err = reinterpret_cast<int*>(d_ucount + 1);
    unsigned long long* st_members = d_ucount + 8;  // scan status words, one slice per scan
    unsigned long long* st_uoff = st_members + w_scan_n;
    unsigned long long* st_off64 = st_uoff + w_scan_n;
    unsigned long long* st_poff = st_off64 + w_scan_n;
    auto slice = [](unsigned long long* p, int64_t words) { return words > 0 ? p : nullptr; };
    // edges of the one-pass join: 2 x (records bound), split in kEdgeSegs segments
    const int64_t seg_cap = ceil_div(2 * R_max + 64, kEdgeSegs);
    const int64_t ecap = seg_cap * kEdgeSegs;

    // ---- 1. dedup
    int64_t S = 1024;
    while (S < 2 * n) S <<= 1;
    DevBuf table, slot_of, slot_u;
    TCR_CHECK(table.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(slot_of.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(slot_u.alloc(sizeof(int32_t) * S, s));
    const int64_t* d_U = reinterpret_cast<const int64_t*>(d_ucount);  // distinct strings, on the device
    DevBuf ucanon, ulen, umult, uid, mem_off, mcur, members, mpos;
    if (keep_index) TCR_CHECK(ucanon.alloc_owned(sizeof(Canon) * n, s));
    else TCR_CHECK(ucanon.alloc(sizeof(Canon) * n, s));
    TCR_CHECK(ulen.alloc(n, s));
    if (keep_index) TCR_CHECK(umult.alloc_owned(sizeof(int32_t) * n, s));
    else TCR_CHECK(umult.alloc(sizeof(int32_t) * n, s));
    DevBuf pcnt, wsum;  // the join's counters
    TCR_CHECK(wsum.alloc(sizeof(int32_t) * n, s));
    if (join) TCR_CHECK(pcnt.alloc(sizeof(int32_t) * P, s));
    {
        const int64_t zwords = (int64_t)(zeroed.bytes() / sizeof(unsigned long long));
        const int64_t total = zwords + S + 2 * n + (join ? P : 0);
        k_build_clear<<<(unsigned)std::min<int64_t>(grid_for(total), (int64_t)num_sms * 8), kThreads, 0, s>>>(
            zeroed.as<unsigned long long>(), zwords, table.as<int32_t>(), S, umult.as<int32_t>(), wsum.as<int32_t>(),
            n, join ? pcnt.as<int32_t>() : nullptr, join ? P : 0);
        TCR_LAUNCH_CHECK();
    }
    k_dedup_insert<<<grid_for(n), kThreads, 0, s>>>(
        pk.canon_in.as<Canon>(), pk.lens.as<uint8_t>(), n, table.as<int32_t>(), (uint32_t)(S - 1),
        slot_of.as<int32_t>(), slot_u.as<int32_t>(), d_ucount, ucanon.as<Canon>(), ulen.as<uint8_t>(), d_err);
    TCR_LAUNCH_CHECK();
    // the arrays the dedup does not use are allocated while it runs (the
    // host's allocation calls were the GPU's wait before it)
    if (keep_index) TCR_CHECK(uid.alloc_owned(sizeof(int32_t) * n, s));
    else TCR_CHECK(uid.alloc(sizeof(int32_t) * n, s));
    if (keep_index) TCR_CHECK(mem_off.alloc_owned(sizeof(int64_t) * (n + 1), s));
    else TCR_CHECK(mem_off.alloc(sizeof(int64_t) * (n + 1), s));
    TCR_CHECK(mcur.alloc(sizeof(int32_t) * n, s));
    if (keep_index) TCR_CHECK(members.alloc_owned(sizeof(int32_t) * n, s));
    else TCR_CHECK(members.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(mpos.alloc(sizeof(int32_t) * n, s));
    // node ids, multiplicities and member lists M_u are first needed by the
    // confirmation's weights and the closed lists: built on the side stream
    // while the records and the join run (the records need only the distinct
    // strings); s waits for them (ev[1]) before the confirmation
    const SideStream* side = leased_side_stream();
    cudaStream_t ms = s;
    if (side) {
        TCR_CUDA(cudaEventRecord(side->ev[0], s));
        TCR_CUDA(cudaStreamWaitEvent(side->stream, side->ev[0], 0));
        ms = side->stream;
        k_uid<<<grid_for(n), kThreads, 0, ms>>>(slot_of.as<int32_t>(), slot_u.as<int32_t>(), n, uid.as<int32_t>(),
                                                umult.as<int32_t>());
        TCR_LAUNCH_CHECK();
    } else {
        TCR_CUDA(launch_dependent(k_uid, dim3(grid_for(n)), dim3(kThreads), 0, s, slot_of.as<int32_t>(),
                                  slot_u.as<int32_t>(), n, uid.as<int32_t>(), umult.as<int32_t>()));
        note_launch();
    }
    TCR_CHECK(scan_exclusive_i32_to_i64(umult.as<int32_t>(), mem_off.as<int64_t>(), n, ms, slice(st_members, w_scan_n)));
    TCR_CUDA(cudaMemsetAsync(mcur.as<void>(), 0, sizeof(int32_t) * n, ms));
    k_members<<<grid_for(n), kThreads, 0, ms>>>(uid.as<int32_t>(), n, mem_off.as<int64_t>(), mcur.as<int32_t>(),
                                                members.as<int32_t>(), mpos.as<int32_t>());
    TCR_LAUNCH_CHECK();
    if (side) TCR_CUDA(cudaEventRecord(side->ev[1], ms));
    const int t1 = tm.mark();

    // ---- 2. records
    DevBuf poff, recs, fb_list, big_list, pedges, eoff, ucur, uoff, edges;
    TCR_CHECK(ucur.alloc(sizeof(unsigned long long) * n, s));
    TCR_CHECK(uoff.alloc(sizeof(int64_t) * (n + 1), s));
    const Weigh weigh{umult.as<int32_t>(), wsum.as<int32_t>()};
    int jgrid = 1;
    int t2 = t1, t3 = t1;
    int64_t E2_cap = 0, R2 = 0, NC2 = 0;  // l_max = 2: edge buffer capacity, records, candidates
    if (join) {
        if (keep_index) TCR_CHECK(poff.alloc_owned(sizeof(int64_t) * (P + 1), s));
        else TCR_CHECK(poff.alloc(sizeof(int64_t) * (P + 1), s));
        if (keep_index) TCR_CHECK(recs.alloc_owned(sizeof(uint64_t) * R_max, s));
        else TCR_CHECK(recs.alloc(sizeof(uint64_t) * R_max, s));
        TCR_CHECK(fb_list.alloc(sizeof(int32_t) * P, s));
        TCR_CHECK(big_list.alloc(sizeof(int32_t) * P, s));
        TCR_CHECK(pedges.alloc(sizeof(int64_t) * P, s));
        TCR_CHECK(eoff.alloc(sizeof(int64_t) * (P + 1), s));
        TCR_CHECK(edges.alloc(sizeof(int2) * ecap, s));
        const unsigned rgrid = grid_for(n);
        TCR_CUDA(launch_dependent(k_records<false>, dim3(rgrid), dim3(kThreads), 0, s, ucanon.as<Canon>(),
                                  ulen.as<uint8_t>(), d_U, n, (uint32_t)P, pcnt.as<int32_t>(), nullptr, nullptr, 0u,
                                  R_max, 0xffffffffull));
        note_launch();
        // the scan turns the counts behind itself into the scatter's slot cursors
        // (each at its partition's start)
        TCR_CHECK(scan_exclusive_i32_to_i64_cursors(pcnt.as<int32_t>(), poff.as<int64_t>(), P, s,
                                                    slice(st_poff, w_scan_p)));
        // the partitions over 32 records are listed on the second side stream
        // while the records are scattered; their joins then run there beside
        // k_join_small (without a lease: all in order on s, listed by k_join_small)
        const SideStream* jside = side;
        if (jside) {
            TCR_CUDA(cudaEventRecord(jside->ev[4], s));
            TCR_CUDA(cudaStreamWaitEvent(jside->stream2, jside->ev[4], 0));
            k_part_classes<<<(unsigned)std::min<int64_t>(grid_for(P), (int64_t)num_sms * 8), kThreads, 0,
                             jside->stream2>>>(poff.as<int64_t>(), P, cap, big_list.as<int32_t>(), d_err + 3,
                                               fb_list.as<int32_t>(), d_err + 2);
            TCR_LAUNCH_CHECK();
        }
        TCR_CUDA(launch_dependent(k_records<true>, dim3(rgrid), dim3(kThreads), 0, s, ucanon.as<Canon>(),
                                  ulen.as<uint8_t>(), d_U, n, (uint32_t)P, pcnt.as<int32_t>(), poff.as<int64_t>(),
                                  recs.as<uint64_t>(), 0u, R_max,
                                  record_hash_bits >= 32 ? 0xffffffffull : ((1ull << record_hash_bits) - 1ull)));
        note_launch();
        t2 = tm.mark();
        if (jside) {  // the records are in place: the sorted and quadratic joins on the side stream
            TCR_CUDA(cudaEventRecord(jside->ev[5], s));
            TCR_CUDA(cudaStreamWaitEvent(jside->stream2, jside->ev[5], 0));
            k_join_sorted<false><<<num_sms * 4, kThreads, 0, jside->stream2>>>(
                big_list.as<int32_t>(), d_err + 3, poff.as<int64_t>(), recs.as<uint64_t>(), T, pedges.as<int64_t>(),
                nullptr, edges.as<int2>(), d_ecur, seg_cap);
            TCR_LAUNCH_CHECK();
            k_join_fallback<false><<<num_sms * 2, kThreads, 0, jside->stream2>>>(
                fb_list.as<int32_t>(), d_err + 2, poff.as<int64_t>(), recs.as<uint64_t>(), T, pedges.as<int64_t>(),
                nullptr, edges.as<int2>(), d_ecur, seg_cap);
            TCR_LAUNCH_CHECK();
            TCR_CUDA(cudaEventRecord(jside->ev[7], jside->stream2));
        }
        // ---- 3a. join, pass 1: candidate pairs, then their confirmation (edges, weighted degrees W_u)
        jgrid = (int)std::min<int64_t>(ceil_div(P, 32 * kWarps), (int64_t)num_sms * 16);
        TCR_CUDA(launch_dependent(k_join_small<false>, dim3(jgrid), dim3(kThreads), 0, s, poff.as<int64_t>(), P,
                                  recs.as<uint64_t>(), cap, T, pedges.as<int64_t>(), nullptr, edges.as<int2>(),
                                  d_ecur, seg_cap, jside ? nullptr : big_list.as<int32_t>(), d_err + 3,
                                  jside ? nullptr : fb_list.as<int32_t>(), d_err + 2, R_max));
        note_launch();
        if (jside) {
            TCR_CUDA(cudaStreamWaitEvent(s, jside->ev[7], 0));  // all candidates written
        } else {
            TCR_CUDA(launch_dependent(k_join_sorted<false>, dim3(num_sms * 4), dim3(kThreads), 0, s,
                                      big_list.as<int32_t>(), d_err + 3, poff.as<int64_t>(), recs.as<uint64_t>(), T,
                                      pedges.as<int64_t>(), nullptr, edges.as<int2>(), d_ecur, seg_cap));
            note_launch();
            TCR_CUDA(launch_dependent(k_join_fallback<false>, dim3(num_sms * 2), dim3(kThreads), 0, s,
                                      fb_list.as<int32_t>(), d_err + 2, poff.as<int64_t>(), recs.as<uint64_t>(), T,
                                      pedges.as<int64_t>(), nullptr, edges.as<int2>(), d_ecur, seg_cap));
            note_launch();
        }
        if (side) TCR_CUDA(cudaStreamWaitEvent(s, side->ev[1], 0));  // multiplicities for the weights
        TCR_CUDA(launch_dependent(k_confirm, dim3(confirm_blocks_x(num_sms), kEdgeSegs), dim3(kThreads), 0, s,
                                  edges.as<int2>(), seg_cap, (const unsigned long long*)d_ecur, 1,
                                  (const Canon*)ucanon.as<Canon>(), weigh, d_err + 5));
        note_launch();
        t3 = tm.mark();
    } else if (cand2) {
        // records of every variant with up to two deletions, partitioned by hash
        DevBuf tot;
        TCR_CHECK(tot.alloc(sizeof(unsigned long long) * 2, s));
        TCR_CUDA(cudaMemsetAsync(tot.as<void>(), 0, sizeof(unsigned long long) * 2, s));
        unsigned long long* d_tot = tot.as<unsigned long long>();
        k_var2_count<<<grid_for(n), kThreads, 0, s>>>(ucanon.as<Canon>(), ulen.as<uint8_t>(), d_U, n, d_tot);
        TCR_LAUNCH_CHECK();
        unsigned long long h_tot = 0;
        TCR_CUDA(cudaMemcpyAsync(&h_tot, d_tot, sizeof(h_tot), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        R2 = (int64_t)h_tot;
        const int target = partition_target > 0 ? partition_target : kTargetPartSmall;
        P = std::max<int64_t>(1, std::min<int64_t>(R2 / target + 1, 1LL << 30));
        DevBuf pcnt;
        TCR_CHECK(pcnt.alloc(sizeof(int32_t) * P, s));
        if (keep_index) {  // the variant records are the handle's query index
            TCR_CHECK(poff.alloc_owned(sizeof(int64_t) * (P + 1), s));
            TCR_CHECK(recs.alloc_owned(sizeof(uint64_t) * std::max<int64_t>(R2, 1), s));
        } else {
            TCR_CHECK(poff.alloc(sizeof(int64_t) * (P + 1), s));
            TCR_CHECK(recs.alloc(sizeof(uint64_t) * std::max<int64_t>(R2, 1), s));
        }
        TCR_CUDA(cudaMemsetAsync(pcnt.as<void>(), 0, sizeof(int32_t) * P, s));
        k_var2_records<false><<<grid_for(n), kThreads, 0, s>>>(ucanon.as<Canon>(), ulen.as<uint8_t>(), d_U, n,
                                                               (uint32_t)P, pcnt.as<int32_t>(), nullptr, nullptr);
        TCR_LAUNCH_CHECK();
        TCR_CHECK(scan_exclusive_i32_to_i64(pcnt.as<int32_t>(), poff.as<int64_t>(), P, s));
        TCR_CUDA(cudaMemsetAsync(pcnt.as<void>(), 0, sizeof(int32_t) * P, s));
        k_var2_records<true><<<grid_for(n), kThreads, 0, s>>>(ucanon.as<Canon>(), ulen.as<uint8_t>(), d_U, n,
                                                              (uint32_t)P, pcnt.as<int32_t>(), poff.as<int64_t>(),
                                                              recs.as<uint64_t>());
        TCR_LAUNCH_CHECK();
        t2 = tm.mark();
        // candidate pairs filed under their smaller string: counted per row,
        // rows placed, then written; sorted rows put repeats side by side
        const unsigned pgrid = (unsigned)std::min<int64_t>(ceil_div(P, kWarps), (int64_t)num_sms * 16);
        DevBuf ccur_b, coff, ccols;
        TCR_CHECK(ccur_b.alloc(sizeof(int32_t) * n, s));
        TCR_CHECK(coff.alloc(sizeof(int64_t) * (n + 1), s));
        TCR_CUDA(cudaMemsetAsync(ccur_b.as<void>(), 0, sizeof(int32_t) * n, s));
        k_var2_pairs<false><<<pgrid, kThreads, 0, s>>>(poff.as<int64_t>(), P, recs.as<uint64_t>(),
                                                       ccur_b.as<int32_t>(), nullptr, nullptr);
        TCR_LAUNCH_CHECK();
        TCR_CHECK(scan_exclusive_i32_to_i64(ccur_b.as<int32_t>(), coff.as<int64_t>(), n, s));
        int64_t NC = 0;
        TCR_CUDA(cudaMemcpyAsync(&NC, coff.as<int64_t>() + n, sizeof(NC), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        NC2 = NC;
        TCR_CHECK(ccols.alloc(sizeof(int32_t) * std::max<int64_t>(NC, 1), s));
        TCR_CUDA(cudaMemsetAsync(ccur_b.as<void>(), 0, sizeof(int32_t) * n, s));
        k_var2_pairs<true><<<pgrid, kThreads, 0, s>>>(poff.as<int64_t>(), P, recs.as<uint64_t>(),
                                                      ccur_b.as<int32_t>(), coff.as<int64_t>(), ccols.as<int32_t>());
        TCR_LAUNCH_CHECK();
        if (!keep_index) recs.reset();
        TCR_CHECK(sort_rows(coff.as<int64_t>(), ccols.as<int32_t>(), n, s, num_sms));
        E2_cap = std::max<int64_t>(NC, 1);
        TCR_CHECK(edges.alloc(sizeof(int2) * E2_cap, s));
        const unsigned vgrid = (unsigned)std::min<int64_t>(ceil_div(n, kVerifyWarps), (int64_t)num_sms * 32);
        if (side) TCR_CUDA(cudaStreamWaitEvent(s, side->ev[1], 0));  // multiplicities for the weights
        k_cand_verify<<<vgrid, 32 * kVerifyWarps, 0, s>>>(coff.as<int64_t>(), ccols.as<int32_t>(), d_U, ucanon.as<Canon>(),
                                                 ulen.as<uint8_t>(), weigh, edges.as<int2>(), d_ecur + kEdgeSegs,
                                                 E2_cap, d_err + 1);
        TCR_LAUNCH_CHECK();
        t3 = tm.mark();
    }

    // ---- 4. list sizes D_u = m_u + W_u, list offsets, node degrees
    DevBuf deg, off64;
    TCR_CHECK(deg.alloc_owned(sizeof(int32_t) * n, s));  // results are handed to the handle
    TCR_CHECK(off64.alloc_owned(sizeof(int64_t) * (n + 1), s));
    static_assert(sizeof(MidReadback) <= kPinnedScratchBytes, "readback fits the pinned scratch");
    MidReadback pageable;
    MidReadback* rb = static_cast<MidReadback*>(pinned_scratch());
    const unsigned long long* d_pack_flags = pk.flags.as<unsigned long long>();
    // The size scan lists the long lists by sort class, so that the list
    // sort's long classes start with its short-list kernel (at 8e5 strings the
    // list sort takes 0.146 -> 0.122 ms and the size scan ~10 us more; at 8e6
    // the block class dominates the sort and the listing cost 0.2 ms more than
    // it saved, measured on a B300): up to kListClassesMaxN strings.
    constexpr int64_t kListClassesMaxN = 2000000;
    const bool list_classes = w_scan_n > 0 && n <= kListClassesMaxN;
    DevBuf off32, cls_lists;
    if (list_classes) TCR_CHECK(cls_lists.alloc(sizeof(int32_t) * 3 * n, s));  // long lists by sort class
    // the list sizes and offsets from W_u, then the sizes of the lists and of
    // the CSR, the candidate counts, the longest list, the rejected candidates
    // and the encoder's error word in one synchronisation
    auto sizes_and_readback = [&]() -> tcrnet_status {
        if (w_scan_n > 0) {  // several tiles: sizes and both scans in one launch
            const int64_t tiles = ceil_div(n, kScanTile);
            TCR_CUDA(launch_dependent(k_fill_sizes, dim3((unsigned)tiles, 2), dim3(kScanThreads), 0, s,
                                      wsum.as<int32_t>(), umult.as<int32_t>(), uid.as<int32_t>(), n,
                                      ucur.as<unsigned long long>(), d_err + 4, deg.as<int32_t>(), uoff.as<int64_t>(),
                                      off64.as<int64_t>(), st_uoff, st_off64, tiles,
                                      list_classes ? cls_lists.as<int32_t>() : nullptr,
                                      list_classes ? d_err + 6 : nullptr));
            note_launch();
        } else {
            TCR_CUDA(launch_dependent(k_closed_size, dim3(grid_for(n)), dim3(kThreads), 0, s, umult.as<int32_t>(),
                                      n, wsum.as<int32_t>(), d_err + 4));
            note_launch();
            TCR_CHECK(scan_exclusive_i32_to_i64(wsum.as<int32_t>(), uoff.as<int64_t>(), n, s));
            k_list_cursors<<<grid_for(n), kThreads, 0, s>>>(uoff.as<int64_t>(), umult.as<int32_t>(), n,
                                                            ucur.as<unsigned long long>());
            TCR_LAUNCH_CHECK();
            TCR_CUDA(launch_dependent(k_node_degree, dim3(grid_for(n)), dim3(kThreads), 0, s, uid.as<int32_t>(), n,
                                      wsum.as<int32_t>(), deg.as<int32_t>()));
            note_launch();
            TCR_CHECK(scan_exclusive_i32_to_i64(deg.as<int32_t>(), off64.as<int64_t>(), n, s));
        }
        if (rb && pinned_scratch_device()) {
            TCR_CUDA(launch_dependent(k_mid_readback, dim3(1), dim3(96), 0, s, uoff.as<int64_t>() + n,
                                      off64.as<int64_t>() + n, d_ecur, d_err + 4, d_pack_flags,
                                      static_cast<MidReadback*>(pinned_scratch_device())));
            note_launch();
        } else {
            if (!rb) rb = &pageable;
            rb->pack_error = 0;
            TCR_CUDA(cudaMemcpyAsync(&rb->sizes[0], uoff.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            TCR_CUDA(cudaMemcpyAsync(&rb->sizes[1], off64.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                     s));
            TCR_CUDA(cudaMemcpyAsync(rb->segs, d_ecur, sizeof(rb->segs), cudaMemcpyDeviceToHost, s));
            TCR_CUDA(cudaMemcpyAsync(&rb->dmax, d_err + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
            TCR_CUDA(cudaMemcpyAsync(&rb->nfalse, d_err + 5, sizeof(int), cudaMemcpyDeviceToHost, s));
            if (d_pack_flags)
                TCR_CUDA(cudaMemcpyAsync(&rb->pack_error, d_pack_flags, sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost, s));
        }
        // int32 row offsets for the handle, allocated and narrowed on the second
        // stream while the host waits for the readback (dropped below if nnz
        // turns out to need int64 offsets); allocated on the stream that writes
        // it, so that freeing it on any early return is ordered after the narrowing
        off32.reset();
        if (!force_off64 && n + 1 <= 0x7fffffffLL) {
            cudaStream_t ns = s;
            if (side) {
                TCR_CUDA(cudaEventRecord(side->ev[6], s));
                TCR_CUDA(cudaStreamWaitEvent(side->stream, side->ev[6], 0));
                ns = side->stream;
            }
            TCR_CHECK(off32.alloc_owned(sizeof(int32_t) * (n + 1), ns));
            TCR_CHECK(narrow_offsets(off64.as<int64_t>(), off32.as<int32_t>(), n + 1, ns));
        }
        TCR_CUDA(cudaStreamSynchronize(s));
        TCR_CHECK(pack_flags_status(rb->pack_error, &out.bad_index));
        if (off32.as<void>() && rb->sizes[1] > 0x7fffffffLL) off32.reset();  // int64 offsets after all
        return TCRNET_OK;
    };
    TCR_CHECK(sizes_and_readback());
    unsigned long long segs[kEdgeSegs + 1];
    for (int g = 0; g <= kEdgeSegs; ++g) segs[g] = rb->segs[g];
    int h_dmax = rb->dmax;
    int64_t SD = rb->sizes[0], nnz = rb->sizes[1];
    int64_t nfalse = rb->nfalse;  // rejected candidates, (-1, -1) in the list
    int64_t E = 0, seg_max = 0;   // E: entries of the list (edges and rejected candidates)
    bool overflow = false;
    for (int g = 0; g < kEdgeSegs; ++g) {
        E += (int64_t)segs[g];
        seg_max = std::max<int64_t>(seg_max, (int64_t)segs[g]);
        overflow = overflow || (int64_t)segs[g] > seg_cap;
    }
    if (cand2) {  // one contiguous edge list
        E = (int64_t)segs[kEdgeSegs];
        seg_max = E;
        if (E > E2_cap) return TCRNET_EDEVICE;
    }
    // ---- 3b. candidates that did not fit: second join pass at scanned
    // positions, their confirmation, and the list sizes again from the
    // complete weights
    int n_two_pass = 0;
    int64_t fill_segs = kEdgeSegs, fill_cap = seg_cap;
    const unsigned long long* fill_counts = d_ecur;
    if (cand2) {
        fill_segs = 1;
        fill_cap = E2_cap;
        fill_counts = d_ecur + kEdgeSegs;
    }
    if (join && overflow) {
        edges.reset();
        TCR_CHECK(edges.alloc(sizeof(int2) * E, s));
        TCR_CHECK(scan_exclusive_i64(pedges.as<int64_t>(), eoff.as<int64_t>(), P, s));
        k_join_small<true><<<jgrid, kThreads, 0, s>>>(poff.as<int64_t>(), P, recs.as<uint64_t>(), cap, T, nullptr,
                                                      eoff.as<int64_t>(), edges.as<int2>(), nullptr, 0, nullptr,
                                                      nullptr, nullptr, nullptr);
        TCR_LAUNCH_CHECK();
        k_join_sorted<true><<<num_sms * 4, kThreads, 0, s>>>(big_list.as<int32_t>(), d_err + 3, poff.as<int64_t>(),
                                                             recs.as<uint64_t>(), T, nullptr, eoff.as<int64_t>(),
                                                             edges.as<int2>(), nullptr, 0);
        TCR_LAUNCH_CHECK();
        k_join_fallback<true><<<num_sms * 2, kThreads, 0, s>>>(fb_list.as<int32_t>(), d_err + 2, poff.as<int64_t>(),
                                                               recs.as<uint64_t>(), T, nullptr, eoff.as<int64_t>(),
                                                               edges.as<int2>(), nullptr, 0);
        TCR_LAUNCH_CHECK();
        n_two_pass = 1;
        // the list is now contiguous: one segment of E entries
        const unsigned long long e64 = (unsigned long long)E;
        TCR_CUDA(cudaMemcpyAsync(d_ecur + kEdgeSegs, &e64, sizeof(e64), cudaMemcpyHostToDevice, s));
        fill_segs = 1;
        fill_cap = E;
        fill_counts = d_ecur + kEdgeSegs;
        seg_max = E;
        // the first confirmation skipped the overflowed buffer: weights from
        // the complete list, then the sizes again (their status words and the
        // longest-list maximum cleared first)
        TCR_CUDA(cudaMemsetAsync(wsum.as<void>(), 0, sizeof(int32_t) * n, s));
        TCR_CUDA(cudaMemsetAsync(d_err + 4, 0, 5 * sizeof(int), s));
        if (w_scan_n > 0) TCR_CUDA(cudaMemsetAsync(st_uoff, 0, 2 * sizeof(unsigned long long) * w_scan_n, s));
        k_confirm<<<dim3(grid_for(E), 1), kThreads, 0, s>>>(edges.as<int2>(), E, d_ecur + kEdgeSegs, 0,
                                                           ucanon.as<Canon>(), weigh, d_err + 5);
        TCR_LAUNCH_CHECK();
        TCR_CHECK(sizes_and_readback());
        h_dmax = rb->dmax;
        SD = rb->sizes[0];
        nnz = rb->sizes[1];
        nfalse = rb->nfalse;
    }
    DevBuf Sbuf;
    TCR_CHECK(Sbuf.alloc(sizeof(int32_t) * SD, s));
    // a build handle keeps the edges between distinct strings (analytics run on
    // that graph of U nodes instead of the n-node network)
    DevBuf uedges;
    const int64_t E_true = E - nfalse;
    const bool keep_edges = keep_index && (join || cand2) && E_true > 0;
    // each list's own members (after its member list exists) and the kept
    // edges go to the side stream, next to the neighbour appends on this one
    cudaStream_t fs = s;
    if (side) {
        TCR_CUDA(cudaEventRecord(side->ev[2], s));
        TCR_CUDA(cudaStreamWaitEvent(side->stream, side->ev[2], 0));
        TCR_CUDA(cudaStreamWaitEvent(s, side->ev[1], 0));  // member lists ready for the appends
        fs = side->stream;
    }
    k_closed_self<<<grid_for(n), kThreads, 0, fs>>>(uid.as<int32_t>(), mpos.as<int32_t>(), n, uoff.as<int64_t>(),
                                                    Sbuf.as<int32_t>());
    TCR_LAUNCH_CHECK();
    // the kept edges are allocated and gathered after the neighbour appends are
    // launched, so the allocation's host time overlaps them
    auto gather_edges = [&]() -> tcrnet_status {
        TCR_CHECK(uedges.alloc_owned(sizeof(int2) * E_true, fs));  // stream-ordered on the stream that fills it
        if (cand2 || (n_two_pass && nfalse == 0)) {  // already one contiguous list
            TCR_CUDA(cudaMemcpyAsync(uedges.as<void>(), edges.as<void>(), sizeof(int2) * E_true,
                                     cudaMemcpyDeviceToDevice, fs));
        } else if (nfalse == 0) {  // the one-pass buffer holds every edge: segments to one array
            SegBases sb;
            sb.base[0] = 0;
            for (int g = 0; g < kEdgeSegs; ++g) sb.base[g + 1] = sb.base[g] + (int64_t)segs[g];
            const dim3 cgrid(grid_for(std::max<int64_t>(seg_max, 1)), (unsigned)kEdgeSegs);
            k_compact_edges<<<cgrid, kThreads, 0, fs>>>(edges.as<int2>(), seg_cap, sb, uedges.as<int2>());
            TCR_LAUNCH_CHECK();
        } else {  // rejected candidates among them (rare): edges gathered at a shared cursor
            DevBuf cur;
            TCR_CHECK(cur.alloc(sizeof(unsigned long long), fs));
            TCR_CUDA(cudaMemsetAsync(cur.as<void>(), 0, sizeof(unsigned long long), fs));
            const dim3 cgrid(grid_for(std::max<int64_t>(seg_max, 1)), (unsigned)fill_segs);
            k_gather_edges<<<cgrid, kThreads, 0, fs>>>(edges.as<int2>(), fill_cap, fill_counts, uedges.as<int2>(),
                                                       cur.as<unsigned long long>());
            TCR_LAUNCH_CHECK();
        }
        return TCRNET_OK;
    };
    if ((join || cand2) && E > 0) {
        if (!keep_index) recs.reset();
        const dim3 fgrid(grid_for(2 * seg_max), (unsigned)fill_segs);
        k_closed_edges<<<fgrid, kThreads, 0, s>>>(edges.as<int2>(), fill_cap, fill_counts, umult.as<int32_t>(),
                                                            mem_off.as<int64_t>(), members.as<int32_t>(),
                                                            ucur.as<unsigned long long>(), Sbuf.as<int32_t>(), SD,
                                                            d_err + 1);
        TCR_LAUNCH_CHECK();
    }
    if (keep_edges) TCR_CHECK(gather_edges());
    if (side) {  // own members, narrowed offsets and kept edges written
        TCR_CUDA(cudaEventRecord(side->ev[3], fs));
        TCR_CUDA(cudaStreamWaitEvent(s, side->ev[3], 0));
    }
    const int t4 = tm.mark();
    if (!keep_index) recs.reset();
    edges.reset();
    SortClasses classes;  // the long lists, listed by the size scan
    classes.wide = cls_lists.as<int32_t>();
    classes.mid = classes.wide + n;
    classes.big = classes.wide + 2 * n;
    classes.counts = d_err + 6;
    classes.zeroed4 = d_err + 10;
    TCR_CHECK(sort_rows(uoff.as<int64_t>(), Sbuf.as<int32_t>(), n, s, num_sms, h_dmax,
                        list_classes ? &classes : nullptr));
    const int t5 = tm.mark();

    // ---- 5. expand
    DevBuf cols;
    TCR_CHECK(cols.alloc_owned(sizeof(int32_t) * nnz, s));
    k_expand<<<(unsigned)std::min<int64_t>(ceil_div(n, 32 * kWarps), (int64_t)num_sms * 16), kThreads, 0, s>>>(
        uid.as<int32_t>(), n, uoff.as<int64_t>(), Sbuf.as<int32_t>(), off64.as<int64_t>(), cols.as<int32_t>());
    TCR_LAUNCH_CHECK();
    const int t6 = tm.mark();
    EndReadback pageable_end;
    EndReadback* eb = static_cast<EndReadback*>(pinned_scratch());
    if (eb && pinned_scratch_device()) {
        TCR_CUDA(launch_dependent(k_end_readback, dim3(1), dim3(32), 0, s, d_err, d_U,
                                  join ? poff.as<int64_t>() + P : nullptr,
                                  static_cast<EndReadback*>(pinned_scratch_device())));
        note_launch();
    } else {
        if (!eb) eb = &pageable_end;
        eb->U = eb->R = 0;
        TCR_CUDA(cudaMemcpyAsync(eb->err, d_err, sizeof(eb->err), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaMemcpyAsync(&eb->U, d_U, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (join)
            TCR_CUDA(cudaMemcpyAsync(&eb->R, poff.as<int64_t>() + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    TCR_CUDA(cudaStreamSynchronize(s));
    int h_err[4] = {eb->err[0], eb->err[1], eb->err[2], eb->err[3]};
    const int64_t h_U = eb->U;
    int64_t h_R = eb->R;
    if (cand2) h_R = R2;
    if (h_err[0] || h_err[1]) return TCRNET_EDEVICE;

    out.off64 = std::move(off64);
    out.off32 = std::move(off32);
    out.cols = std::move(cols);
    out.degree = std::move(deg);
    out.nnz = nnz;
    out.n_unique = h_U;
    out.n_records = h_R;
    out.candidates = NC2;
    out.unique_edges = E_true;
    out.n_fallback = h_err[2];
    out.closed_total = SD;
    out.two_pass_join = n_two_pass;
    out.rejected = nfalse;
    if (keep_index && (join || cand2)) {
        out.index.ucanon = static_cast<Canon*>(ucanon.release());
        out.index.umult = static_cast<int32_t*>(umult.release());
        out.index.mem_off = static_cast<int64_t*>(mem_off.release());
        out.index.members = static_cast<int32_t*>(members.release());
        out.index.recs = static_cast<uint64_t*>(recs.release());
        out.index.poff = static_cast<int64_t*>(poff.release());
        out.index.uid = static_cast<int32_t*>(uid.release());
        out.index.uedges = static_cast<int2*>(uedges.release());
        out.index.E = out.index.uedges ? E_true : 0;
        out.index.U = h_U;
        out.index.P = P;
        out.index.R = h_R;
        out.index.n = n;
        if (join && record_hash_bits < 32) out.index.hmask = (uint32_t)((1ull << record_hash_bits) - 1ull);
    }
    out.ms_phase[0] = tm.ms(t0, t1);  // dedup
    out.ms_phase[1] = tm.ms(t1, t2);  // records
    out.ms_phase[2] = tm.ms(t2, t3);  // join pass 1 (weighted degrees)
    out.ms_phase[3] = tm.ms(t3, t4);  // list sizes, join pass 2 (edges), list fill
    out.ms_phase[4] = 0.0;
    out.ms_phase[5] = tm.ms(t4, t5);  // list sort
    out.ms_phase[6] = tm.ms(t5, t6);  // expand
    out.ms_phase[7] = tm.ms(t0, t6);
    out.ms_join = tm.ms(t2, t4);
    out.ms_scan = 0.0;
    out.ms_fill = tm.ms(t3, t4);
    out.ms_sort = tm.ms(t4, t6);
    return TCRNET_OK;
}

// ---- queries against the resident index -----------------------------------

namespace {

struct IndexView {
    const Canon* ucanon;
    const int32_t* umult;
    const int64_t* mem_off;
    const int32_t* members;
    const uint64_t* recs;
    const int64_t* poff;
    uint32_t P;
};

// Exact check of a candidate match (equal 32-bit hash, fitting position tags)
// between variant vp of query string qc (-1: the full string) and record r:
// equal contents, and an identical resident string counted once (full to full).
__device__ __forceinline__ bool verify_candidate(const IndexView& ix, const Canon& qc, uint64_t r, int vp,
                                                 uint32_t& u) {
    const bool full = vp < 0;
    const Canon cq = full ? qc : delete_at(qc, vp);
    if (!canon_eq(cq, record_content(r, ix.ucanon))) return false;  // hash collision
    u = rec_u(r);
    if (!full && rec_p(r) != kTagF && canon_eq(qc, load_canon(ix.ucanon + u))) return false;
    return true;
}

// Neighbours of a query string among the distinct resident strings, found
// through the string's own records (full string and every deletion) in the
// resident partitions; each match is confirmed by content and each neighbour is
// found exactly once (see the file comment; an identical resident string
// matches full-to-full only, its deletion matches are skipped).
//
// A warp takes one query string. Lane v computes the key of variant g0 + v
// (-1: the full string) and its partition; the words of the (up to 32)
// partitions are then read as one flat sequence, 32 consecutive words per
// step, each lane finding the variant that owns its word by a binary search
// over the partition sizes' prefix sums. COUNT adds the multiplicities of the
// matches; WRITE emits their member lists at qoff[q] onwards (a lane copies
// short lists itself, long ones are queued and copied by the whole warp).
template <bool WRITE>
__global__ void __launch_bounds__(kThreads, 4)
k_query(IndexView ix, const Canon* __restrict__ qcanon, const uint8_t* __restrict__ qlen, int64_t m, int T,
        int64_t* __restrict__ qcount, const int64_t* __restrict__ qoff, int32_t* __restrict__ out,
        int2* __restrict__ hits, unsigned long long* __restrict__ hit_cur, int64_t hit_cap) {
    constexpr int kLaneCopyMax = 8, kQueued = 16;
    __shared__ int64_t big_src[kWarps][kQueued], big_dst[kWarps][kQueued];
    __shared__ int32_t big_len[kWarps][kQueued];
    __shared__ int big_n[kWarps];
    // COUNT: candidates wait in a per-warp queue and are verified 32 at a time,
    // one per lane, instead of one lane at a time as they turn up
    __shared__ uint64_t cand_r[kWarps][64];
    __shared__ int8_t cand_p[kWarps][64];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < m; q += stride) {
        const Canon qc = load_canon(qcanon + q);
        const int Lq = qlen[q];
        int64_t mine = 0;                           // COUNT: members found by this lane
        int qn = 0;                                 // COUNT: queued candidates (warp-uniform)
        auto flush = [&](int cnt) {                 // COUNT: verify the first cnt queued candidates
            bool hit = false;
            uint32_t u = 0;
            if (lane < cnt) hit = verify_candidate(ix, qc, cand_r[w][lane], cand_p[w][lane], u);
            mine += hit ? ix.umult[u] : 0;
            const unsigned hm = __ballot_sync(kFull, hit);
            if (hm && hits) {  // keep the match (query, distinct string) for the emit pass
                unsigned long long hb = 0;
                if (lane == 0) hb = atomicAdd(hit_cur, (unsigned long long)__popc(hm));
                hb = __shfl_sync(kFull, hb, 0);
                const int64_t slot = (int64_t)hb + __popc(hm & lt_mask);
                if (hit && slot < hit_cap) hits[slot] = make_int2((int32_t)q, (int32_t)u);
            }
            const int rest = qn - cnt;
            uint64_t tr = 0;
            int8_t tp = 0;
            if (lane < rest) {
                tr = cand_r[w][cnt + lane];
                tp = cand_p[w][cnt + lane];
            }
            __syncwarp();
            if (lane < rest) {
                cand_r[w][lane] = tr;
                cand_p[w][lane] = tp;
            }
            __syncwarp();
            qn = rest;
        };
        int64_t base = WRITE ? qoff[q] : 0;         // WRITE: next output slot (warp-uniform)
        if constexpr (WRITE) {
            if (lane == 0) big_n[w] = 0;
            __syncwarp();
        }
        const int last = T >= 1 ? Lq - 1 : -1;      // l_max = 0: the full string only
        for (int g0 = -1; g0 <= last; g0 += 32) {
            const int p = g0 + lane;
            const bool active = p <= last;
            uint32_t h32 = 0;
            int64_t b0 = 0;
            int32_t sz = 0;  // partition sizes and their sums fit 32 bits
            bool q_rs = false;
            if (active) {
                const Canon cq = p < 0 ? qc : delete_at(qc, p);
                q_rs = p >= 0 && run_start(qc, p);
                const uint64_t h = hash_canon(cq);
                h32 = (uint32_t)h;
                const uint32_t pid = part_of(h, ix.P);
                b0 = ix.poff[pid];
                sz = (int32_t)(ix.poff[pid + 1] - b0);
            }
            int32_t excl = sz;  // inclusive, then exclusive prefix sum over the lanes
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, excl, d);
                if (lane >= d) excl += y;
            }
            const int32_t S = __shfl_sync(kFull, excl, 31);
            excl -= sz;
            const int64_t rb = b0 - excl;  // word f of this lane's partition is recs[rb + f]
            // kRounds steps of 32 words: their loads are issued before any is tested
            constexpr int kRounds = 4;
            for (int32_t f00 = 0; f00 < S; f00 += 32 * kRounds) {
            uint64_t rr[kRounds];
            int vv[kRounds];
#pragma unroll
            for (int t = 0; t < kRounds; ++t) {
                const int32_t f = f00 + 32 * t + lane;
                int v = 0;  // owner: the last variant whose words start at or before f
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int32_t e = __shfl_sync(kFull, excl, v + step);
                    if (e <= f) v += step;
                }
                vv[t] = v;
                const int64_t vrb = __shfl_sync(kFull, rb, v);
                rr[t] = f < S ? ix.recs[vrb + f] : 0ull;
            }
#pragma unroll
            for (int t = 0; t < kRounds; ++t) {
                if (f00 + 32 * t >= S) break;  // warp-uniform
                const int32_t f = f00 + 32 * t + lane;
                const int v = vv[t];
                const uint32_t vh = __shfl_sync(kFull, h32, v);
                const bool vq_rs = __shfl_sync(kFull, q_rs, v);
                const int vp = g0 + v;
                bool cand = false;  // equal hash and fitting position tags
                if (f < S) {
                    const uint64_t r = rr[t];
                    if ((uint32_t)(r >> 32) == vh) {
                        const uint32_t rp = rec_p(r);
                        if (vp < 0) cand = (rp == kTagF) || (T >= 1 && rec_runstart(r));  // identical / q one shorter
                        else cand = (rp == kTagF) ? vq_rs : (rp == (uint32_t)vp);          // q one longer / substitution
                    }
                }
                if constexpr (!WRITE) {
                    const unsigned cm = __ballot_sync(kFull, cand);
                    if (cm) {
                        if (cand) {
                            const int slot = qn + __popc(cm & lt_mask);
                            cand_r[w][slot] = rr[t];
                            cand_p[w][slot] = (int8_t)vp;
                        }
                        qn += __popc(cm);
                        if (qn >= 32) {
                            __syncwarp();
                            flush(32);
                        }
                    }
                } else {
                    uint32_t u = 0;
                    const bool hit = cand && verify_candidate(ix, qc, rr[t], vp, u);
                    const int32_t mu = hit ? ix.umult[u] : 0;
                    if (!__any_sync(kFull, hit)) continue;
                    int64_t ex;
                    const int64_t tot = warp_scan((int64_t)mu, ex, lane);
                    if (hit) {
                        const int64_t src = ix.mem_off[u];
                        const int64_t pos = base + ex;
                        int slot = kQueued;
                        if (mu > kLaneCopyMax) {
                            slot = atomicAdd(&big_n[w], 1);
                            if (slot < kQueued) {
                                big_src[w][slot] = src;
                                big_dst[w][slot] = pos;
                                big_len[w][slot] = mu;
                            }
                        }
                        if (slot >= kQueued)
                            for (int32_t y = 0; y < mu; ++y) out[pos + y] = ix.members[src + y];
                    }
                    base += tot;
                }
            }
            }
        }
        if constexpr (!WRITE) {
            if (qn > 0) {
                __syncwarp();
                flush(qn);
            }
            int64_t ex;
            const int64_t total = warp_scan(mine, ex, lane);
            if (lane == 0) qcount[q] = total;
        } else {
            __syncwarp();
            const int nb = big_n[w] < kQueued ? big_n[w] : kQueued;
            for (int t = 0; t < nb; ++t) {
                const int64_t src = big_src[w][t], dst = big_dst[w][t];
                const int32_t len = big_len[w][t];
                for (int32_t y = lane; y < len; y += 32) out[dst + y] = ix.members[src + y];
            }
            __syncwarp();
        }
    }
}

// Emit pass over the matches kept by the count pass: the member list of u at
// qoff[q] + a slot taken from the query's cursor (rows are sorted afterwards).
// Short lists are copied by their lane, long ones by the whole warp.
__global__ void __launch_bounds__(kThreads)
k_query_emit(IndexView ix, const int2* __restrict__ hits, int64_t nh, const int64_t* __restrict__ qoff,
             int32_t* __restrict__ qcur, int32_t* __restrict__ out) {
    constexpr int kLaneCopyMax = 8;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; h0 < nh; h0 += nw * 32) {
        const int64_t k = h0 + lane;
        int64_t src = 0, pos = 0;
        int32_t mu = 0;
        if (k < nh) {
            const int2 hq = hits[k];
            src = ix.mem_off[hq.y];
            mu = ix.umult[hq.y];
            pos = qoff[hq.x] + atomicAdd(&qcur[hq.x], mu);
            if (mu <= kLaneCopyMax)
                for (int32_t y = 0; y < mu; ++y) out[pos + y] = ix.members[src + y];
        }
        unsigned todo = __ballot_sync(kFull, mu > kLaneCopyMax);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t js = __shfl_sync(kFull, src, j), jp = __shfl_sync(kFull, pos, j);
            const int32_t jm = __shfl_sync(kFull, mu, j);
            for (int32_t y = lane; y < jm; y += 32) out[jp + y] = ix.members[js + y];
        }
    }
}

// ---- l_max = 2 queries against the resident variant records ----------------
//
// A query string's variants with up to two deletions (the run-start rule of
// the records) are looked up in the resident partitions; every resident
// distinct string with a record of equal 32-bit hash is a candidate (repeats
// and hash collisions included: two strings within two edits share a variant,
// so no neighbour is missed), and each distinct candidate is checked with the
// exact bit-parallel distance, the query being the pattern.

// Length of a canonical string: the number of its nonzero 5-bit codes.
__device__ __forceinline__ int canon_len(const Canon& c) {
    constexpr uint64_t kFieldLow = 0x84210842108421ull;  // bit 0 of each of the 12 fields
    int L = 0;
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const uint64_t x = c.w[w] & ~kTagBits;
        L += __popcll((x | (x >> 1) | (x >> 2) | (x >> 3) | (x >> 4)) & kFieldLow);
    }
    return L;
}

// This lane's share of the variants of c (length L): the full string (lane 0)
// and every variant whose first deletion is at position lane or lane + 32.
template <typename Fn>
__device__ __forceinline__ void lane_variants2(const Canon& c, int L, int lane, Fn fn) {
    if (lane == 0) fn(c);
    for (int p = lane; p < L; p += 32) {
        if (!run_start(c, p)) continue;
        const Canon d = delete_at(c, p);
        fn(d);
        for (int q = p + 1; q < L; ++q)
            if (q == p + 1 || run_start(c, q)) fn(delete_at(d, q - 1));  // position q of c is q - 1 of d
    }
}

// Candidates of each query, a warp per query: COUNT stores their number in
// qcnt[j]; WRITE stores the candidate strings at qoff[j] onwards (slots from a
// per-warp counter; both passes see the same records).
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_q2_cand(IndexView ix, const Canon* __restrict__ qcanon, const uint8_t* __restrict__ qlen, int64_t m,
          int64_t* __restrict__ qcnt, const int64_t* __restrict__ qoff, int32_t* __restrict__ out) {
    __shared__ unsigned long long wpos[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        const Canon c = load_canon(qcanon + j);
        const int L = qlen[j];
        const int64_t base = WRITE ? qoff[j] : 0;
        if (lane == 0) wpos[w] = 0;
        __syncwarp();
        long long cnt = 0;
        lane_variants2(c, L, lane, [&](const Canon& v) {
            const uint64_t h = hash_canon(v);
            const uint32_t pid = part_of(h, ix.P);
            for (int64_t k = ix.poff[pid], k1 = ix.poff[pid + 1]; k < k1; ++k) {
                const uint64_t r = ix.recs[k];
                if ((uint32_t)(r >> 32) != (uint32_t)h) continue;
                if constexpr (!WRITE) ++cnt;
                else out[base + (int64_t)atomicAdd(&wpos[w], 1ull)] = (int32_t)(uint32_t)r;
            }
        });
        if constexpr (!WRITE) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
            if (lane == 0) qcnt[j] = cnt;
        }
        __syncwarp();
    }
}

// Each query's distinct candidates (sorted row, repeats adjacent) checked with
// the bit-parallel distance (Myers 1999, Hyyro 2001), the query's letter masks
// in shared memory (lane k builds letter k + 1's), the candidate as the text:
// flag[e] = 1 for a resident string within two edits, and ocnt[j] = the total
// of their member counts.
__global__ void __launch_bounds__(kThreads)
k_q2_verify(IndexView ix, const Canon* __restrict__ qcanon, const uint8_t* __restrict__ qlen, int64_t m,
            const int64_t* __restrict__ coff, const int32_t* __restrict__ ccols, uint8_t* __restrict__ flag,
            int64_t* __restrict__ ocnt) {
    __shared__ uint64_t speq[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        const Canon cq = load_canon(qcanon + j);
        const int Lq = qlen[j];
        uint64_t mk = 0;
        for (int k = 0; k < Lq; ++k)
            if (code_at(cq, k) == (uint32_t)(lane + 1)) mk |= 1ull << k;
        speq[w][lane] = mk;
        __syncwarp();
        const uint64_t top = 1ull << (Lq - 1);
        long long tot = 0;
        const int64_t a = coff[j], b = coff[j + 1];
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t u = ccols[e];
            uint8_t f = 0;
            if (e == a || ccols[e - 1] != u) {  // first of its repeats
                const Canon cu = load_canon(ix.ucanon + u);
                const int Lu = canon_len(cu);
                if (Lu - Lq <= 2 && Lq - Lu <= 2) {
                    uint64_t vp = ~0ull, vn = 0;
                    int score = Lq;
                    for (int k = 0; k < Lu; ++k) {
                        const uint64_t eq = speq[w][code_at(cu, k) - 1];
                        const uint64_t xv = eq | vn;
                        const uint64_t xh = (((eq & vp) + vp) ^ vp) | eq;
                        uint64_t hp = vn | ~(xh | vp);
                        uint64_t hn = vp & xh;
                        score += ((hp & top) ? 1 : 0) - ((hn & top) ? 1 : 0);
                        hp = (hp << 1) | 1ull;
                        hn <<= 1;
                        vp = hn | ~(xv | hp);
                        vn = hp & xv;
                    }
                    f = score <= 2 ? 1 : 0;
                }
            }
            flag[e] = f;
            if (f) tot += ix.umult[u];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(kFull, tot, d);
        if (lane == 0) ocnt[j] = tot;
        __syncwarp();
    }
}

// The members of each query's accepted resident strings into its row at
// ooff[j] onwards (a warp per query, the lanes over each member list).
__global__ void __launch_bounds__(kThreads)
k_q2_emit(IndexView ix, int64_t m, const int64_t* __restrict__ coff, const int32_t* __restrict__ ccols,
          const uint8_t* __restrict__ flag, const int64_t* __restrict__ ooff, int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        int64_t pos = ooff[j];
        const int64_t a = coff[j], b = coff[j + 1];
        for (int64_t e0 = a; e0 < b; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool f = e < b && flag[e];
            const int32_t u = f ? ccols[e] : 0;
            for (unsigned bal = __ballot_sync(kFull, f); bal; bal &= bal - 1) {
                const int32_t uu = __shfl_sync(kFull, u, __ffs(bal) - 1);
                const int64_t m0 = ix.mem_off[uu], m1 = ix.mem_off[uu + 1];
                for (int64_t k = m0 + lane; k < m1; k += 32) out[pos + (k - m0)] = ix.members[k];
                pos += m1 - m0;
            }
        }
    }
}

}  // namespace

// l_max = 2: candidates of the query strings' variants, sorted per query,
// checked, then the accepted strings' members, sorted per query.
static tcrnet_status deletion_query2(const DeletionIndex& ix, const Packed& q, DevBuf& off64, DevBuf& cols,
                                     DevBuf& count, int64_t* nnz_out, cudaStream_t s, int num_sms) {
    const int64_t m = q.n;
    IndexView v{ix.ucanon, ix.umult, ix.mem_off, ix.members, ix.recs, ix.poff, (uint32_t)ix.P};
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(m, kWarps), (int64_t)num_sms * 32);
    DevBuf qcnt, coff, ccols, flag, ocnt;
    TCR_CHECK(qcnt.alloc(sizeof(int64_t) * m, s));
    TCR_CHECK(coff.alloc(sizeof(int64_t) * (m + 1), s));
    k_q2_cand<false><<<grid, kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m,
                                               qcnt.as<int64_t>(), nullptr, nullptr);
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i64(qcnt.as<int64_t>(), coff.as<int64_t>(), m, s));
    int64_t NC = 0;
    TCR_CUDA(cudaMemcpyAsync(&NC, coff.as<int64_t>() + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    TCR_CHECK(ccols.alloc(sizeof(int32_t) * std::max<int64_t>(NC, 1), s));
    TCR_CHECK(flag.alloc(std::max<int64_t>(NC, 1), s));
    TCR_CHECK(ocnt.alloc(sizeof(int64_t) * m, s));
    if (NC > 0) {
        k_q2_cand<true><<<grid, kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m, nullptr,
                                                  coff.as<int64_t>(), ccols.as<int32_t>());
        TCR_LAUNCH_CHECK();
        TCR_CHECK(sort_rows(coff.as<int64_t>(), ccols.as<int32_t>(), m, s, num_sms));
    }
    k_q2_verify<<<grid, kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m, coff.as<int64_t>(),
                                          ccols.as<int32_t>(), flag.as<uint8_t>(), ocnt.as<int64_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(off64.alloc_owned(sizeof(int64_t) * (m + 1), s));
    TCR_CHECK(scan_exclusive_i64(ocnt.as<int64_t>(), off64.as<int64_t>(), m, s));
    int64_t nnz = 0;
    TCR_CUDA(cudaMemcpyAsync(&nnz, off64.as<int64_t>() + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    TCR_CHECK(cols.alloc_owned(sizeof(int32_t) * nnz, s));
    TCR_CHECK(count.alloc_owned(sizeof(int32_t) * m, s));
    if (nnz > 0) {
        k_q2_emit<<<grid, kThreads, 0, s>>>(v, m, coff.as<int64_t>(), ccols.as<int32_t>(), flag.as<uint8_t>(),
                                            off64.as<int64_t>(), cols.as<int32_t>());
        TCR_LAUNCH_CHECK();
        TCR_CHECK(sort_rows(off64.as<int64_t>(), cols.as<int32_t>(), m, s, num_sms));
    }
    TCR_CHECK(degree_from_offsets(off64.as<int64_t>(), count.as<int32_t>(), m, s));
    *nnz_out = nnz;
    return TCRNET_OK;
}

tcrnet_status deletion_query(const DeletionIndex& ix, const Packed& q, int T, DevBuf& off64, DevBuf& cols,
                             DevBuf& count, int64_t* nnz_out, cudaStream_t s, int num_sms) {
    const int64_t m = q.n;
    *nnz_out = 0;
    if (!ix.valid()) return TCRNET_ESTATE;
    if (T == 2) return deletion_query2(ix, q, off64, cols, count, nnz_out, s, num_sms);
    IndexView v{ix.ucanon, ix.umult, ix.mem_off, ix.members, ix.recs, ix.poff, (uint32_t)ix.P};
    DevBuf qcnt;
    TCR_CHECK(qcnt.alloc(sizeof(int64_t) * m, s));
    TCR_CHECK(off64.alloc_owned(sizeof(int64_t) * (m + 1), s));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(m, kWarps), (int64_t)num_sms * 32);
    // the count pass keeps its matches (up to kHitsPerQuery per query on
    // average); when they all fit, an emit pass over them replaces the second
    // scan of the partitions
    constexpr int64_t kHitsPerQuery = 64;
    const int64_t hit_cap = std::max<int64_t>(1 << 16, std::min<int64_t>(kHitsPerQuery * m, 1LL << 27));
    DevBuf hitbuf, hitcur;
    int2* hits = nullptr;
    if (hitbuf.alloc(sizeof(int2) * hit_cap, s) == TCRNET_OK &&
        hitcur.alloc(sizeof(unsigned long long), s) == TCRNET_OK) {
        TCR_CUDA(cudaMemsetAsync(hitcur.as<void>(), 0, sizeof(unsigned long long), s));
        hits = hitbuf.as<int2>();
    }
    k_query<false><<<grid, kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m, T,
                                             qcnt.as<int64_t>(), nullptr, nullptr, hits,
                                             hits ? hitcur.as<unsigned long long>() : nullptr, hit_cap);
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i64(qcnt.as<int64_t>(), off64.as<int64_t>(), m, s));
    int64_t nnz = 0;
    unsigned long long nh = ~0ull;
    {
        const void* src[2] = {off64.as<int64_t>() + m, hits ? hitcur.as<void>() : nullptr};
        void* dst[2] = {&nnz, &nh};
        const size_t bytes[2] = {sizeof(int64_t), sizeof(nh)};
        TCR_CHECK(read_back(s, hits ? 2 : 1, src, dst, bytes));
    }
    TCR_CHECK(cols.alloc_owned(sizeof(int32_t) * nnz, s));
    TCR_CHECK(count.alloc_owned(sizeof(int32_t) * m, s));
    if (nnz > 0) {
        if (hits && (int64_t)nh <= hit_cap) {
            DevBuf qcur;
            TCR_CHECK(qcur.alloc(sizeof(int32_t) * m, s));
            TCR_CUDA(cudaMemsetAsync(qcur.as<void>(), 0, sizeof(int32_t) * m, s));
            const unsigned egrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)nh, kThreads),
                                                                                     (int64_t)num_sms * 16));
            k_query_emit<<<egrid, kThreads, 0, s>>>(v, hits, (int64_t)nh, off64.as<int64_t>(), qcur.as<int32_t>(),
                                                    cols.as<int32_t>());
        } else {
            k_query<true><<<grid, kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m, T, nullptr,
                                                    off64.as<int64_t>(), cols.as<int32_t>(), nullptr, nullptr, 0);
        }
        TCR_LAUNCH_CHECK();
        TCR_CHECK(sort_rows(off64.as<int64_t>(), cols.as<int32_t>(), m, s, num_sms));
    }
    TCR_CHECK(degree_from_offsets(off64.as<int64_t>(), count.as<int32_t>(), m, s));
    *nnz_out = nnz;
    return TCRNET_OK;
}

// ---- merging new strings into a resident network ----------------------------
//
// The network of a repertoire grown by m strings differs from the old one by
// the rows of the new nodes and by new entries appended to old rows (new ids
// are larger than every old id, so an old row stays sorted when they are
// appended in ascending order). The index is grown first: a new string equal
// to a resident distinct string joins its member list; the others become
// fresh distinct strings whose records are added to the same hash partitions.
// Every edge that involves a new string is then found by the query of the new
// strings against the grown index (a row lists the string itself as well).

namespace {

// Distinct id of each new string: the resident distinct string it equals
// (found through the full-string record of its partition), else a slot of a
// table of the new strings; the string that claims a slot numbers a fresh
// distinct string (u0 + running count) and is its representative.
__global__ void k_ins_dedup(IndexView ix, const Canon* __restrict__ qcanon, const uint8_t* __restrict__ qlen,
                            int64_t m, int32_t* __restrict__ table, uint32_t mask, int32_t* __restrict__ slot_of,
                            int32_t* __restrict__ slot_u, unsigned long long* __restrict__ fresh, uint32_t u0,
                            Canon* __restrict__ ucanon_new, uint8_t* __restrict__ flen, int32_t* __restrict__ nuid,
                            uint8_t* __restrict__ is_rep, int* __restrict__ err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const Canon c = load_canon(qcanon + j);
    const uint64_t h = hash_canon(c);
    const uint32_t pid = part_of(h, ix.P);
    for (int64_t k = ix.poff[pid], k1 = ix.poff[pid + 1]; k < k1; ++k) {
        const uint64_t r = ix.recs[k];
        if ((uint32_t)(r >> 32) == (uint32_t)h && rec_p(r) == kTagF && canon_eq(c, load_canon(ix.ucanon + rec_u(r)))) {
            nuid[j] = (int32_t)rec_u(r);
            slot_of[j] = -1;
            is_rep[j] = 0;
            return;
        }
    }
    uint32_t slot = (uint32_t)h & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t r = atomicCAS(&table[slot], -1, (int32_t)j);
        if (r == -1) {
            const uint32_t f = (uint32_t)atomicAdd(fresh, 1ull);
            slot_u[slot] = (int32_t)(u0 + f);
            store_canon(ucanon_new + u0 + f, c);
            flen[f] = qlen[j];
            slot_of[j] = (int32_t)slot;
            is_rep[j] = 1;
            return;
        }
        if (canon_eq(load_canon(qcanon + r), c)) {
            slot_of[j] = (int32_t)slot;
            is_rep[j] = 0;
            return;
        }
        slot = (slot + 1) & mask;
    }
    atomicExch(err, 1);  // unreachable: the table has at least 2m slots
    slot_of[j] = -1;
    nuid[j] = 0;
    is_rep[j] = 0;
}

// Fresh ids resolved (their slots are all numbered now); node ids and
// multiplicities of the grown repertoire.
__global__ void k_ins_uid(const int32_t* __restrict__ slot_of, const int32_t* __restrict__ slot_u, int64_t m,
                          int64_t n0, int32_t* __restrict__ nuid, int32_t* __restrict__ uid_new,
                          int32_t* __restrict__ umult_new) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t sl = slot_of[j];
    const int32_t u = sl >= 0 ? slot_u[sl] : nuid[j];
    nuid[j] = u;
    uid_new[n0 + j] = u;
    atomicAdd(&umult_new[u], 1);
}

// Partition starts after the new records (poff_new = poff + exclusive counts of
// the new records) and the slot cursor of each partition: the absolute position
// after its old records (positions fit int32: at most 2^25 strings of 48
// letters, 1.6e9 records).
__global__ void k_ins_part_base(const int64_t* __restrict__ poff, const int64_t* __restrict__ pscan, int64_t P,
                                int64_t* __restrict__ poff_new, int32_t* __restrict__ pcur) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    poff_new[p] = poff[p] + pscan[p];
    if (p < P) pcur[p] = (int32_t)(poff[p] + pscan[p] + poff[p + 1] - poff[p]);  // after the partition's old records
}

// Segments (rows, partitions) that grow: flag[i] = grow[i] > 0.
__global__ void k_ins_flags(const int32_t* __restrict__ grow, int64_t R, int32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) flag[i] = grow[i] > 0 ? 1 : 0;
}

// Cuts of a segmented array whose segments grow at their ends: the old
// elements after the end of the k-th growing segment move by shifts[k + 1]
// (shifts[0] = 0: elements before the first cut stay).
template <typename OffT>
__global__ void k_ins_cuts(const int32_t* __restrict__ grow, const OffT* __restrict__ old_off,
                           const int64_t* __restrict__ new_off, int64_t R, const int64_t* __restrict__ pos,
                           int64_t* __restrict__ cuts, int64_t* __restrict__ shifts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R || grow[i] <= 0) return;
    const int64_t k = pos[i];
    const int64_t end = (int64_t)old_off[i + 1];
    cuts[k] = end;
    shifts[k + 1] = new_off[i + 1] - end;
}


// Distinct strings that the new strings take: the first new string of each
// (first[u] = smallest j) represents it.
__global__ void k_ins_first(const int32_t* __restrict__ nuid, int64_t m, unsigned* __restrict__ first) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) atomicMin(&first[nuid[j]], (unsigned)j);
}

__global__ void k_ins_rep_flags(const int32_t* __restrict__ nuid, int64_t m, const unsigned* __restrict__ first,
                                int32_t* __restrict__ flag) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) flag[j] = first[nuid[j]] == (unsigned)j ? 1 : 0;
}

// Representatives in new-string order: their strings (the query input), their
// distinct ids and the row index of each represented distinct string.
__global__ void k_ins_reps(const int32_t* __restrict__ nuid, int64_t m, const unsigned* __restrict__ first,
                           const int64_t* __restrict__ rpos, const Canon* __restrict__ qcanon,
                           const uint8_t* __restrict__ qlen, Canon* __restrict__ rcanon, uint8_t* __restrict__ rlen,
                           int32_t* __restrict__ rep_u, int32_t* __restrict__ ridx) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t u = nuid[j];
    if (first[u] != (unsigned)j) return;
    const int64_t r = rpos[j];
    store_canon(rcanon + r, load_canon(qcanon + j));
    rlen[r] = qlen[j];
    rep_u[r] = u;
    ridx[u] = (int32_t)r;
}

// New members of each represented distinct string (new-string ids j).
__global__ void k_ins_new_members(const int32_t* __restrict__ nuid, int64_t m, const int32_t* __restrict__ ridx,
                                  const int64_t* __restrict__ nm_off, int32_t* __restrict__ nm_cur,
                                  int32_t* __restrict__ nm_list, int32_t* __restrict__ nm_cnt, bool place) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t r = ridx[nuid[j]];
    if (!place) atomicAdd(&nm_cnt[r], 1);
    else nm_list[nm_off[r] + atomicAdd(&nm_cur[r], 1)] = (int32_t)j;
}

// Number of entries of the ascending array a[0 .. K) that are <= x: a 32-way
// search (each step probes 32 evenly spaced entries, whose hits form a prefix),
// taken by the whole warp, which gets the result in every lane.
__device__ __forceinline__ int64_t warp_count_le(const int64_t* __restrict__ a, int64_t K, int64_t x) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = K;  // a[< lo] <= x < a[>= hi]
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t idx = lo + lane * step;
        const int c = __popc(__ballot_sync(kFull, idx < hi && a[idx] <= x));
        if (c == 0) return lo;
        const int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
        hi = lo + (int64_t)c * step < hi ? lo + (int64_t)c * step : hi;
        lo = nlo;
    }
    return lo + __popc(__ballot_sync(kFull, lo + lane < hi && a[lo + lane] <= x));
}

// The closed rows' entries [0, nr) are taken in chunks of kRowChunk consecutive
// entries, a warp per chunk, so that a row of many members (a string shared by
// a large part of the repertoire) is spread over many warps. A warp finds the
// row of its first entry by warp_count_le; each lane then steps forward to the
// row of its own entry (rows are consecutive), and lane 31's row starts the
// next 32 entries.
constexpr int kRowChunk = 256;

template <typename Body>
__device__ __forceinline__ void for_row_entries(const int64_t* __restrict__ roff, int64_t nrows, int64_t nr,
                                                Body body) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t chunks = (nr + kRowChunk - 1) / kRowChunk;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < chunks; c += nw) {
        const int64_t e0 = c * kRowChunk;
        const int64_t e1 = e0 + kRowChunk < nr ? e0 + kRowChunk : nr;
        int64_t r = warp_count_le(roff + 1, nrows, e0);
        for (int64_t t0 = e0; t0 < e1; t0 += 32) {
            const int64_t e = t0 + lane;
            int64_t rl = r;
            if (e < e1)
                while (roff[rl + 1] <= e) ++rl;  // e < roff[nrows]: ends within the rows
            body(e < e1, e, rl);
            r = __shfl_sync(kFull, rl, 31);
        }
    }
}

// Edges between distinct strings that involve a fresh one: for each fresh
// distinct string w (a row of its closed neighbourhood), every other distinct
// string x in the row (all members of a neighbour are listed; its first member
// stands for it); a pair of fresh strings is taken from the smaller id's side.
__global__ void k_ins_edges(const int64_t* __restrict__ roff, const int32_t* __restrict__ rcols, int64_t nrep,
                            int64_t nr, const int32_t* __restrict__ rep_u, const int32_t* __restrict__ uid,
                            const int64_t* __restrict__ mem_off, const int32_t* __restrict__ members, int64_t U0,
                            int2* __restrict__ out, unsigned long long* __restrict__ cur, int64_t cap,
                            int* __restrict__ err) {
    for_row_entries(roff, nrep, nr, [&](bool ok, int64_t e, int64_t r) {
        if (!ok) return;
        const int32_t w = rep_u[r];
        if (w < U0) return;  // a resident string: its edges are known
        const int32_t i = rcols[e];
        const int32_t x = uid[i];
        if (x == w || (x >= U0 && x < w) || members[mem_off[x]] != i) return;
        const unsigned long long slot = atomicAdd(cur, 1ull);
        if ((int64_t)slot < cap) out[slot] = make_int2(w, x);
        else atomicExch(err, 1);
    });
}

// New entries of old rows. An old node i gains every new member of every
// represented string whose closed row lists it; that set depends only on i's
// distinct string x (all members of x are listed together), so it is built
// once per x (its "tail") and copied to each old member of x. A closed row
// stands for x by x's first old member. dcnt[x] = tail length of x.
__global__ void k_ins_tail_count(const int64_t* __restrict__ roff, const int32_t* __restrict__ rcols, int64_t nrep,
                                 int64_t nr, const int32_t* __restrict__ nm_cnt, int64_t n0,
                                 const int32_t* __restrict__ uid, const int64_t* __restrict__ mem_off_old,
                                 const int32_t* __restrict__ members_old, int32_t* __restrict__ dcnt) {
    for_row_entries(roff, nrep, nr, [&](bool ok, int64_t e, int64_t r) {
        if (!ok) return;
        const int32_t i = rcols[e];
        if (i >= n0) return;
        const int32_t x = uid[i];
        if (members_old[mem_off_old[x]] == i) atomicAdd(&dcnt[x], nm_cnt[r]);
    });
}

// Tails of the old distinct strings: x takes n0 + j for the new members j of
// every closed row that stands for it, at slots of its tail (sorted
// afterwards). A lane writes up to 4 new members itself; longer lists are
// written by the whole warp, one entry's list after another.
__global__ void k_ins_tails(const int64_t* __restrict__ roff, const int32_t* __restrict__ rcols, int64_t nrep,
                            int64_t nr, const int64_t* __restrict__ nm_off, const int32_t* __restrict__ nm_list,
                            int64_t n0, const int32_t* __restrict__ uid, const int64_t* __restrict__ mem_off_old,
                            const int32_t* __restrict__ members_old, const int64_t* __restrict__ dtoff,
                            int32_t* __restrict__ dcur, int32_t* __restrict__ dtcols) {
    const int lane = threadIdx.x & 31;
    for_row_entries(roff, nrep, nr, [&](bool ok, int64_t e, int64_t r) {
        int64_t base = -1, a = 0;
        int32_t c = 0;
        if (ok) {
            const int32_t i = rcols[e];
            if (i < n0) {
                const int32_t x = uid[i];
                if (members_old[mem_off_old[x]] == i) {
                    a = nm_off[r];
                    c = (int32_t)(nm_off[r + 1] - a);
                    base = dtoff[x] + atomicAdd(&dcur[x], c);
                }
            }
        }
        if (base >= 0 && c <= 4)
            for (int32_t k = 0; k < c; ++k) dtcols[base + k] = (int32_t)(n0 + nm_list[a + k]);
        unsigned todo = __ballot_sync(kFull, base >= 0 && c > 4);
        while (todo) {
            const int t = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t tb = __shfl_sync(kFull, base, t);
            const int64_t ta = __shfl_sync(kFull, a, t);
            const int32_t tc = __shfl_sync(kFull, c, t);
            for (int32_t k = lane; k < tc; k += 32) dtcols[tb + k] = (int32_t)(n0 + nm_list[ta + k]);
        }
    });
}

// Degrees of the grown network (old node: + its string's tail; new node: its
// closed row minus itself) and the growth of each old row.
__global__ void k_ins_degree(const int32_t* __restrict__ deg_old, const int32_t* __restrict__ dcnt,
                             const int32_t* __restrict__ uid, int64_t n0, const int32_t* __restrict__ nuid,
                             const int32_t* __restrict__ ridx, const int32_t* __restrict__ rcnt, int64_t m,
                             int32_t* __restrict__ delta, int32_t* __restrict__ deg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n0) {
        const int32_t d = dcnt[uid[i]];
        delta[i] = d;
        deg[i] = deg_old[i] + d;
    } else if (i < n0 + m) {
        deg[i] = rcnt[ridx[nuid[i - n0]]] - 1;
    }
}

// Tails copied after the old entries of each old row: a lane per row for short
// tails, the whole warp for long ones.
template <typename OffT>
__global__ void k_ins_fill_tails(const OffT* __restrict__ old_off, const int64_t* __restrict__ new_off,
                                 const int32_t* __restrict__ uid, const int32_t* __restrict__ dcnt,
                                 const int64_t* __restrict__ dtoff, const int32_t* __restrict__ dtcols, int64_t n0,
                                 int32_t* __restrict__ cols) {
    constexpr int kLaneTail = 8;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; i0 < n0; i0 += nw * 32) {
        const int64_t i = i0 + lane;
        int32_t len = 0;
        int64_t src = 0, dst = 0;
        if (i < n0) {
            const int32_t x = uid[i];
            len = dcnt[x];
            if (len > 0) {
                src = dtoff[x];
                dst = new_off[i] + ((int64_t)old_off[i + 1] - (int64_t)old_off[i]);
                if (len <= kLaneTail)
                    for (int32_t k = 0; k < len; ++k) cols[dst + k] = dtcols[src + k];
            }
        }
        unsigned todo = __ballot_sync(kFull, len > kLaneTail);
        while (todo) {
            const int t = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t ts = __shfl_sync(kFull, src, t), td = __shfl_sync(kFull, dst, t);
            const int32_t tl = __shfl_sync(kFull, len, t);
            for (int32_t k = lane; k < tl; k += 32) cols[td + k] = dtcols[ts + k];
        }
    }
}

// Rows of the new nodes: the closed row of their distinct string (ascending)
// without the node itself, a warp per node.
__global__ void k_ins_fill_new(const int64_t* __restrict__ roff, const int32_t* __restrict__ rcols,
                               const int32_t* __restrict__ nuid, const int32_t* __restrict__ ridx, int64_t m,
                               int64_t n0, const int64_t* __restrict__ new_off, int32_t* __restrict__ cols) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        const int32_t self = (int32_t)(n0 + j);
        const int32_t r = ridx[nuid[j]];
        int32_t* row = cols + new_off[n0 + j];
        const int64_t q0 = roff[r], len = roff[r + 1] - q0;
        for (int64_t e = lane; e < len; e += 32) {
            const int32_t v = rcols[q0 + e];
            const int64_t at = e - (v > self ? 1 : 0);
            if (v != self && at < len - 1) row[at] = v;
        }
    }
}

// Cuts of a segmented array (segment i = [old_off[i], old_off[i+1]) grows by
// grow[i] at its end; new_off = the grown offsets): K (on the device), cuts
// and shifts for k_shifted_copy.
template <typename OffT>
tcrnet_status growth_cuts(const int32_t* grow, const OffT* old_off, const int64_t* new_off, int64_t R,
                          int64_t max_cuts, DevBuf& cuts, DevBuf& shifts, DevBuf& pos, cudaStream_t s) {
    DevBuf flag;
    TCR_CHECK(flag.alloc(sizeof(int32_t) * (R > 0 ? R : 1), s));
    TCR_CHECK(pos.alloc(sizeof(int64_t) * (R + 1), s));
    TCR_CHECK(cuts.alloc(sizeof(int64_t) * (max_cuts > 0 ? max_cuts : 1), s));
    TCR_CHECK(shifts.alloc(sizeof(int64_t) * (max_cuts + 1), s));
    TCR_CUDA(cudaMemsetAsync(shifts.as<void>(), 0, sizeof(int64_t), s));
    if (R == 0) {
        TCR_CUDA(cudaMemsetAsync(pos.as<void>(), 0, sizeof(int64_t), s));
        return TCRNET_OK;
    }
    k_ins_flags<<<grid_for(R), kThreads, 0, s>>>(grow, R, flag.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(flag.as<int32_t>(), pos.as<int64_t>(), R, s));
    k_ins_cuts<OffT><<<grid_for(R), kThreads, 0, s>>>(grow, old_off, new_off, R, pos.as<int64_t>(),
                                                       cuts.as<int64_t>(), shifts.as<int64_t>());
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

// dst[t + shifts[k(t)]] = src[t], k(t) = number of cuts <= t (cuts sorted,
// possibly equal). Each warp moves one contiguous range: it finds the piece of
// its first element by a 32-way search over the cuts, then copies 32
// consecutive elements per instruction (coalesced), each lane advancing the
// piece index to its own element, whether the pieces are long (few rows grow)
// or a few dozen elements (many do).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_shifted_copy(const T* __restrict__ src, T* __restrict__ dst,
                                                           int64_t count, const int64_t* __restrict__ cuts,
                                                           const int64_t* __restrict__ shifts,
                                                           const int64_t* __restrict__ K_ptr) {
    const int lane = threadIdx.x & 31;
    const int64_t K = *K_ptr;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t per = ((count + nw - 1) / nw + 31) / 32 * 32;
    const int64_t b0 = gw * per;
    const int64_t b1 = b0 + per < count ? b0 + per : count;
    if (b0 >= b1) return;  // warp-uniform
    // 128 consecutive elements per step (loads first), starting in the piece
    // of b0 (the first k with cuts[k] > b0); each lane advances a copy of the
    // warp's piece index to its own element, lane 31's result carries on
    int64_t k = warp_count_le(cuts, K, b0);
    for (int64_t t0 = b0; t0 < b1; t0 += 128) {
        T v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t t = t0 + 32 * r + lane;
            if (t < b1) v[r] = src[t];
        }
        while (k < K && cuts[k] <= t0) ++k;
        if (k >= K || cuts[k] >= t0 + 128) {  // the whole step lies in piece k
            const int64_t sh = shifts[k];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t t = t0 + 32 * r + lane;
                if (t < b1) dst[t + sh] = v[r];
            }
            continue;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t t = t0 + 32 * r + lane;
            int64_t kl = k;
            if (t < b1) {
                while (kl < K && cuts[kl] <= t) ++kl;
                dst[t + shifts[kl]] = v[r];
            }
            k = __shfl_sync(kFull, kl, 31);
        }
    }
}

template <typename T>
tcrnet_status shifted_copy(const T* src, T* dst, int64_t count, const DevBuf& cuts, const DevBuf& shifts,
                           const int64_t* K_dev, cudaStream_t s, int num_sms) {
    if (count <= 0) return TCRNET_OK;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(count, (int64_t)kThreads * 64),
                                                                   (int64_t)num_sms * 16));
    k_shifted_copy<T><<<(unsigned)blocks, kThreads, 0, s>>>(src, dst, count, cuts.as<int64_t>(), shifts.as<int64_t>(),
                                                            K_dev);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

template <typename OffT>
tcrnet_status csr_merge(const CsrView& g, const OffT* old_off, const int32_t* delta, int64_t n_tail,
                        const int64_t* new_off, const int32_t* uid, const int32_t* dcnt, const int64_t* dtoff,
                        const int32_t* dtcols, const int64_t* roff, const int32_t* rcols, const int32_t* nuid,
                        const int32_t* ridx, int64_t m, int32_t* cols, cudaStream_t s, int num_sms) {
    const int64_t n0 = g.n;
    DevBuf cuts, shifts, pos;
    TCR_CHECK(growth_cuts<OffT>(delta, old_off, new_off, n0, std::min<int64_t>(n0, n_tail), cuts, shifts, pos, s));
    TCR_CHECK(shifted_copy<int32_t>(g.cols, cols, g.nnz, cuts, shifts, pos.as<int64_t>() + n0, s, num_sms));
    if (n_tail > 0) {
        k_ins_fill_tails<OffT><<<(unsigned)std::min<int64_t>(ceil_div(n0, 32 * kWarps), (int64_t)num_sms * 16),
                                 kThreads, 0, s>>>(old_off, new_off, uid, dcnt, dtoff, dtcols, n0, cols);
        TCR_LAUNCH_CHECK();
    }
    const unsigned wgrid = (unsigned)std::min<int64_t>(ceil_div(m, kWarps), (int64_t)num_sms * 16);
    k_ins_fill_new<<<wgrid, kThreads, 0, s>>>(roff, rcols, nuid, ridx, m, n0, new_off, cols);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

}  // namespace

tcrnet_status deletion_insert(const DeletionIndex& ix, const CsrView& g, const Packed& q, int T, InsertResult& out,
                              cudaStream_t s, int num_sms, bool profile) {
    const int64_t m = q.n, n0 = g.n, N = n0 + m;
    const int64_t U0 = ix.U, P = ix.P, R0 = ix.R, E0 = ix.E;
    if (!ix.valid() || !ix.uid || ix.n != n0 || m <= 0 || N > kDeletionMaxN || T < 1) return TCRNET_ESTATE;
    Timer tm(profile, s);
    const int t0 = tm.mark();
    IndexView v{ix.ucanon, ix.umult, ix.mem_off, ix.members, ix.recs, ix.poff, (uint32_t)P};

    // 1. distinct ids of the new strings (resident or fresh); ids,
    //    multiplicities and member lists of the grown repertoire
    DevBuf errb, counters;
    TCR_CHECK(errb.alloc(sizeof(int) * 4, s));
    TCR_CHECK(counters.alloc(sizeof(unsigned long long) * 2, s));  // [0] fresh strings, [1] new edges
    TCR_CUDA(cudaMemsetAsync(errb.as<void>(), 0, sizeof(int) * 4, s));
    TCR_CUDA(cudaMemsetAsync(counters.as<void>(), 0, sizeof(unsigned long long) * 2, s));
    int* d_err = errb.as<int>();
    unsigned long long* d_fresh = counters.as<unsigned long long>();
    unsigned long long* d_ecur = d_fresh + 1;
    int64_t S = 1024;
    while (S < 2 * m) S <<= 1;
    DevBuf table, slot_of, slot_u, flen, nuid, is_rep;
    TCR_CHECK(table.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(slot_u.alloc(sizeof(int32_t) * S, s));
    TCR_CHECK(slot_of.alloc(sizeof(int32_t) * m, s));
    TCR_CHECK(flen.alloc(m, s));
    TCR_CHECK(nuid.alloc(sizeof(int32_t) * m, s));
    TCR_CHECK(is_rep.alloc(m, s));
    TCR_CUDA(cudaMemsetAsync(table.as<void>(), 0xff, sizeof(int32_t) * S, s));
    // index arrays of the grown repertoire, sized for N strings like a build's
    DevBuf ucanon, umult, uid, mem_off, members, mcur, mpos;
    TCR_CHECK(ucanon.alloc_owned(sizeof(Canon) * N, s));
    TCR_CHECK(umult.alloc_owned(sizeof(int32_t) * N, s));
    TCR_CHECK(uid.alloc_owned(sizeof(int32_t) * N, s));
    TCR_CHECK(mem_off.alloc_owned(sizeof(int64_t) * (N + 1), s));
    TCR_CHECK(members.alloc_owned(sizeof(int32_t) * N, s));
    TCR_CHECK(mcur.alloc(sizeof(int32_t) * N, s));
    TCR_CHECK(mpos.alloc(sizeof(int32_t) * N, s));
    if (U0 > 0)
        TCR_CUDA(cudaMemcpyAsync(ucanon.as<void>(), ix.ucanon, sizeof(Canon) * U0, cudaMemcpyDeviceToDevice, s));
    TCR_CUDA(cudaMemcpyAsync(umult.as<void>(), ix.umult, sizeof(int32_t) * n0, cudaMemcpyDeviceToDevice, s));
    TCR_CUDA(cudaMemsetAsync(umult.as<int32_t>() + n0, 0, sizeof(int32_t) * m, s));
    TCR_CUDA(cudaMemcpyAsync(uid.as<void>(), ix.uid, sizeof(int32_t) * n0, cudaMemcpyDeviceToDevice, s));
    k_ins_dedup<<<grid_for(m), kThreads, 0, s>>>(v, q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), m,
                                                 table.as<int32_t>(), (uint32_t)(S - 1), slot_of.as<int32_t>(),
                                                 slot_u.as<int32_t>(), d_fresh, (uint32_t)U0, ucanon.as<Canon>(),
                                                 flen.as<uint8_t>(), nuid.as<int32_t>(), is_rep.as<uint8_t>(), d_err);
    TCR_LAUNCH_CHECK();
    k_ins_uid<<<grid_for(m), kThreads, 0, s>>>(slot_of.as<int32_t>(), slot_u.as<int32_t>(), m, n0,
                                               nuid.as<int32_t>(), uid.as<int32_t>(), umult.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(umult.as<int32_t>(), mem_off.as<int64_t>(), N, s));
    TCR_CUDA(cudaMemsetAsync(mcur.as<void>(), 0, sizeof(int32_t) * N, s));
    k_members<<<grid_for(N), kThreads, 0, s>>>(uid.as<int32_t>(), N, mem_off.as<int64_t>(), mcur.as<int32_t>(),
                                               members.as<int32_t>(), mpos.as<int32_t>());
    TCR_LAUNCH_CHECK();
    const int t1 = tm.mark();

    // 2. records of the fresh strings into the same partitions
    const int64_t R_bound = R0 + m + q.lensum;
    DevBuf pcnt, pscan, poff, recs;
    TCR_CHECK(pcnt.alloc(sizeof(int32_t) * P, s));
    TCR_CHECK(pscan.alloc(sizeof(int64_t) * (P + 1), s));
    TCR_CHECK(poff.alloc_owned(sizeof(int64_t) * (P + 1), s));
    TCR_CHECK(recs.alloc_owned(sizeof(uint64_t) * R_bound, s));
    TCR_CUDA(cudaMemsetAsync(pcnt.as<void>(), 0, sizeof(int32_t) * P, s));
    const int64_t* d_F = reinterpret_cast<const int64_t*>(d_fresh);
    k_records<false><<<grid_for(m), kThreads, 0, s>>>(ucanon.as<Canon>() + U0, flen.as<uint8_t>(), d_F, m,
                                                      (uint32_t)P, pcnt.as<int32_t>(), nullptr, nullptr, (uint32_t)U0);
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(pcnt.as<int32_t>(), pscan.as<int64_t>(), P, s));
    DevBuf pcur;
    TCR_CHECK(pcur.alloc(sizeof(int32_t) * P, s));
    k_ins_part_base<<<grid_for(P + 1), kThreads, 0, s>>>(ix.poff, pscan.as<int64_t>(), P, poff.as<int64_t>(),
                                                         pcur.as<int32_t>());
    TCR_LAUNCH_CHECK();
    {
        DevBuf cuts, shifts, pos;
        TCR_CHECK(growth_cuts<int64_t>(pcnt.as<int32_t>(), ix.poff, poff.as<int64_t>(), P,
                                       std::min<int64_t>(P, m + q.lensum), cuts, shifts, pos, s));
        TCR_CHECK(shifted_copy<uint64_t>(ix.recs, recs.as<uint64_t>(), R0, cuts, shifts, pos.as<int64_t>() + P, s,
                                         num_sms));
    }
    k_records<true><<<grid_for(m), kThreads, 0, s>>>(ucanon.as<Canon>() + U0, flen.as<uint8_t>(), d_F, m,
                                                     (uint32_t)P, pcur.as<int32_t>(), poff.as<int64_t>(),
                                                     recs.as<uint64_t>(), (uint32_t)U0);
    TCR_LAUNCH_CHECK();
    const int t2 = tm.mark();

    // 3. closed rows of the distinct strings that the new strings take (each
    //    once, by its first new string): their query against the grown index
    DevBuf first, rflag, rpos;
    TCR_CHECK(first.alloc(sizeof(unsigned) * N, s));  // indexed by distinct id (< N)
    TCR_CHECK(rflag.alloc(sizeof(int32_t) * m, s));
    TCR_CHECK(rpos.alloc(sizeof(int64_t) * (m + 1), s));
    TCR_CUDA(cudaMemsetAsync(first.as<void>(), 0xff, sizeof(unsigned) * N, s));
    k_ins_first<<<grid_for(m), kThreads, 0, s>>>(nuid.as<int32_t>(), m, first.as<unsigned>());
    TCR_LAUNCH_CHECK();
    k_ins_rep_flags<<<grid_for(m), kThreads, 0, s>>>(nuid.as<int32_t>(), m, first.as<unsigned>(),
                                                     rflag.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(rflag.as<int32_t>(), rpos.as<int64_t>(), m, s));
    int64_t nrep = 0;
    {
        const void* src[1] = {rpos.as<int64_t>() + m};
        void* dst[1] = {&nrep};
        const size_t bytes[1] = {sizeof(int64_t)};
        TCR_CHECK(read_back(s, 1, src, dst, bytes));
    }
    if (nrep <= 0 || nrep > m) return TCRNET_EDEVICE;
    Packed qr;  // the representatives' strings, input order
    qr.n = nrep;
    DevBuf rep_u, ridx, nm_cnt, nm_off, nm_cur, nm_list;
    TCR_CHECK(qr.canon_in.alloc(sizeof(Canon) * nrep, s));
    TCR_CHECK(qr.lens.alloc(nrep, s));
    TCR_CHECK(rep_u.alloc(sizeof(int32_t) * nrep, s));
    TCR_CHECK(ridx.alloc(sizeof(int32_t) * N, s));
    TCR_CHECK(nm_cnt.alloc(sizeof(int32_t) * nrep, s));
    TCR_CHECK(nm_off.alloc(sizeof(int64_t) * (nrep + 1), s));
    TCR_CHECK(nm_cur.alloc(sizeof(int32_t) * nrep, s));
    TCR_CHECK(nm_list.alloc(sizeof(int32_t) * m, s));
    k_ins_reps<<<grid_for(m), kThreads, 0, s>>>(nuid.as<int32_t>(), m, first.as<unsigned>(), rpos.as<int64_t>(),
                                                q.canon_in.as<Canon>(), q.lens.as<uint8_t>(), qr.canon_in.as<Canon>(),
                                                qr.lens.as<uint8_t>(), rep_u.as<int32_t>(), ridx.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CUDA(cudaMemsetAsync(nm_cnt.as<void>(), 0, sizeof(int32_t) * nrep, s));
    TCR_CUDA(cudaMemsetAsync(nm_cur.as<void>(), 0, sizeof(int32_t) * nrep, s));
    k_ins_new_members<<<grid_for(m), kThreads, 0, s>>>(nuid.as<int32_t>(), m, ridx.as<int32_t>(), nullptr, nullptr,
                                                       nullptr, nm_cnt.as<int32_t>(), false);
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(nm_cnt.as<int32_t>(), nm_off.as<int64_t>(), nrep, s));
    k_ins_new_members<<<grid_for(m), kThreads, 0, s>>>(nuid.as<int32_t>(), m, ridx.as<int32_t>(),
                                                       nm_off.as<int64_t>(), nm_cur.as<int32_t>(),
                                                       nm_list.as<int32_t>(), nullptr, true);
    TCR_LAUNCH_CHECK();
    DeletionIndex gx;  // a view of the grown index (not owned)
    gx.ucanon = ucanon.as<Canon>();
    gx.umult = umult.as<int32_t>();
    gx.mem_off = mem_off.as<int64_t>();
    gx.members = members.as<int32_t>();
    gx.recs = recs.as<uint64_t>();
    gx.poff = poff.as<int64_t>();
    gx.P = P;
    gx.n = N;
    DevBuf roff, rcols, rcnt;  // closed rows: every member of every neighbour, the string's own included
    int64_t nr = 0;
    TCR_CHECK(deletion_query(gx, qr, T, roff, rcols, rcnt, &nr, s, num_sms));
    const int t3 = tm.mark();

    // 4. edges between distinct strings: the resident ones, then those of the
    //    fresh strings
    const int64_t E_cap = E0 + nr;
    DevBuf uedges;
    TCR_CHECK(uedges.alloc_owned(sizeof(int2) * (E_cap > 0 ? E_cap : 1), s));
    if (E0 > 0)
        TCR_CUDA(cudaMemcpyAsync(uedges.as<void>(), ix.uedges, sizeof(int2) * E0, cudaMemcpyDeviceToDevice, s));
    const unsigned rgrid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ceil_div(nr, kRowChunk), kWarps), (int64_t)num_sms * 16));
    k_ins_edges<<<rgrid, kThreads, 0, s>>>(roff.as<int64_t>(), rcols.as<int32_t>(), nrep, nr, rep_u.as<int32_t>(),
                                           uid.as<int32_t>(), mem_off.as<int64_t>(), members.as<int32_t>(), U0,
                                           uedges.as<int2>() + E0, d_ecur, E_cap - E0, d_err + 1);
    TCR_LAUNCH_CHECK();
    const int t4 = tm.mark();

    // 5. the grown CSR: old rows gain the tails of their strings, new rows are
    //    the closed rows of their strings without themselves
    DevBuf dcnt, dtoff, dcur, dtcols, delta, deg, off64, toff, cols;
    TCR_CHECK(dcnt.alloc(sizeof(int32_t) * U0, s));
    TCR_CHECK(dtoff.alloc(sizeof(int64_t) * (U0 + 1), s));
    TCR_CHECK(dcur.alloc(sizeof(int32_t) * U0, s));
    TCR_CHECK(delta.alloc(sizeof(int32_t) * n0, s));
    TCR_CHECK(toff.alloc(sizeof(int64_t) * (n0 + 1), s));
    TCR_CHECK(deg.alloc_owned(sizeof(int32_t) * N, s));
    TCR_CHECK(off64.alloc_owned(sizeof(int64_t) * (N + 1), s));
    TCR_CUDA(cudaMemsetAsync(dcnt.as<void>(), 0, sizeof(int32_t) * U0, s));
    TCR_CUDA(cudaMemsetAsync(dcur.as<void>(), 0, sizeof(int32_t) * U0, s));
    k_ins_tail_count<<<rgrid, kThreads, 0, s>>>(roff.as<int64_t>(), rcols.as<int32_t>(), nrep, nr, nm_cnt.as<int32_t>(),
                                                n0, uid.as<int32_t>(), ix.mem_off, ix.members, dcnt.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(dcnt.as<int32_t>(), dtoff.as<int64_t>(), U0, s));
    k_ins_degree<<<grid_for(N), kThreads, 0, s>>>(g.degree, dcnt.as<int32_t>(), uid.as<int32_t>(), n0,
                                                  nuid.as<int32_t>(), ridx.as<int32_t>(), rcnt.as<int32_t>(), m,
                                                  delta.as<int32_t>(), deg.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(delta.as<int32_t>(), toff.as<int64_t>(), n0, s));
    TCR_CHECK(scan_exclusive_i32_to_i64(deg.as<int32_t>(), off64.as<int64_t>(), N, s));
    int64_t sizes[3] = {0, 0, 0};  // new entries of old rows, entries of the grown network, tail entries
    {
        const void* src[3] = {toff.as<int64_t>() + n0, off64.as<int64_t>() + N, dtoff.as<int64_t>() + U0};
        void* dst[3] = {&sizes[0], &sizes[1], &sizes[2]};
        const size_t bytes[3] = {sizeof(int64_t), sizeof(int64_t), sizeof(int64_t)};
        TCR_CHECK(read_back(s, 3, src, dst, bytes));
    }
    const int64_t n_tail = sizes[0], nnz = sizes[1], n_dtail = sizes[2];
    if (n_tail < 0 || n_dtail < 0 || nnz < g.nnz + n_tail) return TCRNET_EDEVICE;
    TCR_CHECK(dtcols.alloc(sizeof(int32_t) * (n_dtail > 0 ? n_dtail : 1), s));
    TCR_CHECK(cols.alloc_owned(sizeof(int32_t) * nnz, s));
    if (n_dtail > 0) {
        k_ins_tails<<<rgrid, kThreads, 0, s>>>(roff.as<int64_t>(), rcols.as<int32_t>(), nrep, nr, nm_off.as<int64_t>(),
                                               nm_list.as<int32_t>(), n0, uid.as<int32_t>(), ix.mem_off, ix.members,
                                               dtoff.as<int64_t>(), dcur.as<int32_t>(), dtcols.as<int32_t>());
        TCR_LAUNCH_CHECK();
        TCR_CHECK(sort_rows(dtoff.as<int64_t>(), dtcols.as<int32_t>(), U0, s, num_sms));
    }
    const int t5 = tm.mark();
    if (g.off64)
        TCR_CHECK(csr_merge<int64_t>(g, static_cast<const int64_t*>(g.offsets), delta.as<int32_t>(), n_tail,
                                     off64.as<int64_t>(), uid.as<int32_t>(), dcnt.as<int32_t>(),
                                     dtoff.as<int64_t>(), dtcols.as<int32_t>(), roff.as<int64_t>(),
                                     rcols.as<int32_t>(), nuid.as<int32_t>(), ridx.as<int32_t>(), m,
                                     cols.as<int32_t>(), s, num_sms));
    else
        TCR_CHECK(csr_merge<int32_t>(g, static_cast<const int32_t*>(g.offsets), delta.as<int32_t>(), n_tail,
                                     off64.as<int64_t>(), uid.as<int32_t>(), dcnt.as<int32_t>(),
                                     dtoff.as<int64_t>(), dtcols.as<int32_t>(), roff.as<int64_t>(),
                                     rcols.as<int32_t>(), nuid.as<int32_t>(), ridx.as<int32_t>(), m,
                                     cols.as<int32_t>(), s, num_sms));
    const int t6 = tm.mark();

    // 6. sizes and error flags
    unsigned long long h_cnt[2] = {0, 0};
    int h_err[2] = {0, 0};
    int64_t h_R = 0, h_nnz = 0;
    {
        const void* src[4] = {d_fresh, d_err, poff.as<int64_t>() + P, off64.as<int64_t>() + N};
        void* dst[4] = {h_cnt, h_err, &h_R, &h_nnz};
        const size_t bytes[4] = {sizeof(h_cnt), sizeof(h_err), sizeof(int64_t), sizeof(int64_t)};
        TCR_CHECK(read_back(s, 4, src, dst, bytes));
    }
    if (h_err[0] || h_err[1] || h_nnz != nnz || h_R > R_bound) return TCRNET_EDEVICE;

    out.off64 = std::move(off64);
    out.cols = std::move(cols);
    out.degree = std::move(deg);
    out.nnz = nnz;
    out.fresh = (int64_t)h_cnt[0];
    out.new_edges = (int64_t)h_cnt[1];
    out.index.ucanon = static_cast<Canon*>(ucanon.release());
    out.index.umult = static_cast<int32_t*>(umult.release());
    out.index.mem_off = static_cast<int64_t*>(mem_off.release());
    out.index.members = static_cast<int32_t*>(members.release());
    out.index.recs = static_cast<uint64_t*>(recs.release());
    out.index.poff = static_cast<int64_t*>(poff.release());
    out.index.uid = static_cast<int32_t*>(uid.release());
    out.index.uedges = static_cast<int2*>(uedges.release());
    out.index.U = U0 + out.fresh;
    out.index.P = P;
    out.index.R = h_R;
    out.index.n = N;
    out.index.E = E0 + out.new_edges;
    out.ms_phase[0] = tm.ms(t0, t1);  // distinct ids, multiplicities, member lists
    out.ms_phase[1] = tm.ms(t1, t2);  // records
    out.ms_phase[2] = tm.ms(t2, t3);  // closed rows (query of the represented strings)
    out.ms_phase[3] = tm.ms(t3, t4);  // edges between distinct strings
    out.ms_phase[4] = tm.ms(t4, t5);  // degrees, offsets, tail lists
    out.ms_phase[5] = tm.ms(t5, t6);  // grown CSR (shifted copy, tails, new rows)
    out.ms_phase[6] = 0.0;
    out.ms_phase[7] = tm.ms(t0, t6);
    return TCRNET_OK;
}

}  // namespace tcr
