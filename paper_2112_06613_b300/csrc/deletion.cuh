// Deletion-neighbourhood method (the network of Methods "TCR network" without testing
// all pairs): declarations.
#pragma once

#include "kernels.cuh"

namespace tcr {

// AUTO picks the deletion method from this many strings on (l_max <= 1), and
// for l_max = 2 from kAutoDeletion2MinN on.
constexpr int64_t kAutoDeletionMinN = 2048;
constexpr int64_t kAutoDeletion2MinN = 2560;

// Largest input the deletion records can address (distinct-string ids use 25 bits).
constexpr int64_t kDeletionMaxN = TCRNET_DELETION_MAX_N;
static_assert(kDeletionMaxN == (1LL << 25), "record ids are 25 bits");

// Resident query index of a deletion build (device pointers; owned by the
// handle, freed with cudaFree): distinct strings, their multiplicities and
// member lists, and the hash-partitioned records.
struct DeletionIndex {
    Canon* ucanon = nullptr;
    int32_t* umult = nullptr;
    int64_t* mem_off = nullptr;
    int32_t* members = nullptr;
    uint64_t* recs = nullptr;
    int64_t* poff = nullptr;
    int32_t* uid = nullptr;    // node -> distinct string
    int2* uedges = nullptr;    // edges between distinct strings, each once
    int64_t U = 0, P = 0, n = 0, E = 0;
    int64_t R = 0;             // records (poff[P])
    // bits of the 32-bit content hash the records keep (all but in a testing
    // build, whose records then serve no queries or merged inserts)
    uint32_t hmask = 0xffffffffu;
    bool valid() const { return recs != nullptr && hmask == 0xffffffffu; }
};

struct DeletionResult {
    DevBuf off64;   // int64[n + 1]
    DevBuf off32;   // int32[n + 1] when nnz < 2^31 and int32 offsets were not refused
    DevBuf cols;    // int32[nnz]
    DevBuf degree;  // int32[n]
    int64_t nnz = 0;
    int64_t n_unique = 0;
    int64_t n_records = 0;
    int64_t unique_edges = 0;
    int64_t candidates = 0;    // l_max = 2: distinct-string pairs sharing a variant (before deduplication)
    int64_t n_fallback = 0;    // partitions over the warp capacity, joined by the quadratic pass
    int64_t closed_total = 0;  // sum over distinct strings of closed-neighbourhood sizes
    int two_pass_join = 0;     // 1 when the edges overflowed the one-pass buffer
    int64_t rejected = 0;      // candidate pairs the confirmation rejected (hash collisions)
    int64_t bad_index = -1;    // input index of an encoder error found by the build (see pk.flags)
    double ms_join = 0, ms_scan = 0, ms_fill = 0, ms_sort = 0;
    // dedup, records, join count, join write, closed fill, closed sort, expand, total
    double ms_phase[8] = {0};
    DeletionIndex index;  // filled when the build keeps its index
};

// Network of the packed strings at l_max = T (0, 1 or 2; ENOTSUP above). Test
// knob: partitions larger than `partition_cap` (<= the shared-memory capacity;
// 0 = default) take the quadratic pass of the l_max = 1 join. The query
// index is kept (keep_index) for l_max = 1 builds. If the encoder's error word
// (pk.flags) was not checked by the packing, the build checks it at its first
// readback and returns the input error with out.bad_index; until then its
// record kernels do nothing when the records counted exceed the n +
// pk.lensum they were sized for (possible only for invalid input).
tcrnet_status deletion_build(const Packed& pk, int T, DeletionResult& out, cudaStream_t s, int num_sms,
                             bool profile, int partition_cap = 0, bool keep_index = false,
                             int partition_target = 0, bool force_off64 = false, int record_hash_bits = 32);

// Neighbour lists (l_max = T) of packed query strings against a resident
// index: CSR with int64 offsets (m + 1), columns, per-query counts.
tcrnet_status deletion_query(const DeletionIndex& ix, const Packed& q, int T, DevBuf& off64, DevBuf& cols,
                             DevBuf& count, int64_t* nnz, cudaStream_t s, int num_sms);

// A resident network (device views of a handle's CSR).
struct CsrView {
    const void* offsets = nullptr;  // int32 or int64 [n + 1]
    bool off64 = false;
    const int32_t* cols = nullptr;  // [nnz], rows ascending
    const int32_t* degree = nullptr;
    int64_t n = 0, nnz = 0;
};

struct InsertResult {
    DevBuf off64;   // int64[N + 1]
    DevBuf cols;    // int32[nnz]
    DevBuf degree;  // int32[N]
    int64_t nnz = 0;
    int64_t fresh = 0;      // new distinct strings
    int64_t new_edges = 0;  // new edges between distinct strings
    DeletionIndex index;    // index of the grown repertoire; the caller owns it
    // with profiling: ids and members, records, query, distinct edges,
    // degrees and tails, grown CSR, unused, total (ms)
    double ms_phase[8] = {0};
};

// Network and index of a deletion build's repertoire (ix, g: n0 strings,
// l_max = T >= 1) grown by the m strings of q (input order, not bucketed), as
// nodes n0 .. n0+m-1, merged instead of rebuilt: the index gains the new
// distinct strings and their records in the same partitions; the new strings'
// query against the grown index gives their rows (without themselves); old
// rows gain the new neighbours at their ends. ix and g are only read. The CSR
// equals that of a fresh build of the concatenation.
tcrnet_status deletion_insert(const DeletionIndex& ix, const CsrView& g, const Packed& q, int T, InsertResult& out,
                              cudaStream_t s, int num_sms, bool profile = false);

}  // namespace tcr
