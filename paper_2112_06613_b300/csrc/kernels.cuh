// Host-side launchers of the tcrnet kernels (one translation unit per family).
#pragma once

#include "common.cuh"

namespace tcr {

// ---- scan.cu --------------------------------------------------------------
// out[i] = sum_{k<i} in[k] for i in [0, n] (n + 1 outputs, out[n] = total).
// zeroed_status: optional caller-provided status words, scan_status_words(n)
// of them, all zero when the scan runs (a caller with several scans clears
// them together; nullptr: the scan clears its own). clear_input: the scan
// sets in[0 .. n) to zero behind itself (in place of a memset before the
// input's next use as counters).
int64_t scan_status_words(int64_t n);
tcrnet_status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                                        unsigned long long* zeroed_status = nullptr, bool clear_input = false);
// The same scan, and in[i] = out[i] behind itself: the counts become cursors at
// the segments' starts, for slot atomics that return absolute positions
// (callers guarantee out[n] < 2^31).
tcrnet_status scan_exclusive_i32_to_i64_cursors(int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                                                unsigned long long* zeroed_status = nullptr);
tcrnet_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// int64 offsets -> int32 offsets (caller checked that they fit).
tcrnet_status narrow_offsets(const int64_t* in, int32_t* out, int64_t count, cudaStream_t s);
// degree[i] = off[i+1] - off[i]
tcrnet_status degree_from_offsets(const int64_t* off, int32_t* degree, int64_t n, cudaStream_t s);

// ---- pack.cu --------------------------------------------------------------
// Validated, encoded, length-bucketed strings.
struct Packed {
    int64_t n = 0;
    DevBuf canon;    // Canon[n], bucket order (length ascending, input order within a length)
    DevBuf perm;     // int32[n], bucket position -> input index
    DevBuf lens;     // uint8[n], input order
    DevBuf canon_in; // Canon[n], input order
    int64_t bucket_off[kMaxLen + 2] = {0};  // bucket L = [bucket_off[L], bucket_off[L+1])
    int64_t lensum = 0;                     // total length of the strings
    DevBuf flags;  // device words of the encoder: [0] first error (~(index << 8 | status), 0: none), [1] total length
};
// Status of the encoder's error word (read back to the host): TCRNET_OK, or
// the error with *bad_index set to the lowest offending input index.
tcrnet_status pack_flags_status(unsigned long long first_error, int64_t* bad_index);
// Encodes chars/offsets (device memory) into `out`. On a bad input returns the
// status and sets *bad_index to the lowest offending input index. With
// bucket = false only the input-order copy is made (no bucketed copy,
// bucket_off left zero); keep_input_order allocates that copy for a handle to
// keep (outside the call's workspace). Strings must lie in byte offsets
// [lo, hi) of d_chars (TCRNET_EINVAL with the index otherwise; offsets that
// decrease give an empty or negative length and fail the same way).
// defer_check (only with bucket = false): return right after the encoder is
// launched, without waiting for it; out.lensum is left at -1 and the caller
// sets it (the byte span of the strings, exact for valid input), then reads
// out.flags at its next synchronisation and reports pack_flags_status.
tcrnet_status pack_strings(const uint8_t* d_chars, const int64_t* d_offsets, int64_t n, Packed& out,
                           int64_t* bad_index, cudaStream_t s, bool bucket = true, bool keep_input_order = false,
                           int64_t lo = INT64_MIN, int64_t hi = INT64_MAX, bool defer_check = false);

// Write repertoire numbers into the spare bits of input-order canon
// (repertoire r = strings rep_off[r] .. rep_off[r+1]).
tcrnet_status tag_repertoires(Canon* canon, int64_t n, const int64_t* rep_off_host, int64_t nrep, cudaStream_t s);
// Bucket already encoded strings (out.canon_in, out.lens, out.n set).
tcrnet_status bucket_strings(Packed& out, cudaStream_t s);
// Bucketed copy (out.canon, out.perm, out.bucket_off) of input-order strings
// owned elsewhere.
tcrnet_status bucket_from(const Canon* canon_in, const uint8_t* lens, int64_t n, Packed& out, cudaStream_t s);
// Inverse of the bucketing: input-order canon and lengths from bucket order.
tcrnet_status unbucket_strings(const Canon* canon, const int32_t* perm, const int64_t* bucket_off_host, int64_t n,
                               Canon* canon_in, uint8_t* lens, cudaStream_t s);

// ---- tile.cu --------------------------------------------------------------
struct TileSide {
    const Canon* canon;  // bucket order
    const int32_t* id;   // bucket position -> output id
    const int64_t* bucket_off;  // host copy, kMaxLen + 2 entries
};
// Hits of a count pass, kept so that the write pass can be skipped: each hit
// (row id, column id) goes to pairs[slot], slot from one warp-level atomic on
// *cursor; slots at or above cap are not written (the caller then runs the
// write pass instead).
struct PairSink {
    int2* pairs = nullptr;
    unsigned long long* cursor = nullptr;
    int64_t cap = 0;
};
// Rows of the hits (both directions when sym) at slots from per-row cursors,
// then the caller sorts the rows. Errors (a row fuller than its count) set *err.
tcrnet_status scatter_pairs(const int2* pairs, int64_t npairs, bool sym, const int64_t* off, int32_t* cursor,
                            int32_t* cols_out, int* err, cudaStream_t s);
// Count (write == false) or write (write == true) every adjacent pair.
//  graph mode (rows == cols, sym == true): tests (L, L) upper triangles and
//   (L, L+1) rectangles; count[] gets both endpoints, writes go both ways.
//  query mode (sym == false): rows are queries, cols the resident repertoire;
//   tests (Lq, Lq - 1), (Lq, Lq), (Lq, Lq + 1); only query rows are counted/written.
// Returns the number of candidate pairs tested in *pairs.
tcrnet_status tile_pass(const TileSide& rows, const TileSide& cols, bool sym, int threshold, bool write,
                        int32_t* count, const int64_t* off, int32_t* cursor, int32_t* cols_out,
                        int64_t* pairs, cudaStream_t s, int num_sms, const PairSink* sink = nullptr);

// ---- dp.cu ----------------------------------------------------------------
// Same contract as tile_pass for l_max >= 2 (bit-parallel Levenshtein distance).
tcrnet_status dp_pass(const TileSide& rows, const TileSide& cols, bool sym, int threshold, bool write,
                      int32_t* count, const int64_t* off, int32_t* cursor, int32_t* cols_out, int64_t* pairs,
                      cudaStream_t s, int num_sms, const PairSink* sink = nullptr);

// ---- analytics.cu ---------------------------------------------------------
// Connected components of the CSR restricted to keep[i] != 0 (keep may be null):
// labels[i] = smallest node id of the component, -1 for removed nodes.
// link_attempts bounds the link attempts of each edge (<= 0: the default
// bound); TCRNET_ETIMEOUT when an edge ran out of them.
tcrnet_status components(const void* off, bool off64, const int32_t* cols, int64_t n, const uint8_t* keep,
                         int32_t* labels, int64_t* n_components, int64_t* largest, cudaStream_t s, int num_sms,
                         int link_attempts = 0);
// knn[i] = mean degree of i's neighbours (0 for isolated nodes).
tcrnet_status degree_histogram(const int32_t* deg, int64_t n, int64_t* hist, int64_t nbins, int64_t* max_degree,
                               cudaStream_t s, int num_sms);
// The same analyses on the graph of distinct strings of a deletion build
// (uid: node -> string, edges: each pair of adjacent strings once, umult:
// members per string); identical results, work ~ U + E instead of nnz.
tcrnet_status components_distinct(const int32_t* uid, int64_t n, const int2* edges, int64_t E, int64_t U,
                                  const uint8_t* keep, int32_t* labels, int64_t* n_components, int64_t* largest,
                                  cudaStream_t s, int num_sms, int link_attempts = 0);
tcrnet_status neighbor_degree_distinct(const int32_t* uid, int64_t n, const int2* edges, int64_t E,
                                       const int32_t* umult, int64_t U, double* knn, cudaStream_t s, int num_sms);
tcrnet_status neighbor_degree(const void* off, bool off64, const int32_t* cols, int64_t n, double* knn,
                              cudaStream_t s, int num_sms);

// ---- rowsort.cu -----------------------------------------------------------
// Rows of the long sort classes listed by the caller (row ids, counts on the
// device): 65..256, 257..512 and more than 512 values. With them the classes'
// kernels need not wait for the short-row kernel to list them and run beside
// it on the workspace's side streams.
constexpr int64_t kSortWideMin = 65, kSortMidMin = 257, kSortBigMin = 513;
struct SortClasses {
    const int32_t* wide = nullptr;
    const int32_t* mid = nullptr;
    const int32_t* big = nullptr;
    const int* counts = nullptr;  // [0] wide, [1] mid, [2] big
    int* zeroed4 = nullptr;       // four ints, zero at the call (the sort's own counters; nullable)
};
// Sort every row segment cols[off[i] .. off[i+1]) ascending (repeats allowed).
// max_len: an upper bound of the row lengths when the caller knows one (-1:
// unknown; then the kernels of every class run and the host reads back how many
// rows exceed a block's shared memory). pre: the long rows listed in advance
// (nullable).
tcrnet_status sort_rows(const int64_t* off, int32_t* cols, int64_t n, cudaStream_t s, int num_sms,
                        int64_t max_len = -1, const SortClasses* pre = nullptr);

}  // namespace tcr
